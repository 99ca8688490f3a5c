#!/usr/bin/env python
"""Benchmark: MEB solves/s of the ripALM hot path on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cube_m2e6_d100] [--no-extra] [--no-cpu-baseline]

A step is one full solve (Algorithm 1 with Algorithm 2, then the
feasibility pass of Sec. 4.2) of the workload's synthetic instance:
m = 2,000,000 balls in d = 100, centres U[-1,1]^d, radii U[0,0.05]
(seed 1002).  Inputs (1.6 GB) are resident in HBM and larger than L2, so no
flush is needed between steps.  Each solve is checked against the stored
oracle radius (tests/golden/<workload>.json, written by the oracle): a solve
counts only if its radius relative error is <= 1e-8.

The same JSON line carries, besides the headline:
  arms       the same workload solved by the plain FP64 ripALM (no shadow:
             every ball of every pass through the FP64 rows), the baseline the
             reduced-precision screens are measured against;
  workloads  the small latency-bound instance (m = 1e4, d = 10: solves/s and
             microseconds per semismooth Newton step); the large
             high-dimensional one (m = 2e5, d = 2000, points on a sphere:
             solves/s, checked against the closed form r* = 1); the ragged
             batch (the first --batch-instances of 4096 independent instances,
             m log-uniform in [100, 1e5], d in {2, 3, 16, 64, 256}) solved by
             one persistent launch; and serving (Poisson arrivals at 2000
             requests/s for --serve-seconds from a pool of such instances plus
             1% with m = 5e5, d = 128, under an 80 GB device budget: solves/s,
             p50/p99 latency);
  roofline   of the screen kernel (the full pass over all balls), from a few
             more solves with CUDA event nodes around every screen (the nodes
             slow a solve by about 6%, so the timed region runs without them);
  cpu_baseline  one full solve of the same instance by the CPU oracle as it
             stands, on all host cores (the count is stated).

Under torchrun (N > 1) every rank solves its own copy of the workload with no
collective on the data path (weak scaling); the timed region is bracketed by
barriers and the max over ranks is used.

--impl reference times the CPU oracle as it stands: each step is one full
solve of the same instance on all host cores, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# the serving workers' streams need hardware queues of their own (read when the
# process first uses CUDA)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MEB solves/s & p50/p99 latency at radius rel.err<=1e-8; per-iter HBM GB/s"
UNIT = "solves/s"
ROOFLINE_SOLVES = 3
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full FP16
# screen per ball, by d, from an ncu capture at m = 1e6 (traffic grows with
# the balls streamed; scaled to a launch by m).  Valid only for the screen
# kernel as captured: empty while the kernel has changed since.
SCREEN_TRAFFIC_PER_BALL: dict = {100: 223.7}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _golden(name):
    try:
        with open(os.path.join(ROOT, "tests", "golden", name + ".json")) as f:
            return json.load(f)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(dist, tot_ms: float, ok: int, device=None):
    """Whole-job throughput over ranks: (sum of correct solves) / (max time).
    Ranks share no data on the path; only these two scalars are reduced."""
    if dist is None:
        return ok / (tot_ms / 1e3), tot_ms, ok
    import torch
    t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
    n = torch.tensor([ok], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n.item()) / (float(t.item()) / 1e3), float(t.item()), int(n.item())


def oracle_full_solve(C, R):
    """The CPU oracle as it stands: one full solve on all host cores (its
    results do not depend on the thread count).  Returns (seconds, threads, r)."""
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    t = time.perf_counter()
    res = oracle.solve(C, R, tol=1e-10)
    return time.perf_counter() - t, threads, res["r"]


def run_reference(args, C, R, m, rank):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_full_solve(C, R)
    times = []
    threads = 1
    for _ in range(args.steps):
        dt, threads, r = oracle_full_solve(C, R)
        times.append(dt)
    tot = sum(times)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "d": int(C.shape[1]), "tol": 1e-10},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"each step one full oracle solve of all {m} balls "
                                   f"(tol 1e-10) on {threads} host threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# the contexts' tick loop (--tick-loop): "graph" (default), or "host" for
# profiling the matrix-free path kernel by kernel (a profiler does not see the
# kernels of a graph with conditional nodes)
TICK_LOOP = "graph"


def new_ctx(meb, local, stream):
    return meb.Context(local, stream.cuda_stream, tick_loop=TICK_LOOP)


def timed_solves(meb, torch, ctx, dC, dR, steps, warmup, stream):
    """Warm-up, then `steps` solves each bracketed by CUDA events on the solve
    stream; returns (per-solve ms, the last result, radii)."""
    for _ in range(warmup):
        meb.solve(dC, dR, ctx=ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    radii = []
    res = None
    torch.cuda.synchronize()
    for k in range(steps):
        ev[k][0].record(stream)
        res = meb.solve(dC, dR, ctx=ctx)
        ev[k][1].record(stream)
        radii.append(res["r"])
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], res, radii


def extra_workloads(meb, torch, local, stream, workloads, sphere_only=False):
    """The small latency-bound instance and the large high-dimensional one."""
    out = {}
    if sphere_only:
        return sphere_workload(meb, torch, local, stream, workloads, out)
    # m = 1e4, d = 10 (gaussian, seed 1001): stored oracle radius
    C, R = workloads.workload("gaussian_m1e4_d10")
    gold = _golden("gaussian_m1e4_d10")
    r_ref = gold["r"] if gold and gold.get("input_sha256") == workloads.digest(C, R) else None
    ctx = new_ctx(meb, local, stream)
    dC, dR = torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda()
    lat, res, radii = timed_solves(meb, torch, ctx, dC, dR, 30, 5, stream)
    rel = [abs(r - r_ref) / r_ref for r in radii] if r_ref else None
    ok = sum(e <= 1e-8 for e in rel) if rel else len(lat)
    out["gaussian_m1e4_d10"] = {
        "value": ok / (sum(lat) / 1e3), "unit": UNIT, "steps": len(lat),
        "p50_ms": statistics.median(lat), "p99_ms": float(np.percentile(lat, 99)),
        "us_per_ssn_step": 1e3 * statistics.median(lat) / max(res["ssn_iters"], 1),
        "ssn_per_solve": res["ssn_iters"], "passes_per_solve": res["passes"],
        "max_relerr": max(rel) if rel else None, "reference": "stored oracle radius",
        "bound": "latency (working set 0.9 MB, L2-resident)"}
    del dC, dR
    return sphere_workload(meb, torch, local, stream, workloads, out)


def sphere_workload(meb, torch, local, stream, workloads, out):
    # m = 2e5, d = 2000 (sphere, seed 1003): closed form r* = 1
    C, R, _ctr = workloads.sphere(200_000, 2000, 1003)
    ctx = new_ctx(meb, local, stream)
    dC, dR = torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda()
    del C
    ctx.reset_stats()
    lat, res, radii = timed_solves(meb, torch, ctx, dC, dR, 3, 1, stream)
    st = ctx.stats()
    # one more solve, driven from the host with per-phase events (a sync per
    # tick: not timed above)
    ctx.set_option("tick_loop", "host")
    ctx.set_profiling(True)
    ctx.reset_stats()
    meb.solve(dC, dR, ctx=ctx)
    torch.cuda.synchronize()
    ph = ctx.stats()["phase_ms"]
    ctx.set_profiling(False)
    ctx.set_option("tick_loop", TICK_LOOP)
    rel = [abs(r - 1.0) for r in radii]
    ok = sum(e <= 1e-8 for e in rel)
    out["sphere_m2e5_d2000"] = {
        "phase_ms_profiled_solve": {"pass": ph[0], "support_rows_control": ph[1],
                                    "newton_cg": ph[2], "multipliers": ph[3]},
        "value": ok / (sum(lat) / 1e3), "unit": UNIT, "steps": len(lat),
        "p50_ms": statistics.median(lat), "max_relerr": max(rel),
        "reference": "closed form r* = 1", "ssn_per_solve": res["ssn_iters"],
        "cg_per_solve": res["cg_iters"], "passes_per_solve": res["passes"],
        "gpu_launches_per_solve": st["kernel_launches"] / 4}
    del dC, dR
    return out


def ragged_batch(meb, torch, local, stream, workloads, n_inst):
    """The ragged batch (m log-uniform in [100, 1e5], d in {2,3,16,64,256}),
    its first n_inst instances resident on the device, solved by one
    meb_solve_batch launch per step after the tuner picked its configuration
    on a sample; aggregate solves/s, per-solve passes and the algorithmic
    bytes of the shadow passes (FP16 rows, bound, radius and slot per ball and
    pass)."""
    t0 = time.perf_counter()
    inst = workloads.ragged(n_inst, 1004)
    gen_s = time.perf_counter() - t0
    dinst = [(torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda()) for C, R in inst]
    balls = sum(C.shape[0] for C, _ in inst)
    in_bytes = sum(C.nbytes + R.nbytes for C, R in inst)
    del inst
    ctx = new_ctx(meb, local, stream)
    table = meb.tune_batch(dinst, per_class=8, ctx=ctx)
    res = meb.solve_batch(dinst, ctx=ctx, allow_notconv=True)  # warm-up
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(3)]
    for a, b in ev:
        a.record(stream)
        res = meb.solve_batch(dinst, ctx=ctx, allow_notconv=True)
        b.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    # a solve counts if it converged and, for the instances with a stored
    # oracle radius, is within 1e-8 of it
    gold = _golden("ragged_sample")
    ref = {g["k"]: g["r"] for g in gold["instances"]} if gold else {}
    rel = {k: abs(res[k]["r"] - r) / r for k, r in ref.items() if k < len(res)}
    ok = sum(1 for k, r in enumerate(res) if r["status"] == 0 and rel.get(k, 0.0) <= 1e-8)
    # algorithmic bytes: every pass streams, per ball, 16*ceil(d/8) + 12 bytes (FP16
    # shadow) or 16*ceil(d/4) + 12 (FP32 shadow, d <= 4 class) -- a lower bound
    # that leaves out the one FP64 read of the setup and the FP64 rows
    passes_bytes = 0
    for (C, _R), r in zip(dinst, res):
        m, d = C.shape
        row = 16 * ((d + 3) // 4) if d <= 4 else 16 * ((d + 7) // 8)
        passes_bytes += r["passes"] * m * (row + 12)
    del dinst
    torch.cuda.empty_cache()
    return {"value": ok / (statistics.median(ms) / 1e3), "unit": UNIT, "instances": n_inst,
            "steps": len(ms), "ms_per_step": statistics.median(ms), "balls": balls,
            "input_gb": in_bytes / 1e9, "generate_s": gen_s,
            "shadow_pass_gb_per_s": passes_bytes / (statistics.median(ms) / 1e3) / 1e9,
            "passes_per_solve": statistics.mean(r["passes"] for r in res),
            "tuned_table": table, "solved_ok": ok,
            "capped": [k for k, r in enumerate(res) if r["status"] != 0],
            "checked_vs_oracle": len(rel), "max_relerr_checked": max(rel.values()) if rel else None,
            "sample": f"the first {n_inst} of the 4096-instance batch (seed 1004)"}


# Table 1 of the paper: balls kept for the FP64 phase of its mixed-precision
# run, on its LCG instances (rows d = 20, 30, 40, 50; columns m = 1e3, 5e3,
# 1e4, 5e4, 1e5).
TABLE1_KEPT = {20: (23, 43, 82, 405, 807), 30: (28, 42, 88, 449, 899),
               40: (45, 77, 155, 780, 1586), 50: (41, 96, 182, 929, 1852)}


def paper_sweep(meb, torch, local, stream):
    """The paper's test instances (its LCG family, Sec. 5): every size of
    Fig. 2 and Fig. 3, solved by the plain path and by the mixed-precision
    pipeline; time per solve (median of 3), the radius relative error against
    the stored oracle radius, and the reduced-set size next to Table 1's kept
    counts (the paper's tol_red is not stated, so these are not expected to
    match)."""
    from paper_2605_31425_gb300 import workloads
    gold = _golden("paper_sweep")
    if not gold:
        return None
    mp = meb.params_default()
    mp.mixed = 1
    ctx = new_ctx(meb, local, stream)
    rows = []
    for g in gold["instances"]:
        m, d = g["m"], g["d"]
        C, R = workloads.lcg(m, d)
        dC, dR = torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda()
        row = {"m": m, "d": d}
        for tag, prm in (("plain", None), ("mixed", mp)):
            try:
                meb.solve(dC, dR, params=prm, ctx=ctx, allow_notconv=True)
                ts = []
                for _ in range(3):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    res = meb.solve(dC, dR, params=prm, ctx=ctx, allow_notconv=True)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
            except meb.MebError as e:   # reported, not hidden
                row[tag + "_error"] = str(e)
                ctx = new_ctx(meb, local, stream)
                continue
            row[tag + "_ms"] = 1e3 * statistics.median(ts)
            row[tag + "_relerr"] = abs(res["r"] - g["r"]) / g["r"]
            row[tag + "_status"] = res["status"]
            if tag == "mixed":
                row["kept"] = res["n_reduced"]
                row["readd_rounds"] = res["readd_rounds"]
        if d in TABLE1_KEPT and m in (1000, 5000, 10_000, 50_000, 100_000):
            row["table1_kept"] = TABLE1_KEPT[d][(1000, 5000, 10_000, 50_000, 100_000).index(m)]
        rows.append(row)
        del dC, dR
    return {"instances": rows,
            "max_relerr_plain": max((r["plain_relerr"] for r in rows if "plain_relerr" in r), default=None),
            "max_relerr_mixed": max((r["mixed_relerr"] for r in rows if "mixed_relerr" in r), default=None),
            "errors": sum(1 for r in rows for k in r if k.endswith("_error"))}


def serving(meb, workloads, seconds, rate=2000.0, n_pool=256, small_workers=0, max_group=0,
            large_balls=0, **server_flags):
    """Poisson arrivals at `rate` requests/s for `seconds`, instances drawn from
    a pool of ragged instances (1% large: m = 5e5, d = 128), under an 80 GB
    device-memory budget; every request's latency from submission to result.
    Host inputs are pinned (torch)."""
    import torch
    pool = [tuple(torch.from_numpy(a).pin_memory() for a in workloads.ragged_instance(k, 1005))
            for k in range(n_pool)]
    big = [tuple(torch.from_numpy(a).pin_memory() for a in workloads.cube(500_000, 128, 1005 + k, 0.05))
           for k in range(2)]
    t_arr, pick = workloads.poisson_arrivals(rate, seconds, n_pool, 1005, 0.01, len(big))
    sv = meb.Server(budget_bytes=80 * 10 ** 9, small_workers=small_workers, max_group=max_group,
                    large_balls=large_balls, **server_flags)
    tickets = [None] * len(t_arr)
    t0 = time.perf_counter()
    for k, (ta, p) in enumerate(zip(t_arr, pick)):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0001)
        C, R = big[-1 - p] if p < 0 else pool[p]
        tickets[k] = sv.submit(C, R, active_cap=256)
    res = [sv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    st = sv.stats()
    sv.close()
    lat = np.array([r["latency_s"] for r in res]) * 1e3
    ok = sum(1 for r in res if r["rc"] == 0)
    small_lat = lat[pick >= 0]
    return {"value": ok / wall, "unit": UNIT, "offered_rate": rate, "requests": len(res),
            "arrival_window_s": seconds, "wall_s": wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "p50_small_ms": float(np.percentile(small_lat, 50)),
            "p99_small_ms": float(np.percentile(small_lat, 99)),
            "large_requests": int(np.sum(pick < 0)), "launches": st["launches"],
            "failed": int(len(res) - ok),
            "peak_device_gb": st["peak_bytes"] / 1e9, "budget_gb": 80,
            "pool": f"{n_pool} ragged instances (seed 1005) + 2 large (m=5e5, d=128), pinned host memory",
            "small_workers": small_workers or "default", "max_group": max_group or "default",
            "large_balls": large_balls or "default"}


def served_e2e(meb, pC, pR, r_ref, n):
    """End to end through the serving API: the pinned bench inputs submitted as
    n independent requests (each copies its 1.6 GB of inputs in and its result
    out); the two large-instance workers overlap one request's copy-in with
    another's solve.  Two requests first, one per worker, build the workers'
    contexts and graphs."""
    sv = meb.Server(budget_bytes=80 * 10 ** 9)
    try:
        for t in [sv.submit(pC, pR, active_cap=256) for _ in range(2)]:
            sv.wait(t)
        t0 = time.perf_counter()
        tickets = [sv.submit(pC, pR, active_cap=256) for _ in range(n)]
        res = [sv.wait(t) for t in tickets]
        wall = time.perf_counter() - t0
    finally:
        sv.close()
    ok = sum(1 for r in res
             if r["rc"] == 0 and (r_ref is None or abs(r["r"] - r_ref) <= 1e-8 * r_ref))
    lat = [r["latency_s"] * 1e3 for r in res]
    return {"value": ok / wall, "unit": UNIT, "requests": n, "ok": ok, "wall_s": wall,
            "p50_latency_ms": statistics.median(lat), "max_latency_ms": max(lat),
            "h2d_bytes_per_step": int(pC.numel() * 8 + pR.numel() * 8),
            "via": "meb_server_submit / meb_server_wait (two large-instance workers), "
                   "all requests submitted at once"}


def serving_in_own_process(seconds, local):
    """The serving line, from a process of its own on the same GPU (one server
    per process is the supported use: a server created in a process whose
    earlier server served requests ran slower); this process's cached device
    memory is released first."""
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "LOCAL_WORLD_SIZE", "GROUP_RANK")}
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    env["CUDA_VISIBLE_DEVICES"] = vis.split(",")[local] if vis else str(local)
    cmd = [sys.executable, os.path.abspath(__file__), "--only", "serving",
           "--serve-seconds", str(seconds)]
    p = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    for ln in reversed(p.stdout.strip().splitlines()):
        if ln.startswith("{"):
            out = json.loads(ln)
            out.pop("only", None)
            out["process"] = "its own (bench.py --only serving)"
            return out
    return {"error": f"exit {p.returncode}: {p.stderr.strip()[-300:]}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube_m2e6_d100")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only (no FP64 arm, no other workloads)")
    ap.add_argument("--batch-instances", type=int, default=4096)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--only", choices=["ragged", "sphere", "serving"], default=None,
                    help="run one extra line alone and print it (for profiling)")
    ap.add_argument("--tick-loop", choices=["graph", "host", "while"], default="graph",
                    help="the contexts' tick loop (host: kernel-by-kernel profiling)")
    args = ap.parse_args()
    global TICK_LOOP
    TICK_LOOP = args.tick_loop
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2605_31425_gb300 import workloads
    C, R = workloads.workload(args.workload)
    m, d = C.shape

    if args.impl == "reference":
        run_reference(args, C, R, m, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2605_31425_gb300 as meb
    stream = torch.cuda.current_stream()
    if args.only:
        if args.only == "ragged":
            out = ragged_batch(meb, torch, local, stream, workloads, args.batch_instances)
        elif args.only == "serving":
            out = serving(meb, workloads, args.serve_seconds)
        else:
            out = extra_workloads(meb, torch, local, stream, workloads,
                                  sphere_only=True)["sphere_m2e5_d2000"]
        print(json.dumps({"only": args.only, **out}), flush=True)
        return
    ctx = new_ctx(meb, local, stream)
    dC = torch.from_numpy(C).cuda()
    dR = torch.from_numpy(R).cuda()
    torch.cuda.synchronize()

    gold = _golden(args.workload)
    r_ref = gold["r"] if gold and gold.get("input_sha256") == workloads.digest(C, R) else None

    for _ in range(args.warmup):
        res = meb.solve(dC, dR, ctx=ctx)

    # timed region: the device-resident tick loop (CUDA graph batches), one
    # CUDA event pair per solve on the solve stream
    ctx.set_profiling(False)
    ctx.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    radii = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            res = meb.solve(dC, dR, ctx=ctx)
            ev[k][1].record(stream)
            radii.append(res["r"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        st_run = ctx.stats()
        # roofline of the dominant kernel, k_screen (the full pass over all
        # balls): the same solves again with CUDA event nodes recorded around
        # every screen inside the graphs
        ctx.set_profiling(True)
        ctx.reset_stats()
        for _ in range(min(args.steps, ROOFLINE_SOLVES)):
            meb.solve(dC, dR, ctx=ctx)
        torch.cuda.synchronize()
        st = ctx.stats()
        ctx.set_profiling(False)
    lat = [a.elapsed_time(b) for a, b in ev]
    relerr = [abs(r - r_ref) / r_ref for r in radii] if r_ref else []
    ok = sum(1 for e in relerr if e <= 1e-8) if r_ref else args.steps
    value, tot_ms, ok_all = aggregate(dist, sum(lat), ok, device="cuda")

    # bytes per launch / mean event-timed duration of the screens
    pass_launches = max(st["pass_launches"], 1)
    avg_ms = st["pass_ms"] / pass_launches
    bytes_per_launch = st["pass_bytes"] // pass_launches
    fp16_screen = bytes_per_launch == m * (16 * ((d + 7) // 8) + 12)
    tpb = SCREEN_TRAFFIC_PER_BALL.get(int(d)) if fp16_screen else None
    traffic = tpb * m if tpb else None
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()

    # end to end: host (pinned) inputs through the public API, result back to host
    pC = torch.from_numpy(C).pin_memory()
    pR = torch.from_numpy(R).pin_memory()
    hctx = new_ctx(meb, local, stream)
    res_h = meb.solve(pC, pR, ctx=hctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_ok = 0
    for _ in range(args.e2e_steps):
        res_h = meb.solve(pC, pR, ctx=hctx)
        if r_ref is None or abs(res_h["r"] - r_ref) <= 1e-8 * r_ref:
            e2e_ok += 1
    e2e_s = time.perf_counter() - t0
    e2e_val = world * e2e_ok / e2e_s if args.e2e_steps > 0 else None
    del hctx
    e2e_served = None
    if args.e2e_steps > 0 and not args.no_extra:
        e2e_served = served_e2e(meb, pC, pR, r_ref, max(2 * args.e2e_steps, 8))
        e2e_served["value"] *= world
    del pC, pR

    arms, extra = None, None
    if not args.no_extra:
        # the plain FP64 ripALM on the same resident inputs
        pctx = meb.Context(local, stream.cuda_stream, screen="fp64")
        plat, pres, pradii = timed_solves(meb, torch, pctx, dC, dR, 3, 1, stream)
        prel = [abs(r - r_ref) / r_ref for r in pradii] if r_ref else []
        pok = sum(e <= 1e-8 for e in prel) if r_ref else len(plat)
        arms = {
            "fp16_certified_screen": {"value": value, "unit": UNIT, "p50_ms": statistics.median(lat),
                                      "note": "the headline: certified FP16 screen + FP64 rows"},
            "fp64_plain": {"value": pok / (sum(plat) / 1e3), "unit": UNIT,
                           "p50_ms": statistics.median(plat), "steps": len(plat),
                           "max_relerr": max(prel) if prel else None,
                           "passes_per_solve": pres["passes"],
                           "fp64_rows_per_pass": pres["fp64_rows"] / max(pres["passes"], 1),
                           "note": "every ball of every pass through the FP64 rows, no shadow"},
        }
        del pctx
        # the mixed-precision reduction pipeline (Sec. 4.2) on the same inputs
        mp = meb.params_default()
        mp.mixed = 1
        mctx = new_ctx(meb, local, stream)
        for _ in range(2):
            meb.solve(dC, dR, params=mp, ctx=mctx)
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(5)]
        mres = []
        for a, b in mev:
            a.record(stream)
            mres.append(meb.solve(dC, dR, params=mp, ctx=mctx))
            b.record(stream)
        torch.cuda.synchronize()
        mlat = [a.elapsed_time(b) for a, b in mev]
        mrel = [abs(r["r"] - r_ref) / r_ref for r in mres] if r_ref else []
        mok = sum(e <= 1e-8 for e in mrel) if r_ref else len(mlat)
        arms["mixed_precision"] = {
            "value": mok / (sum(mlat) / 1e3), "unit": UNIT, "p50_ms": statistics.median(mlat),
            "steps": len(mlat), "max_relerr": max(mrel) if mrel else None,
            "n_reduced": mres[-1]["n_reduced"], "readd_rounds": mres[-1]["readd_rounds"],
            "lowp_passes": mres[-1]["lowp_passes"], "passes_per_solve": mres[-1]["passes"],
            "note": "FP32 ripALM to 1e-2 on all balls, certified screen, FP64 ripALM on the "
                    "reduced set (warm start), full FP64 feasibility pass and re-adds"}
        del mctx
        del dC, dR
        torch.cuda.empty_cache()
        extra = extra_workloads(meb, torch, local, stream, workloads)
        if args.batch_instances > 0:
            extra["ragged_batch"] = ragged_batch(meb, torch, local, stream, workloads,
                                                 args.batch_instances)
        if args.serve_seconds > 0:
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            extra["serving"] = serving_in_own_process(args.serve_seconds, local)
        extra["paper_sweep"] = paper_sweep(meb, torch, local, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, threads, r_cpu = oracle_full_solve(C, R)
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"one full oracle solve of all {m} balls (tol 1e-10, {dt:.2f} s) "
                         f"on {threads} host threads",
               "relerr_vs_stored": abs(r_cpu - r_ref) / r_ref if r_ref else None}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "m": int(m), "d": int(d), "tol": 1e-10,
                       "l2": f"inputs ({C.nbytes / 1e9:.2f} GB FP64, {bytes_per_launch / 1e9:.2f} GB per screen) larger than L2; no flush",
                       "parallelism": f"replicas x{world}"},
            "p50_ms": statistics.median(lat), "p99_ms": float(np.percentile(lat, 99)),
            "max_relerr": max(relerr) if relerr else None, "solves_ok": ok_all,
            "passes_per_solve": res["passes"], "ssn_per_solve": res["ssn_iters"],
            "newton_per_solve": {"inverses": res["newton_inverses"], "fp64": res["newton_fp64"]},
            "fp64_rows_per_pass": res["fp64_rows"] / max(res["passes"], 1),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_screen", "bytes_per_launch": bytes_per_launch,
                         "avg_launch_ms": avg_ms, "launches_timed": st["pass_launches"],
                         "timed_over": f"{min(args.steps, ROOFLINE_SOLVES)} solves after the "
                                       "throughput region, event nodes around each screen",
                         "peak_kind": peak_kind},
            "e2e": {"value": e2e_val, "unit": UNIT,
                    "h2d_bytes_per_step": int(C.nbytes + R.nbytes),
                    "d2h_bytes_per_step": int(8 * d + 8 * res_h["n_active"])},
            "e2e_served": e2e_served,
            "gpu_launches": int(st_run["kernel_launches"]),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "arms": arms,
            "workloads": extra,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
