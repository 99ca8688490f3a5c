"""Write the stored oracle results for the full-size benchmark instances.

Calls only the CPU oracle (oracle/) on inputs from the seeded generators and
writes tests/golden/<workload>.json with the input digest, the oracle's radius,
centre, active set and KKT residuals.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2605_31425_gb300 import workloads  # noqa: E402


# The paper's test instances (Sec. 5): its LCG family at the sizes of Fig. 2
# (d in {20, 30, 40, 50}, m in {1e3, 5e3, 1e4, 5e4, 1e5}) and of Fig. 3
# (d in {1e2, 5e2, 1e3, 5e3, 1e4}, m in {1e3, 5e3}).
PAPER_SWEEP = ([(m, d) for d in (20, 30, 40, 50) for m in (1000, 5000, 10_000, 50_000, 100_000)]
               + [(m, d) for d in (100, 500, 1000, 5000, 10_000) for m in (1000, 5000)])


def paper_sweep():
    """tests/golden/paper_sweep.json: the oracle's radius (tol 1e-12) and
    active-set size for every instance of PAPER_SWEEP."""
    out = []
    for m, d in PAPER_SWEEP:
        C, R = workloads.lcg(m, d)
        t = time.time()
        res = oracle.solve(C, R, tol=1e-12)
        dt = time.time() - t
        out.append(dict(m=m, d=d, input_sha256=workloads.digest(C, R), r=res["r"],
                        n_active=int(len(res["active"])), status=res["status"],
                        passes=res["passes"], oracle_seconds=dt))
        print(m, d, res["r"], res["status"], f"{dt:.1f}s", flush=True)
    with open(os.path.join(HERE, "paper_sweep.json"), "w") as f:
        json.dump(dict(tol=1e-12, note="written by tests/golden/make_golden.py from oracle.solve; "
                       "inputs from paper_2605_31425_gb300.workloads.lcg(m, d)", instances=out),
                  f, indent=1)


def ragged_sample(n=64, seed=1004):
    """tests/golden/ragged_sample.json: the oracle's radius (tol 1e-12) of the
    first n instances of the ragged batch."""
    out = []
    for k in range(n):
        C, R = workloads.ragged_instance(k, seed)
        t = time.time()
        res = oracle.solve(C, R, tol=1e-12)
        out.append(dict(k=k, m=int(C.shape[0]), d=int(C.shape[1]),
                        input_sha256=workloads.digest(C, R), r=res["r"], status=res["status"],
                        oracle_seconds=time.time() - t))
        print(k, C.shape, res["r"], res["status"], flush=True)
    with open(os.path.join(HERE, "ragged_sample.json"), "w") as f:
        json.dump(dict(tol=1e-12, seed=seed, note="written by tests/golden/make_golden.py from "
                       "oracle.solve; inputs from workloads.ragged_instance(k, seed)",
                       instances=out), f, indent=1)


def main(names):
    for name in names:
        if name == "paper_sweep":
            paper_sweep()
            continue
        if name == "ragged_sample":
            ragged_sample()
            continue
        C, R = workloads.workload(name)
        t = time.time()
        res = oracle.solve(C, R, tol=1e-12)
        dt = time.time() - t
        out = dict(
            workload=name, m=int(C.shape[0]), d=int(C.shape[1]),
            input_sha256=workloads.digest(C, R),
            r=res["r"], r_alm=res["r_alm"], c=[float(v) for v in res["c"]],
            active=[int(i) for i in res["active"]], kkt_max=res["kkt_max"],
            status=res["status"], outer_iters=res["outer_iters"], ssn_iters=res["ssn_iters"],
            passes=res["passes"], oracle_seconds=dt, tol=1e-12,
            note="written by tests/golden/make_golden.py from oracle.solve; inputs from "
                 "paper_2605_31425_gb300.workloads.workload(name)",
        )
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, res["r"], res["status"], f"{dt:.1f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["cube_m2e6_d100", "gaussian_m1e4_d10"])
