"""The serving loop (meb_server_*): continuous batching under a device-memory
budget.

* A mix of requests in flight together (small ones grouped into batch
  launches by several workers, large ones on the multi-block path) gives each
  request exactly the result it gets alone, and the oracle's result within
  the solve tolerances.
* Admission never lets the admitted requests' footprint exceed the budget; a
  request larger than the budget is refused at submission.
* Poisson arrivals at 2,000 requests/s complete with their latencies recorded.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu


def pool(n, seed, cap_m=20_000):
    inst = [workloads.ragged_instance(k, seed) for k in range(n)]
    return [(np.ascontiguousarray(C[:cap_m]), np.ascontiguousarray(R[:cap_m])) for C, R in inst]


def test_results_same_alone_and_in_the_mix():
    inst = pool(40, 123)
    inst.append(workloads.cube(60_000, 40, 3, 0.05))       # the multi-block path (m*d >= large_balls)
    inst.append(workloads.gaussian(30_000, 16, 4, 0.1))
    sv = meb.Server(budget_bytes=8 << 30, small_workers=3, large_workers=1, large_balls=400_000,
                    max_group=16)
    tickets = [sv.submit(C, R) for C, R in inst]
    mix = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(inst) and st["failed"] == 0
    assert st["launches"] >= 3                                 # several groups overlapped
    for k, (C, R) in enumerate(inst):
        g = mix[k]
        assert g["rc"] == 0 and g["status"] == 0
        if C.shape[0] * C.shape[1] >= 400_000:
            alone = meb.solve(C, R)
        else:
            alone = meb.solve_batch([(C, R)])[0]
        assert g["r"] == alone["r"], k
        assert np.array_equal(g["c"], alone["c"]), k
        assert np.array_equal(g["active"], alone["active"]), k
    for k in (0, 5, 40, 41):
        C, R = inst[k]
        o = oracle.solve(C, R, tol=1e-12)
        assert abs(mix[k]["r"] - o["r"]) <= 1e-8 * o["r"]
        assert np.linalg.norm(mix[k]["c"] - o["c"]) <= 1e-7 * o["r"]


def test_server_flags_same_results():
    """Spinning waits and the device's default pool change how the workers
    wait and allocate, not what they compute."""
    inst = pool(12, 321)
    ref = meb.solve_batch(inst)
    for kw in (dict(spin_waits=True), dict(device_pool=True), dict(spin_waits=True, device_pool=True)):
        sv = meb.Server(budget_bytes=4 << 30, small_workers=4, max_group=2, **kw)
        res = [sv.wait(t) for t in [sv.submit(C, R) for C, R in inst]]
        sv.close()
        for g, a in zip(res, ref):
            assert g["rc"] == 0 and g["r"] == a["r"] and np.array_equal(g["c"], a["c"]), kw


def test_two_servers_share_streams_and_pool():
    """Servers of one process share their workers' streams and memory pool:
    two alive at once, and one after another, still give every request its
    result alone."""
    inst = pool(10, 555)
    ref = meb.solve_batch(inst)
    a = meb.Server(budget_bytes=4 << 30, small_workers=3, max_group=2)
    b = meb.Server(budget_bytes=2 << 30, small_workers=5, max_group=4)
    ta = [a.submit(C, R) for C, R in inst]
    tb = [b.submit(C, R) for C, R in inst]
    ra = [a.wait(t) for t in ta]
    rb = [b.wait(t) for t in tb]
    a.close()
    b.close()
    c = meb.Server(budget_bytes=4 << 30)
    rc = [c.wait(t) for t in [c.submit(C, R) for C, R in inst]]
    c.close()
    for res in (ra, rb, rc):
        for g, r in zip(res, ref):
            assert g["rc"] == 0 and g["r"] == r["r"] and np.array_equal(g["c"], r["c"])


def test_budget_admission():
    inst = pool(30, 7)
    fps = [meb.footprint(C.shape[0], C.shape[1], True) + 8 * C.size + 8 * len(R) for C, R in inst]
    budget = int(3 * max(fps))                                  # a few requests at a time
    sv = meb.Server(budget_bytes=budget, small_workers=2)
    with pytest.raises(meb.MebError) as e:
        big = workloads.cube(400_000, 256, 1, 0.05)            # alone larger than the budget
        sv.submit(*big)
    assert e.value.code == -2
    tickets = [sv.submit(C, R) for C, R in inst]
    res = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.close()
    bad = [(k, r["rc"], r["status"], r["outer_iters"]) for k, r in enumerate(res) if r["rc"] != 0]
    assert not bad, bad
    assert st["completed"] == len(inst)
    assert 0 < st["peak_bytes"] <= budget
    ref = meb.solve_batch(inst)
    for a, b in zip(res, ref):
        assert a["r"] == b["r"] and np.array_equal(a["c"], b["c"])


def test_poisson_stream_latencies():
    inst = pool(64, 99, cap_m=30_000)
    big = [workloads.cube(300_000, 128, 5, 0.05)]
    t_arr, pick = workloads.poisson_arrivals(2000.0, 0.5, len(inst), 1005, 0.01, len(big))
    assert 800 < len(t_arr) < 1200
    sv = meb.Server(budget_bytes=80 << 30, large_balls=1 << 24)
    tickets = [None] * len(t_arr)

    def producer():
        t0 = time.perf_counter()
        for k, (ta, p) in enumerate(zip(t_arr, pick)):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0002)
            C, R = big[-1 - p] if p < 0 else inst[p]
            tickets[k] = sv.submit(C, R, active_cap=64)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    res = [sv.wait(t) for t in tickets]
    sv.close()
    lat = np.array([r["latency_s"] for r in res])
    bad = [(k, r["rc"], r["status"]) for k, r in enumerate(res) if r["rc"] != 0]
    assert not bad, bad
    assert np.all(lat > 0) and np.percentile(lat, 50) < 5.0
    # spot-check results against the batch solver alone
    ref = meb.solve_batch([inst[p] for p in pick[:20] if p >= 0])
    got = [r for r, p in zip(res[:20], pick[:20]) if p >= 0]
    for a, b in zip(got, ref):
        assert a["r"] == b["r"] and np.array_equal(a["c"], b["c"])
