"""GPU parity: libmeb (through its C ABI) against the CPU oracle.

Tolerances follow from the arithmetic (eps = 2^-52): a sum of n terms taken
in two different orders differs by at most (n + k) eps times the sum of the
magnitudes of its terms, and each per-ball term carries (d + 16) eps of
relative rounding.  Integer outputs (case counts, indices, argmax) are
compared exactly.
"""
import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def rand_state(rng, m, d):
    scale = rng.choice([0.15, 1.0, 3.0], size=m)
    C = rng.standard_normal((m, d)) * scale[:, None] / np.sqrt(max(d, 1) / 4.0)
    R = rng.uniform(0, 0.3, m)
    x = np.concatenate([[rng.uniform(0.8, 1.6)], 0.05 * rng.standard_normal(d)])
    xbar = x + 0.1 * rng.standard_normal(d + 1)
    U = rng.uniform(0, 8, m)
    V = rng.standard_normal((m, d))
    V *= (U * rng.uniform(0, 1, m) / np.linalg.norm(V, axis=1))[:, None]
    zero = rng.uniform(0, 1, m) < 0.6
    U[zero] = 0.0
    V[zero] = 0.0
    k = min(3, m)
    C[:k] = x[1:] + 0.05 * rng.standard_normal((k, d))
    U[:k] = 12.0
    V[:k] = 0.0
    return C, R, x, xbar, U, V


def mags(C, R, x, xbar, U, V, sigma, tau):
    """Magnitudes that scale the rounding error of each output (not expected values)."""
    a = R - x[0] + U / sigma
    n = np.linalg.norm(C - x[1:] + V / sigma, axis=1)
    z = np.abs(a) + n
    return z


@pytest.mark.parametrize("m,d", [(1, 3), (255, 2), (257, 1), (1000, 10), (5003, 37), (2049, 100),
                                 (700, 224), (300, 513)])
def test_eval_alm_parity(m, d):
    rng = np.random.default_rng(m * 7 + d)
    C, R, x, xbar, U, V = rand_state(rng, m, d)
    sigma, tau = 3.0, 0.7
    q = rng.standard_normal(d + 1)
    want_H = d <= 224
    g = meb.eval_alm(C, R, x, xbar, U, V, sigma, tau, q=q, want_H=want_H)
    o = oracle.eval_alm(C, R, x, xbar, U, V, sigma, tau, q=q, want_H=want_H)
    np.testing.assert_array_equal(g["counts"], o["counts"])
    z = mags(C, R, x, xbar, U, V, sigma, tau)
    k = (m + d + 64) * EPS
    psi_mag = abs(x[0]) + sigma / 2 * np.sum(z ** 2) + np.sum(U ** 2 + np.sum(V ** 2, 1)) / (2 * sigma) \
        + tau / (2 * sigma) * np.sum((x - xbar) ** 2)
    assert abs(g["psi"] - o["psi"]) <= k * psi_mag
    gmag = 1.0 + sigma * np.sum(z) + tau / sigma * np.sum(np.abs(x - xbar))
    np.testing.assert_allclose(g["grad"], o["grad"], rtol=0, atol=k * gmag)
    tol_row = (d + 16) * EPS * sigma * z
    assert np.all(np.abs(g["Uplus"] - o["Uplus"]) <= tol_row)
    assert np.all(np.abs(g["Vplus"] - o["Vplus"]) <= tol_row[:, None])
    hmag = tau / sigma + sigma * float(np.sum(o["counts"][1:])) + 1.0
    np.testing.assert_allclose(g["Hq"], o["Hq"], rtol=0, atol=k * hmag * np.sum(np.abs(q)))
    if want_H:
        np.testing.assert_allclose(g["H"], o["H"], rtol=0, atol=k * hmag)


def test_eval_alm_kinks():
    """Balls exactly on the kinks ||b|| = a and ||b|| = -a, and the apex a = b = 0,
    built from exact Pythagorean triples so every summation order is exact."""
    C = np.array([[3.0, 4.0], [3.0, 4.0], [0.0, 0.0], [0.0, 0.0], [6.0, 8.0], [0.6, 0.8]])
    x = np.array([0.0, 0.0, 0.0])
    R = np.array([5.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    # ball 0: a = 5, ||b|| = 5 -> I ; ball 1: a = 0 -> M ; ball 2: apex -> I ;
    # ball 3: a = 1, b = 0 -> I ; ball 4: a = 0, n = 10 -> M ; ball 5: M
    xr = x.copy(); xr[0] = 0.0
    U = np.zeros(6); V = np.zeros((6, 2))
    g = meb.eval_alm(C, R, xr, xr, U, V, 1.0, 1.0, want_H=True)
    o = oracle.eval_alm(C, R, xr, xr, U, V, 1.0, 1.0, want_H=True)
    np.testing.assert_array_equal(g["counts"], o["counts"])
    np.testing.assert_allclose(g["grad"], o["grad"], atol=1e-13)
    np.testing.assert_allclose(g["H"], o["H"], atol=1e-13)
    # ||b|| = -a : radius 10 ball at distance 10 -> Z exactly at the kink
    C2 = np.array([[6.0, 8.0]]); R2 = np.array([0.0]); x2 = np.array([10.0, 0.0, 0.0])
    g = meb.eval_alm(C2, R2, x2, x2, np.zeros(1), np.zeros((1, 2)), 1.0, 1.0)
    assert list(g["counts"]) == [1, 0, 0]


@pytest.mark.parametrize("m,d", [(1, 4), (300, 1), (4097, 10), (20000, 64)])
def test_feas_check_parity(m, d):
    rng = np.random.default_rng(m + d)
    C = rng.standard_normal((m, d))
    R = rng.uniform(0, 0.2, m)
    if m > 10:
        C[m // 2] = C[3]; R[m // 2] = R[3]
    c = 0.1 * rng.standard_normal(d)
    e = np.linalg.norm(C - c, axis=1) + R
    r = float(np.quantile(e, 0.8))
    dg, ag, vg, ng = meb.feas_check(C, R, c, r, 1e-3)
    do, ao, vo, no = oracle.feas_check(C, R, c, r, 1e-3)
    assert ag == ao and ng == no
    np.testing.assert_array_equal(vg, vo)
    assert abs(dg - do) <= (d + 8) * EPS * (np.max(e) + abs(r))


def compare_solution(C, R, g, o, margin_rel=1e-6):
    r = o["r"]
    assert abs(g["r"] - r) <= 1e-8 * r, (g["r"], r)
    assert np.linalg.norm(g["c"] - o["c"]) <= 1e-7 * r
    # feasibility of the GPU ball, by the oracle's own feasibility pass
    dmax, _, _, _ = oracle.feas_check(C, R, g["c"], g["r"], 0.0)
    assert dmax <= 1e-10 * r
    # active set: bit-exact outside the band where slack is within 1e-6 r of theta r
    slack = r - R - np.linalg.norm(C - o["c"], axis=1)
    theta = 2e-6
    sure = np.abs(slack - theta * r) > margin_rel * r
    ga = np.zeros(len(R), bool); ga[np.asarray(g["active"])] = True
    oa = np.zeros(len(R), bool); oa[o["active"]] = True
    assert np.array_equal(ga[sure], oa[sure])


@pytest.mark.parametrize("case", ["gaussian_1e4_10", "cube_2e4_100", "lcg_5000_20", "d1_5000",
                                  "gaussian_3000_3", "cube_5000_224"])
def test_solve_parity(case):
    if case == "gaussian_1e4_10":
        C, R = workloads.gaussian(10_000, 10, 1001, 0.1)
    elif case == "cube_2e4_100":
        C, R = workloads.cube(20_000, 100, 7, 0.05)
    elif case == "lcg_5000_20":
        C, R = workloads.lcg(5000, 20)
    elif case == "d1_5000":
        C, R = workloads.cube(5000, 1, 3, 0.05)
    elif case == "gaussian_3000_3":
        C, R = workloads.gaussian(3000, 3, 5, 0.5)
    else:
        C, R = workloads.cube(5000, 224, 11, 0.05)
    o = oracle.solve(C, R, tol=1e-12) if case != "d1_5000" else oracle.solve(C, R, tol=1e-10)
    g = meb.solve(C, R)
    assert g["status"] == 0
    compare_solution(C, R, g, o)


def test_solve_closed_forms():
    C = np.array([[1.0, 2.0], [4.0, 6.0]]); R = np.array([0.3, 1.1])
    g = meb.solve(C, R)
    r = (5.0 + 0.3 + 1.1) / 2
    assert abs(g["r"] - r) <= 1e-10 * r
    np.testing.assert_allclose(g["c"], C[0] + (r - 0.3) * (C[1] - C[0]) / 5.0, atol=1e-9)
    g = meb.solve(np.array([[1.0, 2.0, 3.0]]), np.array([0.7]))
    assert g["r"] == 0.7 and list(g["c"]) == [1.0, 2.0, 3.0]
    g = meb.solve(np.tile([1.5, -2.0], (7, 1)), np.zeros(7))
    assert g["r"] == 0.0 and g["n_active"] == 7
    ctr = np.array([1.0, -2.0, 3.0, 0.5]); Rc = np.linspace(0.1, 2.0, 50)
    g = meb.solve(np.tile(ctr, (50, 1)), Rc)
    assert abs(g["r"] - 2.0) <= 1e-9 and np.linalg.norm(g["c"] - ctr) <= 1e-8
    n = 12
    g = meb.solve(np.eye(n), np.zeros(n))
    assert abs(g["r"] - np.sqrt((n - 1) / n)) <= 1e-9 and g["n_active"] == n


def test_fp64_newton_path():
    """newton_fp64 = 1 solves every dense Newton system by the FP64 Cholesky
    (the fallback of the FP32 Gauss-Jordan path): same solution."""
    C, R = workloads.cube(20_000, 40, 31, 0.05)
    p = meb.params_default()
    p.newton_fp64 = 1
    g64 = meb.solve(C, R, params=p)
    assert g64["status"] == 0
    assert g64["newton_fp64"] > 0 and g64["newton_inverses"] == 0
    g = meb.solve(C, R)
    assert g["newton_fp64"] == 0 and g["newton_inverses"] > 0
    o = oracle.solve(C, R, tol=1e-12)
    compare_solution(C, R, g64, o)
    compare_solution(C, R, g, o)


def test_sphere_cg_path():
    C, R, ctr = workloads.sphere(6000, 300, 4)
    g = meb.solve(C, R)
    assert g["status"] == 0 and g["cg_iters"] > 0
    assert abs(g["r"] - 1.0) <= 1e-8
    assert np.linalg.norm(g["c"] - ctr) <= 1e-7


def test_invalid_inputs():
    C = np.zeros((4, 2)); R = np.ones(4)
    bad = R.copy(); bad[1] = -1.0
    with pytest.raises(meb.MebError) as e:
        meb.solve(C, bad)
    assert e.value.code == -1
    Cn = C.copy(); Cn[2, 1] = np.nan
    with pytest.raises(meb.MebError):
        meb.solve(Cn, R)
    with pytest.raises(meb.MebError):
        meb.solve(np.zeros((0, 2)), np.zeros(0))
    P = meb.params_default()
    P.max_cg = 20001                     # past the device-side CG loop's bound
    with pytest.raises(meb.MebError) as e:
        meb.solve(workloads.cube(100, 3, 1, 0.05)[0], np.zeros(100), params=P)
    assert e.value.code == -1


def test_device_pointer_path():
    torch = pytest.importorskip("torch")
    C, R = workloads.gaussian(5000, 16, 21, 0.1)
    h = meb.solve(C, R)
    dC = torch.from_numpy(C).cuda(); dR = torch.from_numpy(R).cuda()
    g = meb.solve(dC, dR)
    assert g["r"] == h["r"]
    assert np.array_equal(g["c"].cpu().numpy(), h["c"])
    assert np.array_equal(g["active"].cpu().numpy(), h["active"])


def test_screen_shadows_agree():
    """Solves screen the FP16 shadow with register batches (default); the
    fp16_bulk option screens it through the bulk-copy pipeline, fp32 screens
    the FP32 shadow and fp64 screens nothing (every ball through the FP64
    rows).  The certificates only decide which balls skip the FP64 evaluation,
    so the solves agree to the solve tolerance and keep the same active set."""
    C, R = workloads.cube(30_000, 40, 23, 0.05)
    res = {k: meb.solve(C, R, ctx=meb.Context(0, screen=k))
           for k in ("fp16", "fp16_bulk", "fp32", "fp64")}
    ref = oracle.solve(C, R)
    for k, r in res.items():
        assert r["status"] == 0 and r["kkt_max"] <= 1e-10, k
        assert abs(r["r"] - ref["r"]) <= 1e-8 * ref["r"], k
        assert np.array_equal(r["active"], res["fp16"]["active"]), k


@pytest.mark.parametrize("mode", ["fp16", "fp16_bulk"])
def test_screen_ragged_tiles(mode):
    """Both FP16 screens on sizes whose last tile is partial (m not a multiple
    of 256) and on d that leaves padding in the last FP16 row."""
    ctx = meb.Context(0, screen=mode)
    for m, d, seed in [(1, 5, 1), (257, 3, 2), (5000 - 37, 17, 3), (20_011, 100, 4)]:
        C, R = workloads.cube(m, d, seed, 0.05)
        g = meb.solve(C, R, ctx=ctx)
        o = oracle.solve(C, R, tol=1e-12)
        assert g["status"] == 0
        compare_solution(C, R, g, o)


def test_tick_loops_agree():
    """The graph-batched tick loop (default), the host-driven loop and the
    while-node graph run the same kernels in the same order: bit-identical."""
    C, R = workloads.cube(30_000, 40, 17, 0.05)
    ctxs = {k: meb.Context(0, tick_loop=k) for k in ("graph", "host", "while")}
    res = {k: meb.solve(C, R, ctx=c) for k, c in ctxs.items()}
    g = res["graph"]
    for k in ("host", "while"):
        h = res[k]
        assert g["r"] == h["r"] and np.array_equal(g["c"], h["c"]), k
        assert g["passes"] == h["passes"] and g["ssn_iters"] == h["ssn_iters"], k
        assert np.array_equal(g["active"], h["active"]), k
    ctx = ctxs["graph"]
    ctx.set_profiling(True)          # event nodes in the graph: same results
    p = meb.solve(C, R, ctx=ctx)
    ctx.set_profiling(False)
    assert p["r"] == g["r"] and np.array_equal(p["c"], g["c"])
    assert ctx.stats()["pass_launches"] > 0
    g2 = meb.solve(C, R, ctx=ctx)    # graph reused
    assert g2["r"] == g["r"] and np.array_equal(g2["c"], g["c"])
    # waits that sleep, scratch freed after the call: same results
    q = meb.solve(C, R, ctx=meb.Context(0, blocking_sync=1, release_scratch=1))
    assert q["r"] == g["r"] and np.array_equal(q["c"], g["c"])
    assert np.array_equal(q["active"], g["active"])


def test_tick_loops_agree_matrix_free():
    """d + 1 > 225: the CG loop runs inside the tick graph (a conditional
    while node per tick) or from the host: the same kernels in the same
    order, bit-identical."""
    C, R = workloads.cube(6000, 300, 23, 0.05)
    res = {k: meb.solve(C, R, ctx=meb.Context(0, tick_loop=k)) for k in ("graph", "host", "while")}
    g = res["graph"]
    assert g["cg_iters"] > 0
    for k in ("host", "while"):
        h = res[k]
        assert g["r"] == h["r"] and np.array_equal(g["c"], h["c"]), k
        assert g["passes"] == h["passes"] and g["cg_iters"] == h["cg_iters"], k
        assert np.array_equal(g["active"], h["active"]), k
    o = oracle.solve(C, R, tol=1e-12)
    assert abs(g["r"] - o["r"]) <= 1e-8 * o["r"]


def test_options_rejected():
    ctx = meb.Context(0)
    for name, val in (("screen", 7), ("tick_loop", 3), ("wait_cycles", -1),
                      ("eval_shadow_exp", 100), ("blocking_sync", 2), ("batch_slots", -1)):
        with pytest.raises(meb.MebError):
            ctx.set_option(name, val)
