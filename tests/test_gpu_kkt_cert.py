"""GPU parity of what the solve returns beyond (c, r), and of the certificate
the screens rest on.

* KKT residuals (Sec. 5): info.kkt of meb_solve against the oracle's kkt()
  evaluated at the returned point with the multipliers meb_get_multipliers
  reports (Algorithm 1's multiplier update at the last accepted point).
* Weak duality (Sec. 2, dual problem): the GPU's own multipliers, repaired
  into a dual-feasible point, give a lower bound on r*; the returned radius is
  an upper bound.  The oracle's r* must lie in that bracket, and the bracket
  must be tight.
* The FP16 certificate: meb_eval_alm screening the FP16 shadow at adversarial
  states (slack at and around the certificate's margin on both sides, data far
  from the shadow origin, shadow values in the half subnormal range or beyond
  the half range) gives the oracle's case counts exactly and its Psi, grad,
  U+, V+ within the rounding bounds.
* The bounded wait of the bulk-copy screen: a zero wait limit makes it give
  up; the solve reports MEB_ETIMEOUT and the context solves correctly after.
* The plain FP64 mode (no shadow at all) agrees with the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
THETA = 2e-6


def dense_multipliers(m, d, idx, u, v):
    U = np.zeros(m)
    V = np.zeros((m, d))
    U[idx] = u
    V[idx] = v
    return U, V


def dual_lower_bound(C, R, U, V):
    """A dual-feasible point from (U, V) and its objective (dual problem,
    Sec. 2): sum u = 1, sum v = 0, (u_i, v_i) in Q.  Weak duality makes it a
    lower bound on r*."""
    Cc = C - C.mean(axis=0)
    U = np.maximum(U, 0.0).copy()
    V = V.copy()
    V -= np.outer(U, V.sum(axis=0) / U.sum())
    U = np.maximum(U, np.linalg.norm(V, axis=1))
    s = U.sum()
    U /= s
    V /= s
    return float(U @ R + np.sum(V * Cc))


CASES = {
    "gaussian_1e4_10": lambda: workloads.gaussian(10_000, 10, 1001, 0.1),
    "cube_2e4_100": lambda: workloads.cube(20_000, 100, 7, 0.05),
    "lcg_5000_20": lambda: workloads.lcg(5000, 20),
    "cube_5000_224": lambda: workloads.cube(5000, 224, 11, 0.05),
    "sphere_6000_300": lambda: workloads.sphere(6000, 300, 4)[:2],
}


@pytest.mark.parametrize("case", list(CASES))
def test_kkt_residuals_and_multipliers(case):
    C, R = CASES[case]()
    m, d = C.shape
    ctx = meb.Context(0)
    g = meb.solve(C, R, ctx=ctx)
    assert g["status"] == 0
    idx, u, v = ctx.multipliers()
    assert len(idx) >= 2 and np.all(np.diff(idx) > 0)       # ascending, no repeats
    U, V = dense_multipliers(m, d, idx, u, v)
    k_orc = oracle.kkt(C, R, g["r_alm"], g["c"], U, V)
    k_gpu = np.asarray(g["kkt"])
    r = g["r"]
    # rounding scales of each residual (both sides evaluate the same definition
    # at the same point with the same multipliers, in different orders)
    n = len(idx)
    su = np.sum(np.abs(u))
    sv = np.sum(np.linalg.norm(v, axis=1))
    tol = np.array([(n + 16) * EPS * su,
                    (n + d + 16) * EPS * sv,
                    (d + 16) * EPS * 4 * r,
                    (d + 16) * EPS * max(su, 1.0),
                    (d + 16) * EPS * 4 * r * max(su, 1.0)])
    assert np.all(np.abs(k_gpu - k_orc) <= tol), (k_gpu, k_orc, tol)
    assert g["kkt_max"] <= 1e-10
    # multipliers are zero off the active set (complementarity)
    act = set(np.asarray(g["active"]).tolist())
    strong = idx[u > 1e-9 * max(u)]
    assert set(strong.tolist()) <= act
    # weak-duality bracket from the GPU's own multipliers
    lb = dual_lower_bound(C, R, U, V)
    assert lb <= r * (1 + 1e-14)
    assert (r - lb) / r <= 1e-9, (r, lb)
    # cross-certification: each side's dual bound is below the other side's
    # (feasible) radius, and the radii agree
    o = oracle.solve(C, R, tol=1e-12)
    assert lb <= o["r"] * (1 + 1e-13)
    assert dual_lower_bound(C, R, o["U"], o["V"]) <= r * (1 + 1e-13)
    assert abs(r - o["r"]) <= 1e-8 * o["r"]


def test_multipliers_trivial_cases():
    ctx = meb.Context(0)
    meb.solve(np.array([[1.0, 2.0, 3.0]]), np.array([0.7]), ctx=ctx)
    idx, u, v = ctx.multipliers()
    assert list(idx) == [0] and list(u) == [1.0] and not v.any()
    meb.solve(np.tile([1.5, -2.0], (4, 1)), np.zeros(4), ctx=ctx)
    idx, u, v = ctx.multipliers()
    assert list(idx) == [0, 1, 2, 3] and np.all(u == 0.25)
    meb.eval_alm(np.eye(3), np.zeros(3), np.ones(4), np.ones(4), np.zeros(3), np.zeros((3, 3)),
                 1.0, 1.0, ctx=ctx)
    with pytest.raises(meb.MebError):
        ctx.multipliers()     # an evaluation leaves no solve to report


# ------------------------------------------------------------ FP16 certificate
def margin_state(rng, m, d, offset=0.0, far_first=0.0):
    """Balls around the ball (r, c) = (1, c0) at prescribed slacks
    r - r_i - ||c - c_i|| = +-k r, k geometric from 1e-10 to 0.3, on both sides
    of the boundary (far below the FP16 certificate's width, far above the
    rounding of the FP64 rows, so the exact case of every ball is decided the
    same way by both sides); balls 4-6 contain the ball (case I); zero
    multipliers except balls 1-3."""
    c0 = offset + 0.01 * rng.standard_normal(d)
    r = 1.0
    dirs = rng.standard_normal((m, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    mag = 10.0 ** rng.uniform(-10, np.log10(0.3), m)
    slack = np.where(rng.uniform(0, 1, m) < 0.5, mag, -mag)
    Ri = rng.uniform(0, 0.6, m)
    dist = r - Ri - slack
    Ri[4:7] = [1.3, 1.4, 1.5]
    dist[4:7] = [0.05, 0.1, 0.2]
    C = c0 + dirs * dist[:, None]
    if far_first:
        C[0] = c0 + far_first * dirs[0]          # the shadow origin, far from the rest
        Ri[0] = 0.0
    x = np.concatenate([[r], c0])
    xbar = x + 1e-3 * rng.standard_normal(d + 1)
    U = np.zeros(m)
    V = np.zeros((m, d))
    U[1:4] = rng.uniform(0.5, 2, 3)
    V[1:4] = 0.3 * rng.standard_normal((3, d))
    return C, Ri, x, xbar, U, V


def check_eval_against_oracle(g, o, C, R, x, xbar, U, V, sigma, tau):
    np.testing.assert_array_equal(g["counts"], o["counts"])
    m, d = C.shape
    a = R - x[0] + U / sigma
    z = np.abs(a) + np.linalg.norm(C - x[1:] + V / sigma, axis=1)
    k = (m + d + 64) * EPS
    psi_mag = abs(x[0]) + sigma / 2 * np.sum(z ** 2) + np.sum(U ** 2 + np.sum(V ** 2, 1)) / (2 * sigma) \
        + tau / (2 * sigma) * np.sum((x - xbar) ** 2)
    assert abs(g["psi"] - o["psi"]) <= k * psi_mag
    gmag = 1.0 + sigma * np.sum(z) + tau / sigma * np.sum(np.abs(x - xbar))
    np.testing.assert_allclose(g["grad"], o["grad"], rtol=0, atol=k * gmag)
    tol_row = (d + 16) * EPS * sigma * z
    assert np.all(np.abs(g["Uplus"] - o["Uplus"]) <= tol_row)
    assert np.all(np.abs(g["Vplus"] - o["Vplus"]) <= tol_row[:, None])


@pytest.mark.parametrize("m,d,offset,far,exp", [
    (20_000, 16, 0.0, 0.0, 0),        # slack at the margin, shadow scale 1
    (20_011, 100, 0.0, 0.0, 1),       # ragged tail, d leaving padding
    (9_000, 37, 1e5, 0.0, 0),         # all data far from 0 (truncation error of the FP32 shadow)
    (9_000, 37, 0.0, 3e3, 12),        # the shadow origin (first centre) far from the rest
    (9_000, 8, 0.0, 0.0, 20),         # shadow values ~1e-6: half subnormals
    (9_000, 8, 0.0, 0.0, -20),        # shadow values ~1e6: beyond the half range (never certified)
])
def test_fp16_certificate_adversarial(m, d, offset, far, exp):
    rng = np.random.default_rng(m + d + exp)
    C, R, x, xbar, U, V = margin_state(rng, m, d, offset, far)
    sigma, tau = 50.0, 2.0
    o = oracle.eval_alm(C, R, x, xbar, U, V, sigma, tau)
    ctx16 = meb.Context(0, eval_screen="fp16", eval_shadow_exp=exp)
    g16 = meb.eval_alm(C, R, x, xbar, U, V, sigma, tau, ctx=ctx16)
    check_eval_against_oracle(g16, o, C, R, x, xbar, U, V, sigma, tau)
    assert np.all(o["counts"] > 0)      # cases Z, I and M all present
    for mode in ("fp32", "fp64", "fp16_bulk"):
        ctxm = meb.Context(0, eval_screen=mode, eval_shadow_exp=exp)
        gm = meb.eval_alm(C, R, x, xbar, U, V, sigma, tau, ctx=ctxm)
        check_eval_against_oracle(gm, o, C, R, x, xbar, U, V, sigma, tau)


# ------------------------------------------------------------ bounded waits
def test_bulk_screen_wait_limit_gives_timeout_then_recovers():
    C, R = workloads.cube(40_000, 40, 29, 0.05)
    ref = meb.solve(C, R, ctx=meb.Context(0, screen="fp16_bulk"))
    ctx = meb.Context(0, screen="fp16_bulk", wait_cycles=0)
    with pytest.raises(meb.MebError) as e:
        meb.solve(C, R, ctx=ctx)
    assert e.value.code == -5          # MEB_ETIMEOUT
    ctx.set_option("wait_cycles", 2_000_000_000)
    g = meb.solve(C, R, ctx=ctx)
    assert g["status"] == 0
    assert g["r"] == ref["r"] and np.array_equal(g["c"], ref["c"])
    o = oracle.solve(C, R, tol=1e-12)
    assert abs(g["r"] - o["r"]) <= 1e-8 * o["r"]


# ------------------------------------------------------------ plain FP64 mode
@pytest.mark.parametrize("m,d,seed", [(20_000, 40, 3), (5_003, 120, 4)])
def test_plain_fp64_mode(m, d, seed):
    C, R = workloads.cube(m, d, seed, 0.05)
    ctx = meb.Context(0, screen="fp64")
    ctx.reset_stats()
    g = meb.solve(C, R, ctx=ctx)
    o = oracle.solve(C, R, tol=1e-12)
    assert g["status"] == 0
    assert abs(g["r"] - o["r"]) <= 1e-8 * o["r"]
    assert np.linalg.norm(g["c"] - o["c"]) <= 1e-7 * o["r"]
    # every ball went through the FP64 rows in every pass (a trial rejected
    # from the lower bound alone, counted as a backtrack, evaluates no rows)
    assert g["fp64_rows"] >= m * (g["passes"] - g["backtracks"])
    dm, am, viol, nv = meb.feas_check(C, R, g["c"], g["r"], 0.0, ctx=meb.Context(0, eval_screen="fp64"))
    do, ao, _, _ = oracle.feas_check(C, R, g["c"], g["r"], 0.0)
    assert am == ao and nv == 0


def test_device_path_argument_checks():
    torch = pytest.importorskip("torch")
    C = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    R = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        meb.solve(C, R)
    with pytest.raises(ValueError):
        meb.solve(C.double(), R[:9])
    with pytest.raises(ValueError):
        meb.solve(C.double().t().contiguous().t(), R)
    with pytest.raises(ValueError):
        meb.feas_check(C.double(), R, torch.zeros(2, dtype=torch.float64, device="cuda"), 1.0, 0.0)
