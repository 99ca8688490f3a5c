"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle
with a closed form, an independent characterisation (Moreau decomposition,
the dual representation of the augmented Lagrangian, weak duality), finite
differences, or a brute-force solver written here from scratch.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_2605_31425_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def in_Q(a, b, tol):
    return np.linalg.norm(b) <= a + tol


def rand_state(rng, m, d, frac_zero=0.5):
    """Random evaluation state mixing the three cases of the projection."""
    scale = rng.choice([0.15, 1.0, 3.0], size=m)
    C = rng.standard_normal((m, d)) * scale[:, None]
    R = rng.uniform(0, 0.3, m)
    x = np.concatenate([[rng.uniform(1.5, 2.5)], 0.05 * rng.standard_normal(d)])
    xbar = x + 0.1 * rng.standard_normal(d + 1)
    U = rng.uniform(0, 8, m)
    V = rng.standard_normal((m, d))
    V *= (U * rng.uniform(0, 1, m) / np.linalg.norm(V, axis=1))[:, None]
    zero = rng.uniform(0, 1, m) < frac_zero
    U[zero] = 0.0
    V[zero] = 0.0
    # a few balls near the centre with large multipliers: case I
    C[:3] = x[1:] + 0.05 * rng.standard_normal((3, d))
    U[:3] = 12.0
    V[:3] = 0.0
    return C, R, x, xbar, U, V


def brute_force_meb(C, R):
    """Smallest enclosing ball by enumerating every support set S (|S| <= d+1):
    the ball internally tangent to all balls of S with centre in aff(S)."""
    m, d = C.shape
    best_r, best_c = math.inf, None
    for k in range(1, min(m, d + 1) + 1):
        for S in itertools.combinations(range(m), k):
            for c, r in _tangent(C[list(S)], R[list(S)]):
                slack = r - R - np.linalg.norm(C - c, axis=1)
                if slack.min() >= -1e-11 * max(1.0, r) and r < best_r:
                    best_r, best_c = r, c
    return best_r, best_c


def _tangent(Cs, Rs):
    if len(Rs) == 1:
        yield Cs[0].copy(), float(Rs[0])
        return
    dl = Cs[1:] - Cs[0]
    rho = Rs[1:] - Rs[0]
    G = dl @ dl.T
    if np.linalg.matrix_rank(G, tol=1e-10 * max(1.0, np.abs(G).max())) < G.shape[0]:
        return
    h = 0.5 * (np.sum(dl * dl, axis=1) - rho * rho)
    e0 = dl.T @ np.linalg.solve(G, h)
    e1 = dl.T @ np.linalg.solve(G, rho)
    a2, a1, a0 = e1 @ e1 - 1.0, 2.0 * (e0 @ e1), e0 @ e0
    if abs(a2) < 1e-14:
        roots = [] if a1 == 0 else [-a0 / a1]
    else:
        disc = a1 * a1 - 4 * a2 * a0
        if disc < 0:
            return
        sq = math.sqrt(disc)
        roots = [(-a1 + sq) / (2 * a2), (-a1 - sq) / (2 * a2)]
    for s in roots:
        if s >= 0 and np.all(s - rho >= -1e-12):
            yield Cs[0] + e0 + s * e1, float(Rs[0] + s)


def dual_lower_bound(C, R, U, V):
    """A dual-feasible point built from (U, V) and its objective (eq. of the
    dual problem, Sec. 2): a certified lower bound on r* by weak duality."""
    Cc = C - C.mean(axis=0)
    U = np.maximum(U, 0.0).copy()
    V = V.copy()
    V -= np.outer(U, V.sum(axis=0) / U.sum())
    U = np.maximum(U, np.linalg.norm(V, axis=1))
    s = U.sum()
    U /= s
    V /= s
    return float(U @ R + np.sum(V * Cc))


def max_type_radius(C, R, c):
    return float(np.max(cdist(c[None, :], C)[0] + R))


# ---------------------------------------------------------------- LCG (Sec. 5)
def test_lcg_matches_worked_values():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "lcg_psi.txt"))
            if ln.strip() and not ln.startswith("#")]
    psi = workloads.lcg_psi(len(rows))
    for (j, p, v), got in zip(rows, psi):
        assert int(p) == got
        assert float(v) == got / 40.96
    C, R = workloads.lcg(2, 3)
    assert R[0] == 76.07421875 and list(C[0]) == [53.0517578125, 8.056640625, 85.2294921875]
    assert R[1] == 27.1484375


def test_lcg_full_period():
    psi = workloads.lcg_psi(4096 * 2)
    assert len(set(psi[:4096].tolist())) == 4096
    assert np.array_equal(psi[:4096], psi[4096:])


# ---------------------------------------------------------------- projection
@pytest.mark.parametrize("d", [1, 2, 5, 33])
def test_projection_moreau(d):
    """p = Pi_Q(z) iff p in Q, p - z in Q (Q self-dual) and <p, p - z> = 0."""
    rng = np.random.default_rng(d)
    seen = set()
    for _ in range(400):
        a = rng.standard_normal() * 2 * math.sqrt(d)
        b = rng.standard_normal(d)
        pa, pb, cs = oracle.soc_project(a, b)
        seen.add(cs)
        scale = 1.0 + abs(a) + np.linalg.norm(b)
        assert in_Q(pa, pb, 1e-13 * scale)
        assert in_Q(pa - a, pb - b, 1e-13 * scale)
        assert abs(pa * (pa - a) + pb @ (pb - b)) <= 1e-13 * scale ** 2
        # idempotent
        qa, qb, _ = oracle.soc_project(pa, pb)
        assert abs(qa - pa) <= 1e-14 * scale and np.allclose(qb, pb, rtol=0, atol=1e-14 * scale)
        # distance = ||Pi_Q(-z)|| (Moreau, Q self-dual)
        na, nb, _ = oracle.soc_project(-a, -b)
        assert oracle.soc_dist(a, b) == pytest.approx(math.hypot(na, np.linalg.norm(nb)),
                                                      rel=1e-12, abs=1e-14 * scale)
    assert seen == {0, 1, 2}


def test_projection_kinks_and_case_order():
    b = np.array([3.0, 4.0])
    assert oracle.soc_project(5.0, b)[2] == 1          # ||b|| = a : I
    assert oracle.soc_project(-5.0, b)[2] == 0         # ||b|| = -a : Z
    assert oracle.soc_project(0.0, np.zeros(3))[2] == 1  # apex : I
    assert oracle.soc_project(-1.0, np.zeros(3))[2] == 0
    pa, pb, cs = oracle.soc_project(0.0, b)            # a = 0 : M, (0+5)/2 (1, b/5)
    assert cs == 2 and pa == 2.5 and np.allclose(pb, [1.5, 2.0])


def test_projection_firmly_nonexpansive():
    rng = np.random.default_rng(7)
    d = 6
    for _ in range(300):
        z1 = rng.standard_normal(d + 1) * 2
        z2 = rng.standard_normal(d + 1) * 2
        p1 = np.concatenate([[oracle.soc_project(z1[0], z1[1:])[0]], oracle.soc_project(z1[0], z1[1:])[1]])
        p2 = np.concatenate([[oracle.soc_project(z2[0], z2[1:])[0]], oracle.soc_project(z2[0], z2[1:])[1]])
        assert (p1 - p2) @ (z1 - z2) >= np.sum((p1 - p2) ** 2) - 1e-12


@pytest.mark.parametrize("d", [1, 3, 8])
def test_jacobian_finite_differences(d):
    rng = np.random.default_rng(100 + d)
    h = 1e-6
    cases = set()
    for _ in range(60):
        a = rng.standard_normal() * 2 * math.sqrt(d)
        b = rng.standard_normal(d)
        n = np.linalg.norm(b)
        if min(abs(n - a), abs(n + a)) < 1e-3:
            continue
        P, cs = oracle.soc_jacobian(a, b)
        cases.add(cs)
        z = np.concatenate([[a], b])
        FD = np.empty((d + 1, d + 1))
        for k in range(d + 1):
            e = np.zeros(d + 1); e[k] = h
            zp, zm = z + e, z - e
            pp = oracle.soc_project(zp[0], zp[1:]); pm = oracle.soc_project(zm[0], zm[1:])
            FD[:, k] = (np.concatenate([[pp[0]], pp[1]]) - np.concatenate([[pm[0]], pm[1]])) / (2 * h)
        assert np.allclose(P, FD, atol=1e-6)
        assert np.allclose(P, P.T)
        ev = np.linalg.eigvalsh(P)
        assert ev.min() >= -1e-12 and ev.max() <= 1 + 1e-12
    assert cases == {0, 1, 2}


# ---------------------------------------------------------------- eval_alm
def _dual_rep(C, R, x, xbar, U, V, sigma, tau, Y0, Y):
    """r - sum <y_i', G_i(x)> - 1/(2 sigma) sum ||y_i' - y_i||^2 + tau/(2 sigma)||x-xbar||^2,
    G_i(x) = (r - r_i, c - c_i); its maximum over y' in Q^m is Psi(x)."""
    r, c = x[0], x[1:]
    lin = np.sum(Y0 * (r - R)) + np.sum(Y * (c[None, :] - C))
    quad = np.sum((Y0 - U) ** 2) + np.sum((Y - V) ** 2)
    return r - lin - quad / (2 * sigma) + tau / (2 * sigma) * np.sum((x - xbar) ** 2)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eval_psi_is_the_dual_maximum(seed):
    rng = np.random.default_rng(seed)
    m, d = 40, 4
    C, R, x, xbar, U, V = rand_state(rng, m, d)
    sigma, tau = 2.5, 0.7
    out = oracle.eval_alm(C, R, x, xbar, U, V, sigma, tau)
    assert set(np.nonzero(out["counts"])[0]) == {0, 1, 2}
    Up, Vp = out["Uplus"], out["Vplus"]
    for i in range(m):
        assert in_Q(Up[i], Vp[i], 1e-12)
    best = _dual_rep(C, R, x, xbar, U, V, sigma, tau, Up, Vp)
    assert out["psi"] == pytest.approx(best, rel=1e-12, abs=1e-12)
    for _ in range(200):
        Y0 = Up + 0.05 * rng.standard_normal(m)
        Y = Vp + 0.05 * rng.standard_normal((m, d))
        nY = np.linalg.norm(Y, axis=1)
        Y0 = np.maximum(Y0, nY)  # back into Q
        assert _dual_rep(C, R, x, xbar, U, V, sigma, tau, Y0, Y) <= out["psi"] + 1e-12


@pytest.mark.parametrize("seed", [3, 4])
def test_eval_grad_and_hessian_finite_differences(seed):
    rng = np.random.default_rng(seed)
    m, d = 30, 3
    C, R, x, xbar, U, V = rand_state(rng, m, d)
    sigma, tau = 1.7, 0.9
    q = rng.standard_normal(d + 1)
    out = oracle.eval_alm(C, R, x, xbar, U, V, sigma, tau, q=q, want_H=True)
    h = 1e-6
    for k in range(d + 1):
        e = np.zeros(d + 1); e[k] = h
        pp = oracle.eval_alm(C, R, x + e, xbar, U, V, sigma, tau)
        pm = oracle.eval_alm(C, R, x - e, xbar, U, V, sigma, tau)
        assert out["grad"][k] == pytest.approx((pp["psi"] - pm["psi"]) / (2 * h), rel=1e-6, abs=1e-6)
        # H e_k = d grad / d x_k (away from kinks: same cases at x +- e)
        if np.array_equal(pp["counts"], out["counts"]) and np.array_equal(pm["counts"], out["counts"]):
            assert np.allclose(out["H"][:, k], (pp["grad"] - pm["grad"]) / (2 * h), atol=1e-5)
    H = out["H"]
    assert np.allclose(H, H.T)
    assert np.linalg.eigvalsh(H).min() >= tau / sigma * (1 - 1e-12)
    assert np.allclose(out["Hq"], H @ q, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- feasibility
def test_feas_check_against_distance_matrix():
    rng = np.random.default_rng(11)
    C = rng.standard_normal((500, 7))
    R = rng.uniform(0, 0.2, 500)
    C[200] = C[37]; R[200] = R[37]  # a duplicate: ties go to the lower index
    c = rng.standard_normal(7) * 0.1
    e = cdist(c[None, :], C)[0] + R
    r = float(np.quantile(e, 0.9))
    dm, am, viol, nv = oracle.feas_check(C, R, c, r, 0.0)
    assert dm == pytest.approx(e.max() - r, rel=1e-14)
    assert am == int(np.argmax(e))
    assert np.array_equal(viol, np.nonzero(e - r > 0)[0]) and nv == len(viol)
    # ties: make the duplicate the farthest
    C[37] = c + 100.0; C[200] = C[37]
    dm, am, _, _ = oracle.feas_check(C, R, c, r, 0.0)
    assert am == 37


# ---------------------------------------------------------------- KKT_max
def test_kkt_two_ball_closed_form():
    c1, c2 = np.array([0.0, 0.0, 0.0]), np.array([3.0, 4.0, 0.0])
    r1, r2 = 0.5, 1.5
    D = 5.0
    r = (D + r1 + r2) / 2
    c = c1 + (r - r1) * (c2 - c1) / D
    C = np.stack([c1, c2]); R = np.array([r1, r2])
    U = np.array([0.5, 0.5])
    V = np.stack([0.5 * (c1 - c) / (r - r1), 0.5 * (c2 - c) / (r - r2)])
    k = oracle.kkt(C, R, r, c, U, V)
    assert np.all(k <= 1e-15)
    eps = 1e-3
    k = oracle.kkt(C, R, r - eps, c, U, V)
    assert k[2] == pytest.approx(eps / math.sqrt(2), rel=1e-9)   # (n - a)/sqrt(2)
    assert k[4] == pytest.approx(eps / 2, rel=1e-9)              # |eps * u_i|
    assert k[0] <= 1e-15 and k[1] <= 1e-15 and k[3] <= 1e-15


# ---------------------------------------------------------------- solve
def check_solution(C, R, res, r_true=None, c_true=None, rtol=1e-10):
    r, c = res["r"], res["c"]
    assert res["status"] == 0
    # every ball enclosed at the returned radius (max-type value)
    assert r == pytest.approx(max_type_radius(C, R, c), rel=1e-14)
    lb = dual_lower_bound(C, R, res["U"], res["V"])
    assert lb <= r * (1 + 1e-14)
    assert (r - lb) / r <= rtol
    if r_true is not None:
        assert r == pytest.approx(r_true, rel=rtol)
    if c_true is not None:
        assert np.linalg.norm(c - c_true) <= 1e-7 * max(r, 1e-300) + 1e-12


def test_two_balls_closed_form():
    C = np.array([[1.0, 2.0], [4.0, 6.0]])
    R = np.array([0.3, 1.1])
    res = oracle.solve(C, R, tol=1e-12)
    D = 5.0
    r = (D + 0.3 + 1.1) / 2
    check_solution(C, R, res, r, C[0] + (r - 0.3) * (C[1] - C[0]) / D)


def test_two_balls_containment():
    C = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    R = np.array([2.0, 0.25])
    res = oracle.solve(C, R, tol=1e-12)
    check_solution(C, R, res, 2.0, C[0])


def test_concentric_balls():
    rng = np.random.default_rng(5)
    ctr = np.array([1.0, -2.0, 3.0, 0.5])
    R = rng.uniform(0, 2, 25)
    C = np.tile(ctr, (25, 1))
    res = oracle.solve(C, R, tol=1e-12)
    check_solution(C, R, res, R.max(), ctr)


@pytest.mark.parametrize("n", [2, 3, 5, 12])
def test_regular_simplex(n):
    C = np.eye(n)
    res = oracle.solve(C, np.zeros(n), tol=1e-12)
    check_solution(C, np.zeros(n), res, math.sqrt((n - 1) / n), np.full(n, 1.0 / n))
    assert len(res["active"]) == n
    res = oracle.solve(C, np.full(n, 0.25), tol=1e-12)
    check_solution(C, np.full(n, 0.25), res, math.sqrt((n - 1) / n) + 0.25)


def test_cross_polytope_and_hypercube():
    n = 6
    C = np.vstack([np.eye(n), -np.eye(n)])
    check_solution(C, np.zeros(2 * n), oracle.solve(C, np.zeros(2 * n), tol=1e-12), 1.0, np.zeros(n))
    d = 7
    C = np.array(list(itertools.product([-1.0, 1.0], repeat=d)))
    res = oracle.solve(C, np.zeros(len(C)), tol=1e-12)
    check_solution(C, np.zeros(len(C)), res, math.sqrt(d), np.zeros(d))


def test_one_dimensional_large_m():
    rng = np.random.default_rng(9)
    C = rng.uniform(-10, 10, (20000, 1))
    R = rng.uniform(0, 1, 20000)
    hi, lo = np.max(C[:, 0] + R), np.min(C[:, 0] - R)
    # sigma reaches 1e5 here, where |1 - sum u| has a rounding floor near 2e-10
    res = oracle.solve(C, R, tol=1e-9)
    check_solution(C, R, res, (hi - lo) / 2, np.array([(hi + lo) / 2]))


def test_sphere_points():
    C, R, ctr = workloads.sphere(3000, 60, 4)
    res = oracle.solve(C, R, tol=1e-12)
    check_solution(C, R, res, 1.0, ctr, rtol=1e-9)


@pytest.mark.parametrize("seed,d,m", [(s, d, m) for s in range(4) for d, m in [(2, 9), (3, 8)]])
def test_brute_force_tiny(seed, d, m):
    rng = np.random.default_rng(1000 + seed)
    C = rng.standard_normal((m, d))
    R = rng.uniform(0, 0.5, m)
    rb, cb = brute_force_meb(C, R)
    res = oracle.solve(C, R, tol=1e-12)
    check_solution(C, R, res, rb, cb, rtol=1e-10)


def test_single_ball_and_identical_points():
    C = np.array([[1.0, 2.0, 3.0]]); R = np.array([0.7])
    res = oracle.solve(C, R)
    assert res["r"] == 0.7 and np.array_equal(res["c"], C[0])
    C = np.tile([1.5, -2.0], (5, 1)); R = np.zeros(5)
    res = oracle.solve(C, R)
    assert res["r"] == 0.0 and np.allclose(res["c"], [1.5, -2.0])


def test_kkt_invariants_gaussian():
    C, R = workloads.gaussian(3000, 10, 77, 0.1)
    res = oracle.solve(C, R, tol=1e-12)
    check_solution(C, R, res)
    U, V, r, c = res["U"], res["V"], res["r"], res["c"]
    assert abs(1 - U.sum()) <= 1e-10 and np.linalg.norm(V.sum(0)) <= 1e-10
    sup = U > 1e-9
    lam = U[sup] / (r - R[sup])
    lam /= lam.sum()
    assert np.linalg.norm(lam @ C[sup] - c) <= 1e-7 * r
    # every ball enclosed; contacts have zero slack
    slack = r - R - cdist(c[None, :], C)[0]
    assert slack.min() >= -1e-12 * r
    assert np.all(slack[sup] <= 1e-7 * r)


def test_lcg_instance_dual_bracket():
    C, R = workloads.lcg(2000, 20)
    res = oracle.solve(C, R, tol=1e-12)
    check_solution(C, R, res, rtol=1e-10)


def test_cg_path_matches_dense_path():
    C, R = workloads.gaussian(600, 12, 3, 0.05)
    rd = oracle.solve(C, R, tol=1e-12)
    rc = oracle.solve(C, R, tol=1e-12, dense_max_d=4)
    assert rc["cg_iters"] > 0
    assert rc["r"] == pytest.approx(rd["r"], rel=1e-10)
    check_solution(C, R, rc)


# ---------------------------------------------------------------- active set
THETA = 2e-6   # active set: slack r - r_i - ||c - c_i|| <= THETA r (the reading of Sec. 4.2)


def _active_mask(res, m):
    a = np.zeros(m, bool)
    a[res["active"]] = True
    return a


@pytest.mark.parametrize("seed,d,m", [(s, d, m) for s in range(4) for d, m in [(2, 9), (3, 8)]])
def test_active_set_brute_force_tiny(seed, d, m):
    """The returned active set is the set of balls touching the brute-force
    ball (zero slack there), outside the band where the slack is within 1e-6 r
    of THETA r."""
    rng = np.random.default_rng(1000 + seed)
    C = rng.standard_normal((m, d))
    R = rng.uniform(0, 0.5, m)
    rb, cb = brute_force_meb(C, R)
    res = oracle.solve(C, R, tol=1e-12)
    slack = rb - R - np.linalg.norm(C - cb, axis=1)
    expect = slack <= THETA * rb
    sure = np.abs(slack - THETA * rb) > 1e-6 * rb
    assert expect.sum() >= 2 and sure.all()
    assert np.array_equal(_active_mask(res, m)[sure], expect[sure])


def test_active_set_two_balls():
    C = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    res = oracle.solve(C, np.array([2.0, 0.25]), tol=1e-12)     # ball 1 inside ball 0
    assert list(res["active"]) == [0]
    res = oracle.solve(np.array([[1.0, 2.0], [4.0, 6.0]]), np.array([0.3, 1.1]), tol=1e-12)
    assert list(res["active"]) == [0, 1]


@pytest.mark.parametrize("n", [3, 6, 10])
def test_active_set_simplex_with_interior_points(n):
    """Vertices of a regular simplex plus points strictly inside it: exactly the
    vertices are active, whatever their order among the balls."""
    rng = np.random.default_rng(n)
    W = rng.dirichlet(np.ones(n), size=4 * n)
    inner = 0.7 * W + 0.3 / n                  # convex combinations, pulled to the centroid
    C = np.vstack([inner[: 2 * n], np.eye(n), inner[2 * n:]])
    res = oracle.solve(C, np.zeros(len(C)), tol=1e-12)
    assert list(res["active"]) == list(range(2 * n, 3 * n))
    assert res["r"] == pytest.approx(math.sqrt((n - 1) / n), rel=1e-10)


def test_multipliers_only_on_active_balls():
    """Complementarity (KKT, Sec. 2): a ball with a nonzero multiplier touches the
    ball, so it is in the active set; balls strictly inside have u = v = 0."""
    C, R = workloads.gaussian(2000, 6, 41, 0.1)
    res = oracle.solve(C, R, tol=1e-12)
    U, V = res["U"], res["V"]
    holders = np.nonzero((U > 1e-9) | (np.linalg.norm(V, axis=1) > 1e-9))[0]
    assert len(holders) >= 2
    assert set(holders.tolist()) <= set(res["active"].tolist())
    slack = res["r"] - R - np.linalg.norm(C - res["c"], axis=1)
    inside = slack > 1e-6 * res["r"]
    assert np.all(U[inside] == 0.0) and np.all(V[inside] == 0.0)


@pytest.mark.parametrize("scale", [1e3, 1e-3])
def test_active_set_threshold_is_relative(scale):
    """Closed form: balls 0, 1 at (-L, 0), (L, 0) with radius 0 give c* = 0,
    r* = L; balls centred at 0 with radius L (1 - k 1e-6) have slack k 1e-6 L.
    Active iff slack <= THETA r*, i.e. k <= 2: an absolute threshold (THETA) or
    any other power of r would move the boundary by orders of magnitude at
    these scales."""
    L = scale
    ks = [0.5, 1.0, 3.5, 10.0, 1.9, 2.2]
    C = np.zeros((2 + len(ks), 2))
    C[0, 0], C[1, 0] = -L, L
    R = np.concatenate([[0.0, 0.0], [L * (1 - k * 1e-6) for k in ks]])
    res = oracle.solve(C, R, tol=1e-12)
    assert res["r"] == pytest.approx(L, rel=1e-10)
    expect = [0, 1] + [2 + j for j, k in enumerate(ks) if k <= 2.0]
    assert list(res["active"]) == expect


def test_solve_does_not_depend_on_thread_count():
    """The solve's sums are chunk sums added in chunk order (ORC_CHUNK balls per
    chunk), so one thread and many give bit-identical results."""
    C, R = workloads.cube(20_000, 12, 5, 0.05)
    n0 = oracle.set_threads(0)
    try:
        oracle.set_threads(1)
        a = oracle.solve(C, R, tol=1e-12)
        oracle.set_threads(max(n0, 4))
        b = oracle.solve(C, R, tol=1e-12)
    finally:
        oracle.set_threads(n0)
    assert a["r"] == b["r"] and np.array_equal(a["c"], b["c"])
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["active"], b["active"])
    assert a["passes"] == b["passes"]
