"""The mixed-precision reduction pipeline (Sec. 4.2): a low-precision ripALM
(FP32 rows from the FP32 shadow) to tol 1e-2 on all balls, the certified
screen of the balls within tol_red of the boundary, the FP64 ripALM on that
reduced set warm-started from the low-precision point, and the full FP64
feasibility pass that adds violated balls back.

* The result is the oracle's (radius 1e-8 relative, centre 1e-7 r, every ball
  enclosed to 1e-10 r, active set outside the 1e-6 r band), on the dense and
  the matrix-free Newton paths.
* The reduced set is a small part of the balls on these workloads.
* A screening threshold far too tight forces re-add rounds; the result is
  still the oracle's.
* The reported KKT residuals equal the oracle's at the returned point with the
  reported multipliers (their indices mapped back to the whole instance).
"""
import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
THETA = 2e-6


def mixed_params(**kw):
    p = meb.params_default()
    p.mixed = 1
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def check(C, R, g, o):
    r = o["r"]
    assert g["status"] == 0
    assert abs(g["r"] - r) <= 1e-8 * r, (g["r"], r)
    assert np.linalg.norm(g["c"] - o["c"]) <= 1e-7 * r
    dmax, _, _, _ = oracle.feas_check(C, R, g["c"], g["r"], 0.0)
    assert dmax <= 1e-10 * r
    slack = r - R - np.linalg.norm(C - o["c"], axis=1)
    sure = np.abs(slack - THETA * r) > 1e-6 * r
    ga = np.zeros(len(R), bool); ga[np.asarray(g["active"])] = True
    oa = np.zeros(len(R), bool); oa[o["active"]] = True
    assert np.array_equal(ga[sure], oa[sure])


CASES = {
    "gaussian_1e4_10": lambda: workloads.gaussian(10_000, 10, 1001, 0.1),
    "cube_5e4_100": lambda: workloads.cube(50_000, 100, 7, 0.05),
    "lcg_5000_20": lambda: workloads.lcg(5000, 20),
    "cube_5000_224": lambda: workloads.cube(5000, 224, 11, 0.05),
    "sphere_6000_300": lambda: workloads.sphere(6000, 300, 4)[:2],
}


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_matches_oracle(case):
    C, R = CASES[case]()
    g = meb.solve(C, R, params=mixed_params())
    o = oracle.solve(C, R, tol=1e-12)
    check(C, R, g, o)
    assert g["lowp_passes"] > 0
    assert g["n_reduced"] <= len(R)
    if case.startswith(("gaussian", "cube")):
        assert g["n_reduced"] < len(R) // 2        # the FP64 solve ran on a reduced set


def test_mixed_readd_rounds_still_exact():
    C, R = workloads.cube(30_000, 40, 5, 0.05)
    g = meb.solve(C, R, params=mixed_params(tol_red=1e-9))
    assert g["readd_rounds"] >= 1
    o = oracle.solve(C, R, tol=1e-12)
    check(C, R, g, o)


def test_mixed_kkt_with_mapped_multipliers():
    C, R = workloads.gaussian(20_000, 12, 3, 0.1)
    m, d = C.shape
    ctx = meb.Context(0)
    g = meb.solve(C, R, params=mixed_params(), ctx=ctx)
    idx, u, v = ctx.multipliers()
    assert np.all(np.diff(idx) > 0) and idx.max() < m
    U = np.zeros(m); V = np.zeros((m, d))
    U[idx] = u; V[idx] = v
    k_orc = oracle.kkt(C, R, g["r_alm"], g["c"], U, V)
    n = len(idx)
    su = np.sum(np.abs(u)); sv = np.sum(np.linalg.norm(v, axis=1)); r = g["r"]
    tol = np.array([(n + 16) * EPS * su, (n + d + 16) * EPS * sv, (d + 16) * EPS * 4 * r,
                    (d + 16) * EPS * max(su, 1.0), (d + 16) * EPS * 4 * r * max(su, 1.0)])
    assert np.all(np.abs(np.asarray(g["kkt"]) - k_orc) <= tol), (g["kkt"], k_orc)


def test_mixed_same_as_plain_solve_within_tolerance():
    C, R = workloads.cube(80_000, 64, 9, 0.05)
    a = meb.solve(C, R)
    b = meb.solve(C, R, params=mixed_params())
    assert abs(a["r"] - b["r"]) <= 1e-9 * a["r"]
    assert np.linalg.norm(a["c"] - b["c"]) <= 1e-7 * a["r"]
