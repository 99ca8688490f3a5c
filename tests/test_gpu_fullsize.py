"""Full-size GPU parity on the benchmark instances, in the bench's launch
configuration (a context on the current torch stream, inputs resident on the
device).

cube 2e6 x 100: the stored oracle solution (tests/golden/cube_m2e6_d100.json,
oracle run to KKT_max <= 1e-12) gives the radius, centre and active set; the
returned ball is checked over all 2e6 rows by the oracle's own feasibility
pass, and the active set in both directions.

sphere 2e5 x 2000 (r_i = 0, matrix-free Newton path): closed form r* = 1 at
the generating centre (the oracle cannot solve this size in seconds).

gaussian 1e4 x 10: the oracle solves it directly.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _device_solve(C, R):
    torch = pytest.importorskip("torch")
    stream = torch.cuda.current_stream()
    ctx = meb.Context(0, stream.cuda_stream)
    dC = torch.from_numpy(C).cuda()
    dR = torch.from_numpy(R).cuda()
    res = meb.solve(dC, dR, ctx=ctx)
    torch.cuda.synchronize()
    res["c"] = res["c"].cpu().numpy()
    res["active"] = res["active"].cpu().numpy()
    return res


def test_cube_m2e6_d100_against_stored_oracle():
    C, R = workloads.workload("cube_m2e6_d100")
    with open(os.path.join(HERE, "golden", "cube_m2e6_d100.json")) as f:
        gold = json.load(f)
    assert gold["input_sha256"] == workloads.digest(C, R)
    g = _device_solve(C, R)
    r = gold["r"]
    assert g["status"] == 0
    assert abs(g["r"] - r) <= 1e-8 * r
    assert np.linalg.norm(g["c"] - np.asarray(gold["c"])) <= 1e-7 * r
    # the returned ball over every row, by the oracle's feasibility pass:
    # enclosed to rounding, and the radius attained
    dmax, amax, _, _ = oracle.feas_check(C, R, g["c"], g["r"], 0.0)
    assert abs(dmax) <= 1e-12 * r
    dg, ag, _, _ = meb.feas_check(C, R, g["c"], g["r"], 0.0)
    assert ag == amax
    # active set at the returned ball, both directions, outside the band where
    # the slack is within 1e-12 r of theta r (rounding of the slack itself)
    theta = 2e-6
    slack = np.empty(len(R))
    for lo in range(0, len(R), 250_000):
        hi = lo + 250_000
        slack[lo:hi] = g["r"] - R[lo:hi] - np.linalg.norm(C[lo:hi] - g["c"], axis=1)
    ga = np.zeros(len(R), bool); ga[g["active"]] = True
    sure = np.abs(slack - theta * g["r"]) > 1e-12 * g["r"]
    assert np.array_equal(ga[sure], (slack <= theta * g["r"])[sure])
    assert g["n_active"] == len(g["active"])
    # against the stored oracle solution, both directions, outside the 1e-6 r band
    oc = np.asarray(gold["c"])
    oa = np.zeros(len(R), bool); oa[np.asarray(gold["active"])] = True
    cand = np.nonzero(ga | oa)[0]
    s_o = r - R[cand] - np.linalg.norm(C[cand] - oc, axis=1)
    far = np.abs(s_o - theta * r) > 1e-6 * r
    assert np.array_equal(ga[cand][far], oa[cand][far])


def test_gaussian_m1e4_d10_against_oracle():
    C, R = workloads.workload("gaussian_m1e4_d10")
    g = _device_solve(C, R)
    o = oracle.solve(C, R, tol=1e-12)
    assert g["status"] == 0
    assert abs(g["r"] - o["r"]) <= 1e-8 * o["r"]
    assert np.linalg.norm(g["c"] - o["c"]) <= 1e-7 * o["r"]
    slack = o["r"] - R - np.linalg.norm(C - o["c"], axis=1)
    sure = np.abs(slack - 2e-6 * o["r"]) > 1e-6 * o["r"]
    ga = np.zeros(len(R), bool); ga[g["active"]] = True
    oa = np.zeros(len(R), bool); oa[o["active"]] = True
    assert np.array_equal(ga[sure], oa[sure])


def test_sphere_m2e5_d2000_closed_form():
    C, R, ctr = workloads.sphere(200_000, 2000, 1003)
    g = _device_solve(C, R)
    assert g["status"] == 0 and g["cg_iters"] > 0
    assert abs(g["r"] - 1.0) <= 1e-8
    assert np.linalg.norm(g["c"] - ctr) <= 1e-7
    # feasibility of the returned ball on a sample, by the oracle
    rng = np.random.default_rng(7)
    sample = rng.choice(len(R), 20_000, replace=False)
    dmax, _, _, _ = oracle.feas_check(C[sample], R[sample], g["c"], g["r"], 0.0)
    assert dmax <= 1e-10
