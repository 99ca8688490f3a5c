"""The ragged-batch solver (meb_solve_batch): one persistent launch solving
many independent instances.

* Every instance of a mixed batch (d from 1 to 256, m from 1 to 20,000, ragged
  tails, an all-identical-points instance, the paper's LCG family) matches the
  oracle to the solve's tolerances (radius 1e-8 relative, centre 1e-7 r,
  feasibility 1e-10 r, active set outside the 1e-6 r band).
* An instance's result is bit-identical alone and inside the mix, in any
  position of the batch (the block that solves it runs the same steps in the
  same order whatever else is queued).
* Invalid instances are reported (status -1, MEB_EINVAL) without stopping the
  others; an instance whose support outgrows its block's rows is solved again
  by the multi-block path.
* The tuner picks a configuration per class of d; the tuned batch still
  matches the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu
THETA = 2e-6


def check(C, R, g, o):
    r = o["r"]
    assert g["status"] == 0
    assert abs(g["r"] - r) <= 1e-8 * r, (g["r"], r)
    assert np.linalg.norm(np.asarray(g["c"]) - o["c"]) <= 1e-7 * r
    dmax, _, _, _ = oracle.feas_check(C, R, np.asarray(g["c"]), g["r"], 0.0)
    assert dmax <= 1e-10 * r
    slack = r - R - np.linalg.norm(C - o["c"], axis=1)
    sure = np.abs(slack - THETA * r) > 1e-6 * r
    ga = np.zeros(len(R), bool); ga[np.asarray(g["active"])] = True
    oa = np.zeros(len(R), bool); oa[o["active"]] = True
    assert np.array_equal(ga[sure], oa[sure])
    assert g["n_active"] == len(g["active"])


def mixed_batch():
    inst = [workloads.ragged_instance(k, 77) for k in range(24)]
    inst = [(C[:20_000], R[:20_000]) for C, R in inst]             # keep the oracle quick
    inst.append(workloads.gaussian(10_000, 10, 1001, 0.1))
    inst.append(workloads.lcg(3000, 20))
    inst.append(workloads.cube(4097, 1, 5, 0.05))                  # d = 1
    inst.append((np.array([[0.5, -1.0, 2.0]]), np.array([0.25])))  # m = 1
    inst.append((np.tile([1.5, -2.0], (6, 1)), np.zeros(6)))       # every ball the same point
    inst.append(workloads.cube(257, 111, 9, 0.05))                 # largest dense d, ragged tail
    inst.append(workloads.cube(3000, 130, 10, 0.05))               # CG path
    return inst


def test_batch_matches_oracle_every_instance():
    inst = mixed_batch()
    res = meb.solve_batch(inst)
    assert len(res) == len(inst)
    for (C, R), g in zip(inst, res):
        if C.shape[0] == 1:
            assert g["r"] == R[0] and np.array_equal(g["c"], C[0])
            continue
        if np.all(C == C[0]):
            assert g["r"] == 0.0 and g["n_active"] == len(R)
            continue
        o = oracle.solve(C, R, tol=1e-12)
        check(C, R, g, o)


def test_batch_alone_and_in_the_mix_bit_identical():
    inst = mixed_batch()
    mix = meb.solve_batch(inst)
    rev = meb.solve_batch(inst[::-1])[::-1]                         # other positions, other blocks
    for k in (0, 3, 7, 24, 25, len(inst) - 1):
        alone = meb.solve_batch([inst[k]])[0]
        for other in (mix[k], rev[k]):
            assert alone["r"] == other["r"], k
            assert np.array_equal(alone["c"], other["c"]), k
            assert np.array_equal(alone["active"], other["active"]), k
            assert alone["passes"] == other["passes"], k


def test_batch_device_pointers_match_host():
    torch = pytest.importorskip("torch")
    inst = [workloads.ragged_instance(k, 5) for k in range(6)]
    h = meb.solve_batch(inst)
    dinst = [(torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda()) for C, R in inst]
    g = meb.solve_batch(dinst)
    for a, b in zip(h, g):
        assert a["r"] == b["r"] and np.array_equal(a["c"], b["c"].cpu().numpy())
        assert np.array_equal(a["active"], b["active"].cpu().numpy())


def test_batch_invalid_instance_reported_others_solved():
    inst = [workloads.ragged_instance(k, 11) for k in range(4)]
    C, R = inst[2]
    R = R.copy(); R[5] = np.nan
    inst[2] = (C, R)
    ctx = meb.Context(0)
    items = inst
    with pytest.raises(meb.MebError) as e:
        meb.solve_batch(items, ctx=ctx)
    assert e.value.code == -1
    # the same call, looking at the per-instance results through the C ABI
    import ctypes as ct
    from paper_2605_31425_gb300 import _lib
    its, outs, _keep, flags = _lib._batch_items(items, None)
    infos = (_lib.MebInfo * 4)()
    rc = ctx._lib.meb_solve_batch(ctx._h, 4, its, 0.0, None, flags, infos)
    assert rc == -1 and infos[2].status == -1
    for k in (0, 1, 3):
        C, R = inst[k]
        o = oracle.solve(C, R, tol=1e-12)
        assert infos[k].status == 0 and abs(infos[k].r - o["r"]) <= 1e-8 * o["r"]


def test_batch_support_overflow_falls_back():
    """3000 points on a circle: every point is active with a multiplier, more
    than the block's support rows (2048), so the multi-block path solves it."""
    t = np.linspace(0, 2 * np.pi, 3000, endpoint=False)
    C = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], 1) + np.array([0.3, -0.2, 1.0])
    R = np.zeros(3000)
    ctx = meb.Context(0)
    ctx.reset_stats()
    small = workloads.gaussian(4000, 10, 8, 0.1)    # keeps the batch's support rows at 2048
    res = meb.solve_batch([small, (C, R)], ctx=ctx)
    assert ctx.stats()["batch_fallbacks"] == 1
    assert abs(res[1]["r"] - 1.0) <= 1e-8
    o = oracle.solve(*small, tol=1e-12)
    check(*small, res[0], o)


def test_tune_batch_then_solve():
    inst = [workloads.ragged_instance(k, 21) for k in range(30)]
    inst = [(C[:8000], R[:8000]) for C, R in inst]
    ctx = meb.Context(0)
    table = meb.tune_batch(inst, per_class=3, ctx=ctx)
    assert len(table) == 6
    for half, tpvb, nsvb in table[:5]:
        assert half in (0, 1) and tpvb >= 1 and 1 <= nsvb <= 16
    res = meb.solve_batch(inst, ctx=ctx)
    for (C, R), g in zip(inst[:10], res[:10]):
        check(C, R, g, oracle.solve(C, R, tol=1e-12))
