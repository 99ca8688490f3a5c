"""The chunked copy-in of host centres, and centres off a 16-byte boundary.

* Host centres of more than 128 MB are copied in chunks, the shadow sweep of
  each chunk running under the copy of the next; the solve is bit-identical to
  one on device-resident inputs, and an invalid ball in the last chunk is
  still reported.
* Device centres 8 bytes past a 16-byte boundary (any float64 array the API
  accepts): no kernel may assume more alignment than 8 bytes for them, and a
  solve, an evaluation of Psi and a feasibility check on them are
  bit-identical to the same calls on aligned centres.
"""
import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu


def offset_view(C):
    """C on the device 8 bytes past a 16-byte boundary."""
    import torch
    m, d = C.shape
    buf = torch.empty(m * d + 1, dtype=torch.float64, device="cuda")
    v = buf[1:].view(m, d)
    v.copy_(torch.from_numpy(np.ascontiguousarray(C)))
    assert v.data_ptr() % 16 == 8
    return v


def same_solve(a, b):
    assert a["status"] == 0 and b["status"] == 0
    assert a["r"] == b["r"]
    assert np.array_equal(np.asarray(a["c"].cpu()), np.asarray(b["c"].cpu()))
    assert np.array_equal(np.sort(np.asarray(a["active"].cpu())),
                          np.sort(np.asarray(b["active"].cpu())))
    assert a["passes"] == b["passes"] and a["fp64_rows"] == b["fp64_rows"]


# m leaves a ragged last shadow block of 64 balls, except 12,800
@pytest.mark.parametrize("m,d,seed", [(10_007, 100, 41), (7_001, 128, 42), (20_011, 2, 43),
                                      (12_800, 10, 44), (3_001, 257, 51)])
def test_unaligned_centres_bit_identical(m, d, seed):
    import torch
    C, R = workloads.cube(m, d, seed, 0.05)
    dR = torch.from_numpy(R).cuda()
    ga = meb.solve(torch.from_numpy(C).cuda(), dR, ctx=meb.Context(0))
    gb = meb.solve(offset_view(C), dR, ctx=meb.Context(0))
    same_solve(ga, gb)
    if m * d <= 1_000_000:
        o = oracle.solve(C, R, tol=1e-12)
        assert abs(ga["r"] - o["r"]) <= 1e-8 * o["r"]


def test_unaligned_centres_eval_and_feas_bit_identical():
    import torch
    m, d = 9_001, 64
    C, R = workloads.cube(m, d, 45, 0.05)
    rng = np.random.default_rng(46)
    c = C.mean(axis=0) + 0.01 * rng.standard_normal(d)
    r = float(np.max(np.linalg.norm(C - c, axis=1) + R)) * 0.999
    x = np.concatenate([[r], c])
    U = np.zeros(m)
    V = np.zeros((m, d))
    dR = torch.from_numpy(R).cuda()
    outs = []
    for dC in (torch.from_numpy(C).cuda(), offset_view(C)):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        ev = meb.eval_alm(dC, dR, t(x), t(x), t(U), t(V), 2.0, 0.5, ctx=meb.Context(0))
        fc = meb.feas_check(dC, dR, t(c), r, 1e-12, ctx=meb.Context(0))
        outs.append((ev, fc))
    (ea, fa), (eb, fb) = outs
    for k in ea:
        va, vb = ea[k], eb[k]
        if hasattr(va, "cpu"):
            assert torch.equal(va, vb), k
        else:
            assert np.array_equal(np.asarray(va), np.asarray(vb)), k
    assert fa[0] == fb[0] and fa[1] == fb[1] and fa[3] == fb[3]
    assert torch.equal(fa[2], fb[2])


@pytest.mark.parametrize("m,d,seed", [(200_003, 100, 47), (10_007, 2000, 48)])
def test_chunked_copy_in_bit_identical(m, d, seed):
    import torch
    C, R = workloads.cube(m, d, seed, 0.05)
    assert C.nbytes > (128 << 20)
    gd = meb.solve(torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda(), ctx=meb.Context(0))
    gh = meb.solve(C, R, ctx=meb.Context(0))
    assert gh["status"] == 0
    assert gh["r"] == gd["r"]
    assert np.array_equal(gh["c"], gd["c"].cpu().numpy())
    assert np.array_equal(np.sort(gh["active"]), np.sort(gd["active"].cpu().numpy()))


@pytest.mark.parametrize("what", ["nan_centre", "negative_radius"])
def test_chunked_copy_in_reports_invalid_last_chunk(what):
    m, d = 200_003, 100
    C, R = workloads.cube(m, d, 49, 0.05)
    if what == "nan_centre":
        C[m - 2, d - 1] = np.nan
    else:
        R[m - 1] = -1.0
    ctx = meb.Context(0)
    with pytest.raises(meb.MebError) as e:
        meb.solve(C, R, ctx=ctx)
    assert e.value.code == -1          # MEB_EINVAL
    C2, R2 = workloads.cube(20_000, 10, 50, 0.05)
    assert meb.solve(C2, R2, ctx=ctx)["status"] == 0
