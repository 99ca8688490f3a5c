"""The allocation-free feasibility check against the context-based one.

meb_feas_check_noalloc serves callers that cannot call cudaMalloc (engines whose
device memory belongs to their own pool or to another framework's caching
allocator, loops that forbid allocation once running): it keeps its scratch in a
fixed static device array.  This file is collected last, so a run that stops at
its first failure has already run every other test; it also passes alone in a
fresh process.  Two calls in a row check that the shared scratch left by one call
does not leak into the next.
"""
import numpy as np
import pytest

import oracle
import paper_2605_31425_gb300 as meb
from paper_2605_31425_gb300 import workloads

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def test_noalloc_matches_feas_check_twice():
    torch = pytest.importorskip("torch")
    m, d = 300_007, 24
    C, R = workloads.cube(m, d, 31, 0.05)
    C[m // 3] = C[17]; R[m // 3] = R[17]          # a duplicated ball: ties -> lower index
    dC = torch.from_numpy(C).cuda(); dR = torch.from_numpy(R).cuda()
    rng = np.random.default_rng(5)
    for call in range(2):
        c = 0.05 * rng.standard_normal(d)
        e = np.linalg.norm(C - c, axis=1) + R
        r = float(np.quantile(e, 0.999 if call == 0 else 0.99))
        eps = 1e-3 * call
        viol = torch.full((500,), -1, dtype=torch.int64, device="cuda")
        dm, am, nv = meb.feas_check_noalloc(dC, dR, torch.from_numpy(c).cuda(), r, eps, viol)
        torch.cuda.synchronize()
        ref_dm, ref_am, ref_v, ref_nv = meb.feas_check(C, R, c, r, eps)
        assert am == ref_am and nv == ref_nv
        assert abs(dm - ref_dm) <= (d + 8) * EPS * (np.max(e) + abs(r))
        k = min(nv, 500)
        np.testing.assert_array_equal(viol[:k].cpu().numpy(), ref_v[:k])
        assert (viol[k:].cpu().numpy() == -1).all()
        # and against the CPU oracle's definition (Sec. 4.2), not only the GPU
        o_dm, o_am, o_v, o_nv = oracle.feas_check(C, R, c, r, eps)
        assert am == o_am and nv == o_nv
        assert abs(dm - o_dm) <= (d + 8) * EPS * (np.max(e) + abs(r))
        np.testing.assert_array_equal(viol[:k].cpu().numpy(), o_v[:k])


def test_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    C = torch.zeros((4, 5000), dtype=torch.float64, device="cuda")
    R = torch.zeros(4, dtype=torch.float64, device="cuda")
    c = torch.zeros(5000, dtype=torch.float64, device="cuda")
    viol = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(meb.MebError) as e:
        meb.feas_check_noalloc(C, R, c, 1.0, 0.0, viol)
    assert e.value.code == -1


def test_noalloc_rejects_invalid_values():
    torch = pytest.importorskip("torch")
    C, R = workloads.cube(5000, 6, 3, 0.05)
    c = np.zeros(6)
    viol = torch.zeros(8, dtype=torch.int64, device="cuda")
    for bad in ("radius_nan", "radius_neg", "row_inf", "query_nan"):
        Cb, Rb, cb = C.copy(), R.copy(), c.copy()
        if bad == "radius_nan":
            Rb[77] = np.nan
        elif bad == "radius_neg":
            Rb[4000] = -0.5
        elif bad == "row_inf":
            Cb[123, 2] = np.inf
        else:
            cb[1] = np.nan
        with pytest.raises(meb.MebError) as e:
            meb.feas_check_noalloc(torch.from_numpy(Cb).cuda(), torch.from_numpy(Rb).cuda(),
                                   torch.from_numpy(cb).cuda(), 1.0, 0.0, viol)
        assert e.value.code == -1, bad
    with pytest.raises(ValueError):     # float32 centres: refused before any launch
        meb.feas_check_noalloc(torch.from_numpy(C).float().cuda(), torch.from_numpy(R).cuda(),
                               torch.from_numpy(c).cuda(), 1.0, 0.0, viol)
