"""Thin ctypes binding of libmeb (include/meb.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays (host path) or torch CUDA tensors (device path, ``MEB_PTR_DEVICE``) to
pointers and sizes, and results back.  If the library cannot be built or
loaded the calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import threading

import numpy as np

from . import build as _build

MEB_OK, MEB_EINVAL, MEB_ENOMEM, MEB_ECUDA, MEB_ENOTCONV, MEB_ETIMEOUT = 0, -1, -2, -3, -4, -5
MEB_PTR_DEVICE = 1
# context options and screen modes (include/meb.h)
MEB_OPT_SCREEN, MEB_OPT_EVAL_SCREEN, MEB_OPT_EVAL_SHADOW_EXP, MEB_OPT_TICK_LOOP, \
    MEB_OPT_WAIT_CYCLES, MEB_OPT_BATCH_SLOTS, MEB_OPT_RELEASE_SCRATCH, \
    MEB_OPT_BLOCKING_SYNC = 1, 2, 3, 4, 5, 6, 7, 8
SCREEN_MODES = {"fp16": 0, "fp16_bulk": 1, "fp32": 2, "fp64": 3}
MEB_SERVER_SPIN_WAITS, MEB_SERVER_DEVICE_POOL = 1, 2
TICK_LOOPS = {"graph": 0, "host": 1, "while": 2}

_D = ct.POINTER(ct.c_double)
_I64 = ct.POINTER(ct.c_int64)


class MebParams(ct.Structure):
    _fields_ = [
        ("tol", ct.c_double), ("rho", ct.c_double), ("sigma0", ct.c_double),
        ("sigma_max", ct.c_double), ("sigma_growth", ct.c_double), ("sigma_ratio", ct.c_double),
        ("tau", ct.c_double), ("armijo_mu", ct.c_double), ("active_theta", ct.c_double),
        ("max_outer", ct.c_int32), ("max_ssn", ct.c_int32), ("max_backtrack", ct.c_int32),
        ("dense_max_d", ct.c_int32), ("max_cg", ct.c_int32), ("newton_fp64", ct.c_int32),
        ("mixed", ct.c_int32), ("max_readd", ct.c_int32), ("tol_lp", ct.c_double),
        ("tol_red", ct.c_double),
    ]


class MebInfo(ct.Structure):
    _fields_ = [
        ("r", ct.c_double), ("r_alm", ct.c_double), ("kkt", ct.c_double * 5),
        ("kkt_max", ct.c_double), ("delta_max", ct.c_double), ("scale", ct.c_double),
        ("n_active", ct.c_int64), ("fp64_rows", ct.c_int64),
        ("outer_iters", ct.c_int32), ("ssn_iters", ct.c_int32), ("cg_iters", ct.c_int32),
        ("passes", ct.c_int32), ("backtracks", ct.c_int32), ("status", ct.c_int32),
        ("newton_inverses", ct.c_int32), ("newton_fp64", ct.c_int32),
        ("n_reduced", ct.c_int64), ("readd_rounds", ct.c_int32), ("lowp_passes", ct.c_int32),
    ]


class MebBatchItem(ct.Structure):
    _fields_ = [
        ("centers", _D), ("radii", _D), ("m", ct.c_int64), ("d", ct.c_int32),
        ("reserved", ct.c_int32), ("c_out", _D), ("active_idx", _I64), ("active_cap", ct.c_int64),
    ]


class MebServerConfig(ct.Structure):
    _fields_ = [
        ("budget_bytes", ct.c_int64), ("large_balls", ct.c_int64), ("small_workers", ct.c_int32),
        ("large_workers", ct.c_int32), ("max_group", ct.c_int32), ("flags", ct.c_int32),
    ]


class MebServerStats(ct.Structure):
    _fields_ = [
        ("submitted", ct.c_int64), ("completed", ct.c_int64), ("failed", ct.c_int64),
        ("launches", ct.c_int64), ("in_use_bytes", ct.c_int64), ("peak_bytes", ct.c_int64),
        ("pending", ct.c_int64),
    ]


class MebStats(ct.Structure):
    _fields_ = [
        ("kernel_launches", ct.c_int64), ("pass_launches", ct.c_int64), ("pass_ms", ct.c_double),
        ("pass_balls", ct.c_int64), ("pass_fp64_rows", ct.c_int64), ("pass_bytes", ct.c_int64),
        ("batch_instances", ct.c_int64), ("batch_fallbacks", ct.c_int64),
        ("phase_ms", ct.c_double * 4),
    ]


class MebError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmeb error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load():
    """Build (if stale) and load libmeb.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ct.CDLL(path)
            lib.meb_create.argtypes = [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_void_p]
            lib.meb_create.restype = ct.c_int
            lib.meb_destroy.argtypes = [ct.c_void_p]
            lib.meb_params_default.argtypes = [ct.POINTER(MebParams)]
            lib.meb_last_error.argtypes = [ct.c_void_p]
            lib.meb_last_error.restype = ct.c_char_p
            lib.meb_solve.argtypes = [ct.c_void_p, _D, _D, ct.c_int64, ct.c_int32, ct.c_double,
                                      ct.POINTER(MebParams), ct.c_uint, _D, _I64, ct.c_int64,
                                      ct.POINTER(MebInfo)]
            lib.meb_solve.restype = ct.c_int
            lib.meb_eval_alm.argtypes = [ct.c_void_p, _D, _D, ct.c_int64, ct.c_int32, _D, _D, _D,
                                         _D, ct.c_double, ct.c_double, _D, ct.c_uint, _D, _D, _D,
                                         _D, _D, _D, _I64]
            lib.meb_eval_alm.restype = ct.c_int
            lib.meb_feas_check.argtypes = [ct.c_void_p, _D, _D, ct.c_int64, ct.c_int32, _D,
                                           ct.c_double, ct.c_double, ct.c_uint, _D, _I64, _I64,
                                           ct.c_int64, _I64]
            lib.meb_feas_check.restype = ct.c_int
            lib.meb_feas_check_noalloc.argtypes = [_D, _D, ct.c_int64, ct.c_int32, _D, ct.c_double,
                                                   ct.c_double, ct.c_void_p, _D, _I64, _I64,
                                                   ct.c_int64, _I64]
            lib.meb_feas_check_noalloc.restype = ct.c_int
            lib.meb_set_option.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int64]
            lib.meb_set_option.restype = ct.c_int
            lib.meb_get_multipliers.argtypes = [ct.c_void_p, ct.c_uint, _I64, _D, _D, ct.c_int64,
                                                _I64]
            lib.meb_get_multipliers.restype = ct.c_int
            lib.meb_solve_batch.argtypes = [ct.c_void_p, ct.c_int32, ct.POINTER(MebBatchItem),
                                             ct.c_double, ct.POINTER(MebParams), ct.c_uint,
                                             ct.POINTER(MebInfo)]
            lib.meb_solve_batch.restype = ct.c_int
            lib.meb_tune_batch.argtypes = [ct.c_void_p, ct.c_int32, ct.POINTER(MebBatchItem),
                                           ct.c_int32, ct.c_uint, ct.POINTER(ct.c_int32)]
            lib.meb_tune_batch.restype = ct.c_int
            lib.meb_footprint.argtypes = [ct.c_int64, ct.c_int32, ct.c_int32, _I64]
            lib.meb_footprint.restype = ct.c_int
            lib.meb_server_create.argtypes = [ct.POINTER(ct.c_void_p), ct.c_int,
                                              ct.POINTER(MebServerConfig), ct.POINTER(MebParams)]
            lib.meb_server_create.restype = ct.c_int
            lib.meb_server_submit.argtypes = [ct.c_void_p, _D, _D, ct.c_int64, ct.c_int32, _D, _I64,
                                              ct.c_int64, ct.POINTER(MebInfo), _I64]
            lib.meb_server_submit.restype = ct.c_int
            lib.meb_server_wait.argtypes = [ct.c_void_p, ct.c_int64, ct.c_double,
                                            ct.POINTER(ct.c_int), ct.POINTER(ct.c_double)]
            lib.meb_server_wait.restype = ct.c_int
            lib.meb_server_get_stats.argtypes = [ct.c_void_p, ct.POINTER(MebServerStats)]
            lib.meb_server_get_stats.restype = ct.c_int
            lib.meb_server_destroy.argtypes = [ct.c_void_p]
            lib.meb_set_profiling.argtypes = [ct.c_void_p, ct.c_int]
            lib.meb_reset_stats.argtypes = [ct.c_void_p]
            lib.meb_get_stats.argtypes = [ct.c_void_p, ct.POINTER(MebStats)]
            _lib = lib
    return _lib


def params_default() -> MebParams:
    p = MebParams()
    load().meb_params_default(ct.byref(p))
    return p


class Context:
    """One libmeb context (device + stream).  ``stream`` is a raw cudaStream_t
    handle (int) or None for a private stream.  Keyword options map to
    meb_set_option: screen ("fp16", "fp16_bulk", "fp32", "fp64"), eval_screen
    (same names), eval_shadow_exp (int), tick_loop ("graph", "host", "while"),
    wait_cycles (int), batch_slots, release_scratch, blocking_sync (0 or 1)."""

    def __init__(self, device: int = 0, stream: int | None = None, **options):
        self._lib = load()
        h = ct.c_void_p()
        rc = self._lib.meb_create(ct.byref(h), int(device), ct.c_void_p(stream) if stream else None)
        if rc != MEB_OK:
            raise MebError(rc, "meb_create failed")
        self._h = h
        self.device = device
        for k, v in options.items():
            self.set_option(k, v)

    def set_option(self, name: str, value):
        table = {"screen": (MEB_OPT_SCREEN, SCREEN_MODES),
                 "eval_screen": (MEB_OPT_EVAL_SCREEN, SCREEN_MODES),
                 "eval_shadow_exp": (MEB_OPT_EVAL_SHADOW_EXP, None),
                 "tick_loop": (MEB_OPT_TICK_LOOP, TICK_LOOPS),
                 "wait_cycles": (MEB_OPT_WAIT_CYCLES, None),
                 "batch_slots": (MEB_OPT_BATCH_SLOTS, None),
                 "release_scratch": (MEB_OPT_RELEASE_SCRATCH, None),
                 "blocking_sync": (MEB_OPT_BLOCKING_SYNC, None)}
        if name not in table:
            raise ValueError(f"unknown option {name!r}")
        opt, names = table[name]
        val = names[value] if names is not None and isinstance(value, str) else int(value)
        self._check(self._lib.meb_set_option(self._h, opt, val))

    def multipliers(self, cap: int | None = None):
        """meb_get_multipliers on host arrays: (idx, u, v) of the last solve's
        final point (balls with nonzero multipliers, ascending)."""
        n = ct.c_int64()
        self._check(self._lib.meb_get_multipliers(self._h, 0, None, None, None, 0, ct.byref(n)))
        k = n.value if cap is None else min(cap, n.value)
        d = self._last_d
        idx = np.empty(max(k, 1), dtype=np.int64)
        u = np.empty(max(k, 1))
        v = np.empty((max(k, 1), d))
        self._check(self._lib.meb_get_multipliers(self._h, 0, idx.ctypes.data_as(_I64),
                                                  u.ctypes.data_as(_D), v.ctypes.data_as(_D),
                                                  k, ct.byref(n)))
        return idx[:k], u[:k], v[:k]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.meb_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_profiling(self, on: bool):
        self._check(self._lib.meb_set_profiling(self._h, 1 if on else 0))

    def reset_stats(self):
        self._check(self._lib.meb_reset_stats(self._h))

    def stats(self) -> dict:
        st = MebStats()
        self._check(self._lib.meb_get_stats(self._h, ct.byref(st)))
        out = {k: getattr(st, k) for k, _ in MebStats._fields_}
        out["phase_ms"] = list(st.phase_ms)
        return out

    def _check(self, rc: int, ok=(MEB_OK,)):
        if rc not in ok:
            raise MebError(rc, self._lib.meb_last_error(self._h).decode())
        return rc


_default_ctx = {}


def default_context(device: int = 0, stream: int | None = None) -> Context:
    key = (device, stream)
    if key not in _default_ctx:
        _default_ctx[key] = Context(device, stream)
    return _default_ctx[key]


# ---------------------------------------------------------------- marshalling
def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _check_dev(name, t, shape, dtype="float64"):
    """A device-path argument must be a contiguous CUDA tensor of the given
    dtype and shape on the current device: the kernels read exactly that many
    elements from its pointer."""
    import torch
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != "torch." + dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, not the current device")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _ptr(a):
    """(pointer, keepalive) of a float64/int64 array: numpy (host) or torch CUDA."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), a
    return a.ctypes.data, a


def _as_d(p):
    return ct.cast(p, _D) if p is not None else None


def _as_i(p):
    return ct.cast(p, _I64) if p is not None else None


def _host_f64(a):
    if hasattr(a, "data_ptr") and not getattr(a, "is_cuda", False):
        # a torch CPU tensor (possibly pinned): keep it, pass its pointer
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise ValueError("host tensors must be contiguous float64")
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _ctx_for(device_path: bool, ctx: Context | None) -> Context:
    if ctx is not None:
        return ctx
    if device_path:
        import torch
        dev = torch.cuda.current_device()
        return default_context(dev, torch.cuda.current_stream(dev).cuda_stream)
    return default_context(0, None)


def solve(centers, radii, tol: float = 0.0, params: MebParams | None = None,
          active_cap: int | None = None, ctx: Context | None = None, allow_notconv=False):
    """meb_solve.  numpy inputs: host path (results in numpy).  torch CUDA float64
    tensors: device path (c is a CUDA tensor, active a CUDA int64 tensor)."""
    dev = _is_torch_cuda(centers)
    if dev:
        import torch
        if centers.dim() != 2:
            raise ValueError("centers must be m x d")
        m, d = centers.shape
        _check_dev("centers", centers, (m, d))
        _check_dev("radii", radii, (m,))
        c_out = torch.empty(d, dtype=torch.float64, device=centers.device)
        cap = m if active_cap is None else active_cap
        act = torch.empty(max(cap, 1), dtype=torch.int64, device=centers.device)
        C, R = centers, radii
    else:
        C = _host_f64(centers)
        if C.ndim == 1:
            C = C.reshape(-1, 1)
        R = _host_f64(radii)
        m, d = C.shape
        c_out = np.empty(d)
        cap = m if active_cap is None else active_cap
        act = np.empty(max(cap, 1), dtype=np.int64)
    if R.shape[0] != m:
        raise ValueError("radii must have m entries")
    cx = _ctx_for(dev, ctx)
    info = MebInfo()
    pc, _k1 = _ptr(C)
    pr, _k2 = _ptr(R)
    po, _k3 = _ptr(c_out)
    pa, _k4 = _ptr(act)
    rc = cx._lib.meb_solve(cx._h, _as_d(pc), _as_d(pr), m, d, float(tol),
                           ct.byref(params) if params is not None else None,
                           MEB_PTR_DEVICE if dev else 0, _as_d(po), _as_i(pa), cap,
                           ct.byref(info))
    cx._last_d = d
    cx._check(rc, ok=(MEB_OK, MEB_ENOTCONV) if allow_notconv else (MEB_OK,))
    na = int(info.n_active)
    return dict(
        r=info.r, r_alm=info.r_alm, c=c_out, active=act[:min(na, cap)], n_active=na,
        kkt=list(info.kkt), kkt_max=info.kkt_max, delta_max=info.delta_max, scale=info.scale,
        fp64_rows=int(info.fp64_rows), outer_iters=info.outer_iters, ssn_iters=info.ssn_iters,
        cg_iters=info.cg_iters, passes=info.passes, backtracks=info.backtracks,
        status=info.status, rc=rc, newton_inverses=info.newton_inverses,
        newton_fp64=info.newton_fp64, n_reduced=int(info.n_reduced),
        readd_rounds=info.readd_rounds, lowp_passes=info.lowp_passes,
    )


def eval_alm(centers, radii, x, xbar, U, V, sigma, tau, q=None, want_H=False,
             ctx: Context | None = None):
    """meb_eval_alm on host numpy arrays (or torch CUDA tensors)."""
    dev = _is_torch_cuda(centers)
    if dev:
        import torch
        if centers.dim() != 2:
            raise ValueError("centers must be m x d")
        m, d = centers.shape
        for nm, t, shp in (("centers", centers, (m, d)), ("radii", radii, (m,)),
                           ("x", x, (d + 1,)), ("xbar", xbar, (d + 1,)), ("U", U, (m,)),
                           ("V", V, (m, d))):
            _check_dev(nm, t, shp)
        if q is not None:
            _check_dev("q", q, (d + 1,))
        mk = lambda *s: torch.empty(*s, dtype=torch.float64, device=centers.device)  # noqa: E731
        C, R, X, XB, UU, VV, Q = centers, radii, x, xbar, U, V, q
    else:
        C = _host_f64(centers)
        m, d = C.shape
        R, X, XB = _host_f64(radii), _host_f64(x), _host_f64(xbar)
        UU, VV = _host_f64(U), _host_f64(V)
        Q = _host_f64(q) if q is not None else None
        mk = lambda *s: np.empty(s)  # noqa: E731
    grad = mk(d + 1)
    Up = mk(m)
    Vp = mk(m, d)
    Hq = mk(d + 1) if q is not None else None
    H = mk(d + 1, d + 1) if want_H else None
    psi = ct.c_double()
    counts = np.zeros(3, dtype=np.int64)
    cx = _ctx_for(dev, ctx)
    ptrs = [_ptr(a) for a in (C, R, X, XB, UU, VV, Q, grad, Up, Vp, Hq, H)]
    p = [_as_d(t[0]) for t in ptrs]
    rc = cx._lib.meb_eval_alm(cx._h, p[0], p[1], m, d, p[2], p[3], p[4], p[5], float(sigma),
                              float(tau), p[6], MEB_PTR_DEVICE if dev else 0, ct.byref(psi),
                              p[7], p[8], p[9], p[10], p[11], counts.ctypes.data_as(_I64))
    cx._check(rc)
    return dict(psi=psi.value, grad=grad, Uplus=Up, Vplus=Vp, Hq=Hq, H=H, counts=counts)


def feas_check(centers, radii, c, r, eps, cap=None, ctx: Context | None = None):
    """meb_feas_check: (delta_max, argmax, ascending violated indices, n_viol)."""
    dev = _is_torch_cuda(centers)
    if dev:
        import torch
        if centers.dim() != 2:
            raise ValueError("centers must be m x d")
        m, d = centers.shape
        _check_dev("centers", centers, (m, d))
        _check_dev("radii", radii, (m,))
        _check_dev("c", c, (d,))
        cap = m if cap is None else cap
        viol = torch.empty(max(cap, 1), dtype=torch.int64, device=centers.device)
        C, R, cc = centers, radii, c
    else:
        C = _host_f64(centers)
        m, d = C.shape
        R, cc = _host_f64(radii), _host_f64(c)
        cap = m if cap is None else cap
        viol = np.empty(max(cap, 1), dtype=np.int64)
    cx = _ctx_for(dev, ctx)
    dm = ct.c_double()
    am = ct.c_int64()
    nv = ct.c_int64()
    (pc, _a), (pr, _b), (p3, _c), (pv, _d) = _ptr(C), _ptr(R), _ptr(cc), _ptr(viol)
    rc = cx._lib.meb_feas_check(cx._h, _as_d(pc), _as_d(pr), m, d, _as_d(p3), float(r),
                                float(eps), MEB_PTR_DEVICE if dev else 0, ct.byref(dm),
                                ct.byref(am), _as_i(pv), cap, ct.byref(nv))
    cx._check(rc)
    return dm.value, am.value, viol[:min(nv.value, cap)], nv.value


def feas_check_noalloc(centers, radii, c, r, eps, viol, stream: int | None = None):
    """meb_feas_check_noalloc: the allocation-free feasibility check, for callers
    that cannot call cudaMalloc.  centers, radii, c and viol (int64, its length
    is the cap) are torch CUDA tensors on the current device; no context, no
    allocation inside the library.  The work runs on ``stream`` (a raw
    cudaStream_t), by default torch's current stream.  Returns
    (delta_max, argmax, n_viol)."""
    import torch
    lib = load()
    if centers.dim() != 2:
        raise ValueError("centers must be m x d")
    m, d = centers.shape
    _check_dev("centers", centers, (m, d))
    _check_dev("radii", radii, (m,))
    _check_dev("c", c, (d,))
    _check_dev("viol", viol, (viol.numel(),), dtype="int64")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    dm = ct.c_double()
    am = ct.c_int64()
    nv = ct.c_int64()
    rc = lib.meb_feas_check_noalloc(_as_d(centers.data_ptr()), _as_d(radii.data_ptr()), m, d,
                                    _as_d(c.data_ptr()), float(r), float(eps),
                                    ct.c_void_p(stream) if stream else None, ct.byref(dm),
                                    ct.byref(am), _as_i(viol.data_ptr()), int(viol.numel()),
                                    ct.byref(nv))
    if rc != MEB_OK:
        raise MebError(rc, "meb_feas_check_noalloc failed")
    return dm.value, am.value, nv.value


def _info_dict(info):
    return dict(r=info.r, r_alm=info.r_alm, kkt=list(info.kkt), kkt_max=info.kkt_max,
                delta_max=info.delta_max, scale=info.scale, n_active=int(info.n_active),
                fp64_rows=int(info.fp64_rows), outer_iters=info.outer_iters,
                ssn_iters=info.ssn_iters, cg_iters=info.cg_iters, passes=info.passes,
                backtracks=info.backtracks, status=info.status,
                newton_inverses=info.newton_inverses, newton_fp64=info.newton_fp64,
                n_reduced=int(info.n_reduced), readd_rounds=info.readd_rounds,
                lowp_passes=info.lowp_passes)


def _batch_items(instances, active_cap):
    """(items, outputs, keepalive, flags) for a list of (centers, radii): all
    numpy arrays (host path) or all torch CUDA float64 tensors (device path)."""
    n = len(instances)
    dev = n > 0 and _is_torch_cuda(instances[0][0])
    items = (MebBatchItem * max(n, 1))()
    outs, keep = [], []
    for k, (C, R) in enumerate(instances):
        if dev:
            import torch
            if C.dim() != 2:
                raise ValueError("centers must be m x d")
            m, d = C.shape
            _check_dev("centers", C, (m, d))
            _check_dev("radii", R, (m,))
            cap = m if active_cap is None else min(active_cap, m)
            c_out = torch.empty(d, dtype=torch.float64, device=C.device)
            act = torch.empty(max(cap, 1), dtype=torch.int64, device=C.device)
        else:
            C = _host_f64(C)
            if C.ndim == 1:
                C = C.reshape(-1, 1)
            R = _host_f64(R)
            m, d = C.shape
            if R.shape[0] != m:
                raise ValueError("radii must have m entries")
            cap = m if active_cap is None else min(active_cap, m)
            c_out = np.empty(d)
            act = np.empty(max(cap, 1), dtype=np.int64)
        keep += [C, R]
        items[k].centers = _as_d(_ptr(C)[0])
        items[k].radii = _as_d(_ptr(R)[0])
        items[k].m = m
        items[k].d = d
        items[k].c_out = _as_d(_ptr(c_out)[0])
        items[k].active_idx = _as_i(_ptr(act)[0])
        items[k].active_cap = cap
        outs.append((c_out, act, cap))
    return items, outs, keep, (MEB_PTR_DEVICE if dev else 0)


def solve_batch(instances, tol: float = 0.0, params: MebParams | None = None,
                active_cap: int | None = None, ctx: Context | None = None, allow_notconv=False):
    """meb_solve_batch over a list of (centers, radii): one persistent launch
    solving every instance.  Returns one result dict per instance (as solve)."""
    n = len(instances)
    items, outs, _keep, flags = _batch_items(instances, active_cap)
    cx = _ctx_for(flags != 0, ctx)
    infos = (MebInfo * max(n, 1))()
    rc = cx._lib.meb_solve_batch(cx._h, n, items, float(tol),
                                 ct.byref(params) if params is not None else None, flags, infos)
    cx._check(rc, ok=(MEB_OK, MEB_ENOTCONV) if allow_notconv else (MEB_OK,))
    res = []
    for k in range(n):
        r = _info_dict(infos[k])
        c_out, act, cap = outs[k]
        r["c"] = c_out
        r["active"] = act[:min(r["n_active"], cap)]
        res.append(r)
    return res


def tune_batch(instances, per_class: int = 16, ctx: Context | None = None):
    """meb_tune_batch: time the batch solver's candidate configurations on up
    to per_class instances of each class of d and keep the fastest in the
    context.  Returns the chosen table (per class: FP16 shadow, tiles per pass
    block, support blocks; then blocks per SM)."""
    n = len(instances)
    items, _outs, _keep, flags = _batch_items(instances, None)
    cx = _ctx_for(flags != 0, ctx)
    cfg = (ct.c_int32 * 16)()
    cx._check(cx._lib.meb_tune_batch(cx._h, n, items, int(per_class), flags, cfg))
    return [tuple(cfg[3 * c:3 * c + 3]) for c in range(5)] + [cfg[15]]


def footprint(m: int, d: int, batched: bool) -> int:
    """meb_footprint: device scratch bytes of one solve (batched: one instance
    of a batch with per-instance slots)."""
    b = ct.c_int64()
    rc = load().meb_footprint(int(m), int(d), 1 if batched else 0, ct.byref(b))
    if rc != MEB_OK:
        raise MebError(rc, "meb_footprint: size out of range")
    return b.value


class Server:
    """meb_server_*: continuous batching of requests under a device-memory
    budget.  submit() takes host float64 arrays and returns a ticket at once;
    wait(ticket) returns the result dict with its latency (seconds)."""

    def __init__(self, budget_bytes: int, device: int = 0, small_workers: int = 0,
                 large_workers: int = 0, large_balls: int = 0, max_group: int = 0,
                 params: MebParams | None = None, spin_waits: bool = False,
                 device_pool: bool = False):
        self._lib = load()
        flags = (MEB_SERVER_SPIN_WAITS if spin_waits else 0) | \
            (MEB_SERVER_DEVICE_POOL if device_pool else 0)
        cfg = MebServerConfig(int(budget_bytes), int(large_balls), int(small_workers),
                              int(large_workers), int(max_group), flags)
        h = ct.c_void_p()
        rc = self._lib.meb_server_create(ct.byref(h), int(device), ct.byref(cfg),
                                         ct.byref(params) if params is not None else None)
        if rc != MEB_OK:
            raise MebError(rc, "meb_server_create failed")
        self._h = h
        self._req = {}

    def submit(self, centers, radii, active_cap: int | None = None) -> int:
        C = _host_f64(centers)
        R = _host_f64(radii)
        m, d = C.shape
        if R.shape[0] != m:
            raise ValueError("radii must have m entries")
        cap = m if active_cap is None else min(active_cap, m)
        c_out = np.empty(d)
        act = np.empty(max(cap, 1), dtype=np.int64)
        info = MebInfo()
        t = ct.c_int64()
        rc = self._lib.meb_server_submit(self._h, _as_d(_ptr(C)[0]), _as_d(_ptr(R)[0]), m, d,
                                         _as_d(c_out.ctypes.data), _as_i(act.ctypes.data), cap,
                                         ct.byref(info), ct.byref(t))
        if rc != MEB_OK:
            raise MebError(rc, "meb_server_submit failed")
        self._req[t.value] = (C, R, c_out, act, cap, info)   # alive until wait()
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0):
        rc = ct.c_int()
        lat = ct.c_double()
        w = self._lib.meb_server_wait(self._h, int(ticket), float(timeout), ct.byref(rc), ct.byref(lat))
        if w == MEB_ETIMEOUT:
            return None
        if w != MEB_OK:
            raise MebError(w, "meb_server_wait: unknown ticket")
        _C, _R, c_out, act, cap, info = self._req.pop(ticket)
        res = _info_dict(info)
        res.update(c=c_out, active=act[:min(res["n_active"], cap)], rc=rc.value,
                   latency_s=lat.value)
        return res

    def stats(self) -> dict:
        st = MebServerStats()
        self._lib.meb_server_get_stats(self._h, ct.byref(st))
        return {k: getattr(st, k) for k, _ in MebServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.meb_server_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
