"""ctypes binding of ``meb_oracle.c`` (test infrastructure; see the package docstring).

Every function marshals numpy float64 arrays to the plain C oracle and back;
the arithmetic is all in the C file.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "meb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmeb_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ct.POINTER(ct.c_double)
_I64 = ct.POINTER(ct.c_int64)


class OracleParams(ct.Structure):
    _fields_ = [
        ("tol", ct.c_double), ("rho", ct.c_double), ("sigma0", ct.c_double),
        ("sigma_max", ct.c_double), ("sigma_growth", ct.c_double),
        ("sigma_ratio", ct.c_double), ("tau", ct.c_double),
        ("armijo_mu", ct.c_double), ("active_theta", ct.c_double),
        ("max_outer", ct.c_int), ("max_ssn", ct.c_int), ("max_backtrack", ct.c_int),
        ("dense_max_d", ct.c_int), ("max_cg", ct.c_int),
    ]


class _Info(ct.Structure):
    _fields_ = [
        ("r", ct.c_double), ("r_alm", ct.c_double), ("kkt", ct.c_double * 5),
        ("kkt_max", ct.c_double), ("delta_max", ct.c_double), ("scale", ct.c_double),
        ("n_active", ct.c_int64),
        ("outer_iters", ct.c_int32), ("ssn_iters", ct.c_int32), ("cg_iters", ct.c_int32),
        ("passes", ct.c_int32), ("backtracks", ct.c_int32), ("status", ct.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (plain -O2, no fast-math,
    no contraction into FMAs; OpenMP for the chunk loops when gcc has it, else
    one thread: the results are the same)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp,
                _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            lib.orc_params_default.argtypes = [ct.POINTER(OracleParams)]
            lib.orc_set_threads.argtypes = [ct.c_int]
            lib.orc_set_threads.restype = ct.c_int
            lib.orc_soc_project.argtypes = [ct.c_double, _D, ct.c_int, _D, _D]
            lib.orc_soc_project.restype = ct.c_int
            lib.orc_soc_dist.argtypes = [ct.c_double, _D, ct.c_int]
            lib.orc_soc_dist.restype = ct.c_double
            lib.orc_soc_jacobian.argtypes = [ct.c_double, _D, ct.c_int, _D]
            lib.orc_soc_jacobian.restype = ct.c_int
            lib.orc_eval_alm.argtypes = [ct.c_int64, ct.c_int, _D, _D, _D, _D, _D, _D,
                                         ct.c_double, ct.c_double, _D, _D, _D, _D, _D,
                                         _D, _D, _I64]
            lib.orc_feas_check.argtypes = [ct.c_int64, ct.c_int, _D, _D, _D, ct.c_double,
                                           ct.c_double, _D, _I64, _I64, ct.c_int64, _I64]
            lib.orc_kkt.argtypes = [ct.c_int64, ct.c_int, _D, _D, ct.c_double, _D, _D, _D, _D]
            lib.orc_solve.argtypes = [ct.c_int64, ct.c_int, _D, _D, ct.POINTER(OracleParams),
                                      _D, _D, _D, _I64, ct.c_int64, ct.POINTER(_Info)]
            lib.orc_solve.restype = ct.c_int
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int = 0) -> int:
    """Threads of the solve's chunk loops (0: leave the default); returns the
    count in use.  Results do not depend on it."""
    return _load().orc_set_threads(int(n))


def params_default() -> OracleParams:
    p = OracleParams()
    _load().orc_params_default(ct.byref(p))
    return p


def soc_project(a: float, b):
    b = _f64(b)
    pb = np.empty_like(b)
    pa = ct.c_double()
    cs = _load().orc_soc_project(float(a), _p(b), b.size, ct.byref(pa), _p(pb))
    return pa.value, pb, cs


def soc_dist(a: float, b) -> float:
    b = _f64(b)
    return _load().orc_soc_dist(float(a), _p(b), b.size)


def soc_jacobian(a: float, b):
    b = _f64(b)
    P = np.empty((b.size + 1, b.size + 1))
    cs = _load().orc_soc_jacobian(float(a), _p(b), b.size, _p(P))
    return P, cs


def eval_alm(C, R, x, xbar, U, V, sigma, tau, q=None, want_H=False):
    """One evaluation of Psi, grad, (U+, V+), Hq and H (Sec. 4 / Algorithm 2)."""
    C = _f64(C); R = _f64(R); x = _f64(x); xbar = _f64(xbar)
    m, d = C.shape
    U = _f64(U) if U is not None else np.zeros(m)
    V = _f64(V) if V is not None else np.zeros((m, d))
    q = _f64(q) if q is not None else None
    psi = ct.c_double()
    grad = np.empty(d + 1)
    Up = np.empty(m)
    Vp = np.empty((m, d))
    Hq = np.empty(d + 1) if q is not None else None
    H = np.empty((d + 1, d + 1)) if want_H else None
    counts = np.zeros(3, dtype=np.int64)
    _load().orc_eval_alm(m, d, _p(C), _p(R), _p(x), _p(xbar), _p(U), _p(V), float(sigma),
                         float(tau), _p(q), ct.byref(psi), _p(grad), _p(Up), _p(Vp), _p(Hq),
                         _p(H), counts.ctypes.data_as(_I64))
    return dict(psi=psi.value, grad=grad, Uplus=Up, Vplus=Vp, Hq=Hq, H=H, counts=counts)


def feas_check(C, R, c, r, eps, cap=None):
    """Sec. 4.2: Delta_max, argmax and the ascending violated list."""
    C = _f64(C); R = _f64(R); c = _f64(c)
    m, d = C.shape
    cap = m if cap is None else cap
    viol = np.empty(max(cap, 1), dtype=np.int64)
    dm = ct.c_double(); am = ct.c_int64(); nv = ct.c_int64()
    _load().orc_feas_check(m, d, _p(C), _p(R), _p(c), float(r), float(eps), ct.byref(dm),
                           ct.byref(am), viol.ctypes.data_as(_I64), cap, ct.byref(nv))
    return dm.value, am.value, viol[:min(nv.value, cap)].copy(), nv.value


def kkt(C, R, r, c, U, V):
    """Sec. 5: the five KKT residuals."""
    C = _f64(C); R = _f64(R); c = _f64(c); U = _f64(U); V = _f64(V)
    m, d = C.shape
    k = np.empty(5)
    _load().orc_kkt(m, d, _p(C), _p(R), float(r), _p(c), _p(U), _p(V), _p(k))
    return k


def solve(C, R, params: OracleParams | None = None, **overrides):
    """Algorithms 1 + 2 on the whole instance; returns a dict of results."""
    C = _f64(C); R = _f64(R)
    if C.ndim == 1:
        C = C.reshape(-1, 1)
    m, d = C.shape
    p = params if params is not None else params_default()
    for k, v in overrides.items():
        setattr(p, k, v)
    c = np.empty(d)
    U = np.empty(m)
    V = np.empty((m, d))
    act = np.empty(m, dtype=np.int64)
    info = _Info()
    rc = _load().orc_solve(m, d, _p(C), _p(R), ct.byref(p), _p(c), _p(U), _p(V),
                           act.ctypes.data_as(_I64), m, ct.byref(info))
    if rc < 0:
        raise ValueError("oracle: invalid input")
    return dict(
        r=info.r, r_alm=info.r_alm, c=c, U=U, V=V, active=act[:info.n_active].copy(),
        kkt=np.array(info.kkt[:]), kkt_max=info.kkt_max, delta_max=info.delta_max,
        scale=info.scale, outer_iters=info.outer_iters, ssn_iters=info.ssn_iters,
        cg_iters=info.cg_iters, passes=info.passes, backtracks=info.backtracks,
        status=info.status,
    )
