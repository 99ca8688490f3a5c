"""Seeded synthetic MEB instances (input generators only).

This module holds no arithmetic of the method.  It is the one module both the
CUDA path's tests/bench and the CPU oracle's tests draw inputs from.  It
imports nothing else from the package, so loading it never loads the CUDA
library.

Uniform draws are built from the raw 64-bit output of numpy's PCG64 as
``(x >> 11) * 2**-53`` followed by at most one exactly-rounded multiply/add,
so they are bit-identical on every platform (x86_64 and aarch64 alike).
Gaussian draws use numpy's ``standard_normal``; instances that use them are
regenerated on the machine that compares against the oracle.

Workloads (the shapes and distributions of the paper's experiments and of
the benchmark configurations):

* ``gaussian``  - centres N(0,1)^d, radii U[0, rmax]       (m=1e4, d=10)
* ``cube``      - centres U[-1,1]^d, radii U[0, rmax]      (m=2e6, d=100)
* ``sphere``    - r_i = 0; half the points exactly on the unit sphere about a
                  random centre, half at centre + N(0, 0.3^2/d I) (norm < 0.99)
                  (m=2e5, d=2000)
* ``lcg``       - the deterministic instance family of Sec. 5 (test instances)
* ``ragged``    - a batch of independent instances: m log-uniform in
                  [100, 100000], d drawn from {2, 3, 16, 64, 256}, centres
                  N(0,1), radii U[0, 0.1]; instance k depends only on (seed, k)
"""
from __future__ import annotations

import hashlib

import numpy as np

_TWO_M53 = float(2.0 ** -53)


def _u01(rng: np.random.Generator, n: int) -> np.ndarray:
    """n doubles in [0,1): k * 2^-53 with k the top 53 bits of a raw draw (exact)."""
    raw = rng.bit_generator.random_raw(n)
    return (raw >> np.uint64(11)).astype(np.float64) * _TWO_M53


def gaussian(m: int, d: int, seed: int, rmax: float = 0.1):
    """Centres i.i.d. N(0,1), radii U[0, rmax]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C = rng.standard_normal((m, d))
    R = _u01(rng, m) * rmax
    return C, R


def cube(m: int, d: int, seed: int, rmax: float = 0.05):
    """Centres U[-1,1]^d (2u-1 is exact), radii U[0, rmax]; bit-reproducible."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C = _u01(rng, m * d).reshape(m, d)
    C *= 2.0
    C -= 1.0
    R = _u01(rng, m) * rmax
    return C, R


def sphere(m: int, d: int, seed: int, inner_sigma: float = 0.3):
    """Points (r_i = 0): m//2 on the unit sphere about a N(0,I) centre, the rest
    at centre + N(0, inner_sigma^2/d I) redrawn until their norm is < 0.99.

    Returns (C, R, centre).  The optimum is r* = 1, c* = centre whenever the
    centre lies in the hull of the sphere points (Wendel: probability ~1 for
    m/2 >> d)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ctr = rng.standard_normal(d)
    ns = m // 2
    C = np.empty((m, d))
    for lo in range(0, ns, 8192):
        hi = min(ns, lo + 8192)
        g = rng.standard_normal((hi - lo, d))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        C[lo:hi] = g
    k = ns
    scale = inner_sigma / np.sqrt(d)
    while k < m:
        n = min(m - k, 8192)
        h = rng.standard_normal((n, d)) * scale
        keep = np.linalg.norm(h, axis=1) < 0.99
        h = h[keep]
        C[k:k + h.shape[0]] = h
        k += h.shape[0]
    C += ctr
    return C, np.zeros(m), ctr


def lcg(m: int, d: int):
    """The paper's instance family (Sec. 5, test instances):
    psi_0 = 7, psi_{j+1} = (445 psi_j + 1) mod 4096, values psi_j / 40.96 for
    j >= 1, assigned in the order r_1, c_1(1..d), r_2, c_2(1..d), ..."""
    n = m * (d + 1)
    psi = np.empty(n, dtype=np.int64)
    p = 7
    # the sequence has period 4096: build one period and tile it
    period = np.empty(4096, dtype=np.int64)
    for j in range(4096):
        p = (445 * p + 1) % 4096
        period[j] = p
    reps = -(-n // 4096)
    psi[:] = np.tile(period, reps)[:n]
    vals = psi.astype(np.float64) / 40.96
    a = vals.reshape(m, d + 1)
    return np.ascontiguousarray(a[:, 1:]), np.ascontiguousarray(a[:, 0])


def lcg_psi(n: int) -> np.ndarray:
    """The first n terms psi_1..psi_n of the Sec. 5 generator (integers)."""
    out = np.empty(n, dtype=np.int64)
    p = 7
    for j in range(n):
        p = (445 * p + 1) % 4096
        out[j] = p
    return out


RAGGED_DIMS = (2, 3, 16, 64, 256)


def ragged_shape(k: int, seed: int):
    """(m, d) of instance k of the ragged batch: m = round(10^(2 + 3u)) (log-uniform
    in [100, 100000]), d uniform over RAGGED_DIMS; from its own stream."""
    rng = np.random.Generator(np.random.PCG64([seed, k]))
    u = _u01(rng, 2)
    m = int(round(10.0 ** (2.0 + 3.0 * u[0])))
    d = RAGGED_DIMS[min(int(u[1] * len(RAGGED_DIMS)), len(RAGGED_DIMS) - 1)]
    return m, d


def ragged_instance(k: int, seed: int):
    """Instance k of the ragged batch: centres N(0,1)^d, radii U[0, 0.1]."""
    m, d = ragged_shape(k, seed)
    rng = np.random.Generator(np.random.PCG64([seed, k, 1]))
    C = rng.standard_normal((m, d))
    R = _u01(rng, m) * 0.1
    return C, R


def ragged(n: int, seed: int = 1004):
    """The first n instances of the ragged batch (a list of (C, R))."""
    return [ragged_instance(k, seed) for k in range(n)]


def poisson_arrivals(rate: float, duration: float, n_pool: int, seed: int,
                     large_frac: float = 0.0, n_large: int = 0):
    """Arrival times (seconds, increasing, < duration) of a Poisson stream at
    `rate` requests/s, and for each the index of the instance it carries: with
    probability large_frac one of n_large large instances (returned as
    -1 - k), else one of n_pool ragged instances."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_max = int(rate * duration * 1.5 + 50)
    gaps = -np.log1p(-_u01(rng, n_max)) / rate
    t = np.cumsum(gaps)
    t = t[t < duration]
    u = _u01(rng, 2 * len(t)).reshape(-1, 2) if len(t) else np.zeros((0, 2))
    pick = np.minimum((u[:, 1] * n_pool).astype(np.int64), n_pool - 1)
    if n_large > 0 and large_frac > 0:
        big = u[:, 0] < large_frac
        pick = np.where(big, -1 - np.minimum((u[:, 1] * n_large).astype(np.int64), n_large - 1), pick)
    return t, pick


def digest(*arrays) -> str:
    """SHA-256 of the raw bytes of the given arrays (for stored expected values)."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


# Named workloads of the benchmark (sizes as stated; seeds fixed).
def workload(name: str):
    if name == "gaussian_m1e4_d10":
        return gaussian(10_000, 10, 1001, 0.1)
    if name == "cube_m2e6_d100":
        return cube(2_000_000, 100, 1002, 0.05)
    if name == "cube_m1e6_d100":   # half-size cube instance for counter captures
        return cube(1_000_000, 100, 1012, 0.05)
    if name == "sphere_m2e5_d2000":
        C, R, _ = sphere(200_000, 2000, 1003)
        return C, R
    if name == "sphere_m5e4_d2000":   # quarter-size sphere instance for counter captures
        C, R, _ = sphere(50_000, 2000, 1013)
        return C, R
    raise KeyError(name)
