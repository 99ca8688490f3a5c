// Device side of the solver kernels (the bodies of the kernels in
// meb_solve.cu): the dense Newton systems (SYRK assembly, the FP32
// Gauss-Jordan inverses with refinement, the FP64 Cholesky), the matrix-free
// CG, the multiplier update and the solve's initial and final points.  Each
// body takes its block index and count where it has more than one block.
#pragma once
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "meb_control.cuh"

namespace meb {

// ===========================================================================
// Controller (one block): reduces the pass, forms grad and Psi, and takes the
// decisions of Algorithms 1 and 2.  Vector work is spread over the block.

// ===========================================================================
// Dense Newton system (d + 1 <= kMaxDenseN):
//   H = tau/sigma I + sigma (n_I I + sum_M P_k),
//   sum_M P_k = 1/2 [[n_M, sum w^T], [sum w, sum(1+t) I - sum t w w^T]].
// k_syrk: partial tiles of sum_M t_k w_k w_k^T over row groups.
constexpr int kSyrkGroups = 24;

// Tile `tri` of the lower triangle, row group `grp` of `ngroups` (partials
// summed in group order by syrk_reduce_block with the same ngroups).
__device__ __forceinline__ void syrk_block(const Buffers& B, int d, int tri, int grp,
                                           int ngroups = kSyrkGroups) {
  const DevState* st = B.st;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  if (tri >= ntri) return;
  // tile (ti >= tj) from the linear lower-triangle index
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= tri) ti++;
  const int tj = tri - ti * (ti + 1) / 2;
  const int nS = st->nS;
  const int rpg = (nS + ngroups - 1) / ngroups;
  const int k0 = grp * rpg, k1 = min(nS, k0 + rpg);
  __shared__ double sa[kSyrkRows][kSyrkTile + 1];
  __shared__ double sb[kSyrkRows][kSyrkTile + 1];
  __shared__ double stw[kSyrkRows];
  // thread -> 4 outputs: rows (ty*4 .. ty*4+3)? use (r = tid/32 + 8q, c = tid%32)
  const int cc = threadIdx.x & 31, r0 = threadIdx.x >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int kb = k0; kb < k1; kb += kSyrkRows) {
    const int nr = min(kSyrkRows, k1 - kb);
    for (int e = threadIdx.x; e < kSyrkRows * kSyrkTile; e += 256) {
      const int rr = e / kSyrkTile, c2 = e % kSyrkTile;
      double va = 0.0, vb = 0.0;
      if (rr < nr) {
        const int k = kb + rr;
        const int ja = ti * kSyrkTile + c2, jb = tj * kSyrkTile + c2;
        const bool m = B.S_case[k] == CASE_M;
        if (m && ja < d) va = B.W[(int64_t)k * d + ja];
        if (m && jb < d) vb = B.W[(int64_t)k * d + jb];
      }
      sa[rr][c2] = va;
      sb[rr][c2] = vb;
    }
    if (threadIdx.x < kSyrkRows) {
      const int k = kb + threadIdx.x;
      stw[threadIdx.x] = (threadIdx.x < nr && B.S_case[k] == CASE_M) ? B.S_t[k] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < nr; rr++) {
      const double t = stw[rr];
      const double bv = sb[rr][cc] * t;
#pragma unroll
      for (int q = 0; q < 4; q++) acc[q] = fma(sa[rr][r0 + 8 * q], bv, acc[q]);
    }
    __syncthreads();
  }
  double* out = B.hpart + ((int64_t)grp * ntri + tri) * (kSyrkTile * kSyrkTile);
#pragma unroll
  for (int q = 0; q < 4; q++) out[(r0 + 8 * q) * kSyrkTile + cc] = acc[q];
}

__device__ __forceinline__ bool newton_gate(const DevState* st) {
  return st->status == 0 && st->action == ACT_NEWTON;
}

// Sum the group partials (in group order) into B.H's lower triangle block
// (rows/cols 1..d); block bid of nb strides over the entries.
__device__ __forceinline__ void syrk_reduce_block(const Buffers& B, int d, int bid, int nb,
                                                  int ngroups = kSyrkGroups) {
  const DevState* st = B.st;
  // H = tau/sigma I + sigma (n_I I + 1/2 [[n_M, sum w^T], [sum w, sum(1+t) I - SY]]),
  // SY = sum_M t w w^T from the group partials (summed in group order)
  const DevVecs& V = B.vec;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  const int n1 = d + 1;
  const double sigma = st->sigma, tos = st->tos;
  const double nI = st->last[P_NI], nM = st->last[P_NM], s1t = V.st1[0];
  for (int64_t e = (int64_t)bid * blockDim.x + threadIdx.x; e < (int64_t)n1 * n1;
       e += (int64_t)nb * blockDim.x) {
    const int i = (int)(e / n1), l = (int)(e % n1);
    if (l > i) continue;   // the thread of (i, l) writes (i, l) and (l, i)
    double h;
    if (i == 0) {
      h = tos + sigma * (nI + 0.5 * nM);
    } else if (l == 0) {
      h = sigma * 0.5 * V.sw[i - 1];
    } else {
      const int j = i - 1, k = l - 1;   // k <= j
      const int ti = j / kSyrkTile, tj = k / kSyrkTile;
      const int tri = ti * (ti + 1) / 2 + tj;
      const int loc = (j % kSyrkTile) * kSyrkTile + (k % kSyrkTile);
      double sy = 0.0;
      for (int g = 0; g < ngroups; g++)
        sy += B.hpart[((int64_t)g * ntri + tri) * (kSyrkTile * kSyrkTile) + loc];
      h = -0.5 * sigma * sy;
      if (i == l) h += tos + sigma * (nI + 0.5 * s1t);
    }
    B.H[(int64_t)i * n1 + l] = h;
    B.H[(int64_t)l * n1 + i] = h;
    // the FP32 pair hi + lo = h to 2^-48 relative (Gauss-Jordan and its
    // double-float residual)
    const float hi = __double2float_rn(h);
    const float lo = __double2float_rn(h - (double)hi);
    B.Hhi[(int64_t)i * n1 + l] = hi;
    B.Hhi[(int64_t)l * n1 + i] = hi;
    B.Hlo[(int64_t)i * n1 + l] = lo;
    B.Hlo[(int64_t)l * n1 + i] = lo;
  }
}

// One block: assemble H (packed lower, smem), Cholesky, solve H dx = -g,
// then set the first line-search trial x + dx.
// FP64 Cholesky solve of H dx = -g by one block of 256 threads, with Lp
// (n(n+1)/2 doubles, packed lower: row i at i(i+1)/2) in shared memory.
__device__ inline void newton_chol_body(const Buffers& B, int d, double* Lp) {
  DevState* st = B.st;
  __shared__ double sh[32];
  __shared__ int s_fail;
  const DevVecs& V = B.vec;
  const int n = d + 1;
  const double sigma = st->sigma, tos = st->tos;
  const double nI = st->last[P_NI], nM = st->last[P_NM];
  const double s1t = V.st1[0];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  (void)tos; (void)nI; (void)nM; (void)s1t;
  for (int i = wid; i < n; i += 8) {
    const int64_t ri = (int64_t)i * (i + 1) / 2;
    for (int l = lane; l <= i; l += 32) Lp[ri + l] = B.H[(int64_t)i * n + l];   // assembled H
  }
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  // right-looking Cholesky on the packed lower triangle
  for (int j = 0; j < n; j++) {
    const int64_t jj = (int64_t)j * (j + 1) / 2 + j;
    if (threadIdx.x == 0) {
      const double p = Lp[jj];
      if (!(p > 0.0)) s_fail = 1;
      Lp[jj] = sqrt(fmax(p, DBL_MIN));
    }
    __syncthreads();
    if (s_fail) break;
    const double ljj = Lp[jj];
    for (int i = j + 1 + threadIdx.x; i < n; i += 256) Lp[(int64_t)i * (i + 1) / 2 + j] /= ljj;
    __syncthreads();
    // trailing update: rows i > j, cols j < l <= i (warp per row)
    for (int i = j + 1 + wid; i < n; i += 8) {
      const int64_t ri = (int64_t)i * (i + 1) / 2;
      const double lij = Lp[ri + j];
      for (int l = j + 1 + lane; l <= i; l += 32)
        Lp[ri + l] -= lij * Lp[(int64_t)l * (l + 1) / 2 + j];
    }
    __syncthreads();
  }
  if (s_fail) {
    // Cholesky broke down: end the inner loop here (outer update at x)
    if (threadIdx.x == 0) st->chol_fail += 1;
    do_outer(st, V, d, sh);
    return;
  }
  // forward / backward substitution (single warp; n <= 225)
  double* y = V.dx;
  if (threadIdx.x < 32) {
    for (int i = 0; i < n; i++) {
      const int64_t ri = (int64_t)i * (i + 1) / 2;
      double t = 0.0;
      for (int k = threadIdx.x; k < i; k += 32) t += Lp[ri + k] * y[k];
      t = warp_sum(t);
      if (threadIdx.x == 0) y[i] = (-V.g[i] - t) / Lp[ri + i];
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; i--) {
      double t = 0.0;
      for (int k = i + 1 + threadIdx.x; k < n; k += 32) t += Lp[(int64_t)k * (k + 1) / 2 + i] * y[k];
      t = warp_sum(t);
      if (threadIdx.x == 0) y[i] = (y[i] - t) / Lp[(int64_t)i * (i + 1) / 2 + i];
      __syncwarp();
    }
  }
  __syncthreads();
  double gd = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) {
    gd += V.g[k] * V.dx[k];
    V.xt[k] = V.x[k] + V.dx[k];
  }
  gd = block_sum<256>(gd, sh);
  if (threadIdx.x == 0) {
    st->fp64_solves += 1;
    st->gdx = gd;
    st->eta = 1.0;
    st->phase = 1;
    st->bt = 0;
    st->action = ACT_TRIAL;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

// The Newton direction dx (in shared memory) becomes the first line-search
// trial: dx, gdx = g.dx, xt = x + dx and the trial's query shadow.
__device__ inline void newton_accept(DevState* st, const DevVecs& V, int d, const double* s_x,
                              double* sh) {
  const int n = d + 1;
  double gd = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    V.dx[k] = s_x[k];
    gd += V.g[k] * s_x[k];
    V.xt[k] = V.x[k] + s_x[k];
  }
  gd = block_sum<256>(gd, sh);
  if (threadIdx.x == 0) {
    st->need_fp64_solve = 0;
    st->gdx = gd;
    st->eta = 1.0;
    st->phase = 1;
    st->bt = 0;
    st->action = ACT_TRIAL;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

// One block: FP32 Gauss-Jordan inverse of H (SPD, no pivoting needed), then
// dx = -H^{-1} g refined in FP64: r = -g - H dx (FP64), dx += H32^{-1} r.
// Sets need_fp64_solve when a pivot is not positive or the refinement does
// not converge; otherwise sets up the first line-search trial.
__device__ __forceinline__ void newton_gj_body(const Buffers& B, int d) {
  DevState* st = B.st;
  if (st->force_fp64_solve) {   // the FP64 Cholesky follows
    if (threadIdx.x == 0) st->need_fp64_solve = 1;
    return;
  }
  extern __shared__ float A[];    // n x n, row-major
  __shared__ double sh[32];
  __shared__ int s_fail;
  __shared__ float s_prow[kMaxDenseN];
  __shared__ float s_rf[kMaxDenseN];
  const DevVecs& V = B.vec;
  const int n = d + 1;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < n * n; e += 256) A[e] = (float)B.H[e];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int k = 0; k < n; k++) {
    const float p = A[k * n + k];
    if (!(p > 0.0f) || !isfinite(p)) { if (tid == 0) s_fail = 1; }
    __syncthreads();
    if (s_fail) break;
    const float ip = 1.0f / p;
    for (int j = tid; j < n; j += 256) {
      const float v = (j == k) ? ip : A[k * n + j] * ip;
      s_prow[j] = v;
    }
    __syncthreads();
    for (int j = tid; j < n; j += 256) A[k * n + j] = s_prow[j];
    // rows i != k: A[i][j] -= A[i][k] * prow[j]; A[i][k] = -A[i][k] * ip
    for (int i = wid; i < n; i += 8) {
      if (i == k) continue;
      const float f = A[i * n + k];
      __syncwarp();
      for (int j = lane; j < n; j += 32) {
        if (j == k) continue;
        A[i * n + j] = fmaf(-f, s_prow[j], A[i * n + j]);
      }
      __syncwarp();
      if (lane == 0) A[i * n + k] = -f * ip;
    }
    __syncthreads();
  }
  bool ok = !s_fail;
  if (ok) {
    // dx = A (-g), then refinement: r = -g - H dx (FP64), dx += A r (FP32).
    // Thread i owns component i; A and H are read by columns (H symmetric,
    // A ~ H^{-1} symmetric up to rounding), which coalesces.
    double* x = V.dx;
    for (int i = tid; i < n; i += 256) s_rf[i] = (float)(-V.g[i]);
    __syncthreads();
    double rn0 = 0.0;
    for (int it = 0; it < 5; it++) {
      double dn = 0.0, xn = 0.0;
      for (int i = tid; i < n; i += 256) {
        float t = 0.0f;
        for (int j = 0; j < n; j++) t = fmaf(A[j * n + i], s_rf[j], t);
        const double xi = (it == 0 ? 0.0 : x[i]) + (double)t;
        x[i] = xi;
        dn += (double)t * (double)t;
        xn += xi * xi;
      }
      dn = block_sum<256>(dn, sh);
      xn = block_sum<256>(xn, sh);
      if (dn <= 1e-22 * xn) break;
      double rn = 0.0;
      for (int i = tid; i < n; i += 256) {
        double t = -V.g[i];
        for (int j = 0; j < n; j++) t = fma(-B.H[(int64_t)j * n + i], x[j], t);
        s_rf[i] = (float)t;
        rn += t * t;
      }
      rn = block_sum<256>(rn, sh);
      if (it == 0) rn0 = rn;
      else if (!(rn <= rn0)) { ok = false; break; }   // refinement diverges
      if (it == 4) ok = rn <= 1e-16 * rn0;
    }
  }
  if (tid == 0) st->gj_inverses += 1;
  if (!ok) {
    if (tid == 0) st->need_fp64_solve = 1;
    return;
  }
  double gd = 0.0;
  for (int k = tid; k < n; k += 256) {
    gd += V.g[k] * V.dx[k];
    V.xt[k] = V.x[k] + V.dx[k];
  }
  gd = block_sum<256>(gd, sh);
  if (tid == 0) {
    st->need_fp64_solve = 0;
    st->gdx = gd;
    st->eta = 1.0;
    st->phase = 1;
    st->bt = 0;
    st->action = ACT_TRIAL;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

// Register-blocked variant for n = d + 1 <= 112, on a 16 x 16 thread grid:
// thread (ty, tx) holds rows ty + 16 i and columns tx + 16 j (i, j < 7) of the
// matrix in registers, as column pairs for packed FP32x2 arithmetic.  Each
// Gauss-Jordan pivot publishes the old pivot row and column through shared
// memory (double-buffered: one barrier per pivot) and updates every entry.
// H is SPD: no pivoting.
//
// FP64 instructions are few on this GPU's FP64 pipe, so the refinement runs
// in double-float arithmetic: dx = A (-g) is refined with the residual
// r = -g - H dx, where H = Hhi + Hlo, dx = xh + xl and -g = bh + bl are FP32
// pairs, products are split exactly with fmaf and sums taken by TwoSum
// (about 2^-48 relative).
constexpr int kGjTile = 7;
constexpr int kGjRegN = 16 * kGjTile;

// exact a + b = s + e (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// s + l += (hh + hl)(xh + xl), dropping hl xl (2^-48 relative)
__device__ __forceinline__ void df_mac(float hh, float hl, float xh, float xl, float& s,
                                       float& l) {
  const float p = hh * xh;
  const float e = fmaf(hh, xh, -p);   // exact rounding error of p
  const float c = fmaf(hh, xl, fmaf(hl, xh, e));
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  l += err + c;
}

// block-wide FP32 sums of two values in a fixed order (every thread gets them)
__device__ __forceinline__ float2 block_sum2f(float a, float b, float2* sh8) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(MEB_FULLMASK, a, o);
    b += __shfl_xor_sync(MEB_FULLMASK, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh8[threadIdx.x >> 5] = make_float2(a, b);
  __syncthreads();
  float2 t = sh8[0];
#pragma unroll
  for (int k = 1; k < 8; k++) { t.x += sh8[k].x; t.y += sh8[k].y; }
  return t;
}

// Small systems, n = d + 1 <= 32: one warp.  Lane i holds row i of the matrix
// in registers; each pivot's row comes by shuffles, so the sweep needs no block
// barrier.  The same FP32 Gauss-Jordan sweep and double-float refinement as the
// 256-thread solve (at most two corrections; the second residual must be at
// most half the first, else the FP64 Cholesky).  Warp 0 computes; the block
// then sets up the trial.  No inverse is kept (a fresh one costs little here).
constexpr int kGjWarpN = 32;

__device__ __forceinline__ void newton_gj_warp_body(const Buffers& B, int d) {
  DevState* st = B.st;
  extern __shared__ double dyn_Lp[];   // the Cholesky fallback's factor
  __shared__ double s_x[kGjWarpN];
  __shared__ double sh[32];
  __shared__ int s_ok;
  const DevVecs& V = B.vec;
  const int n = d + 1;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) {
    float a[kGjWarpN];   // a[j] = A[lane][j]; rows and columns past n: identity
#pragma unroll
    for (int j = 0; j < kGjWarpN; j++)
      a[j] = (lane < n && j < n) ? B.Hhi[(int64_t)lane * n + j] : (lane == j ? 1.0f : 0.0f);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < kGjWarpN; k++) {
      if (k < n && ok) {   // the same for every lane
        const float p = __shfl_sync(MEB_FULLMASK, a[k], k);
        ok = (p > 0.0f) && isfinite(p);
        const float ip = __fdividef(1.0f, p);
        const float cik = a[k];   // A[lane][k] before the sweep
#pragma unroll
        for (int j = 0; j < kGjWarpN; j++) {
          const float rkj = __shfl_sync(MEB_FULLMASK, a[j], k);   // A[k][j] before the sweep
          if (lane == k) a[j] = (j == k) ? ip : rkj * ip;
          else a[j] = (j == k) ? -cik * ip : fmaf(-cik, rkj * ip, a[j]);
        }
      }
    }
    // x0 = A (-g) and corrections x += A r, r = -g - H x in double-float
    const double b = (lane < n) ? -V.g[lane] : 0.0;
    const float bh = __double2float_rn(b);
    const float bl = __double2float_rn(b - (double)bh);
    float sb = bh, xh = 0.0f, xl = 0.0f, rn0 = 0.0f;
    bool conv = false;
    for (int it = 0; ok && it < 3; it++) {
      float t = 0.0f;
#pragma unroll
      for (int j = 0; j < kGjWarpN; j++) t = fmaf(a[j], __shfl_sync(MEB_FULLMASK, sb, j), t);
      if (lane >= n) t = 0.0f;
      float h, e;
      two_sum(xh, t, h, e);
      const float l = xl + e;
      const float h2 = h + l;
      xl = l - (h2 - h);
      xh = h2;
      const float dn = warp_sum_t(t * t), xn = warp_sum_t(xh * xh);
      if (dn <= 1e-16f * xn || it == 2) { conv = true; break; }
      float sa = 0.0f, la = 0.0f;
      for (int j = 0; j < n; j++) {
        const float xj = __shfl_sync(MEB_FULLMASK, xh, j), xlj = __shfl_sync(MEB_FULLMASK, xl, j);
        if (lane < n) df_mac(B.Hhi[(int64_t)lane * n + j], B.Hlo[(int64_t)lane * n + j], xj, xlj, sa, la);
      }
      float r = 0.0f;
      if (lane < n) {
        float hh, ee;
        two_sum(bh, -sa, hh, ee);   // exact leading difference
        r = hh + ((ee + bl) - la);
      }
      const float rr = warp_sum_t(r * r);
      if (it == 0) rn0 = rr;
      else if (!(rr <= 0.25f * rn0)) { ok = false; break; }
      sb = r;
    }
    if (lane < n) s_x[lane] = (double)xh + (double)xl;
    if (lane == 0) {
      s_ok = ok && conv;
      st->gj_inverses += 1;
      st->inv_valid = 0;
    }
  }
  __syncthreads();
  if (!s_ok) {
    newton_chol_body(B, d, dyn_Lp);   // the FP64 Cholesky in the same launch
    return;
  }
  newton_accept(st, V, d, s_x, sh);
}

// Kept inverse: while sigma is unchanged, H changes from one Newton step to
// the next only through the t_k and the support, so the inverse of the last
// H is tried first.  The refinement below converges with it when it
// contracts the residual; the iteration count and the required contraction
// bound the cost of a failed try, after which the inverse is recomputed.
constexpr int kGjReuseIters = 8;

__device__ __forceinline__ void newton_gj_reg_body(const Buffers& B, int d) {
  DevState* st = B.st;
  extern __shared__ double dyn_Lp[];   // the Cholesky fallback's factor
  if (st->force_fp64_solve) {
    newton_chol_body(B, d, dyn_Lp);
    return;
  }
  static_assert(4 * kGjTile * 256 == kAinvLen && kGjRegN == kAinvMaxN, "kept inverse layout");
  __shared__ float s_row[2][kGjRegN], s_col[2][kGjRegN];
  __shared__ float s_b[kGjRegN], s_bh[kGjRegN], s_bl[kGjRegN], s_xh[kGjRegN], s_xl[kGjRegN];
  __shared__ float2 s_red[8];
  __shared__ double sh[32];
  __shared__ double s_x[kGjRegN];
  const DevVecs& V = B.vec;
  const int n = d + 1;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // a[i][q] = (A[ty+16i][tx+32q], A[ty+16i][tx+32q+16]); column tx+112 is a zero dummy
  float2 a[kGjTile][4];
  bool fresh = !(B.Ainv && st->inv_valid && st->kept_sigma == st->sigma);
  bool ok = true, solved = false;
  for (int attempt = 0; attempt < 2 && !solved; attempt++) {
    if (fresh) {
#pragma unroll
      for (int i = 0; i < kGjTile; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int row = ty + 16 * i, col = tx + 16 * j;
          const float v = (j == 7) ? 0.0f
                                   : (row < n && col < n) ? B.Hhi[(int64_t)row * n + col]
                                                          : (row == col ? 1.0f : 0.0f);
          if (j & 1) a[i][j >> 1].y = v; else a[i][j >> 1].x = v;
        }
    } else {
#pragma unroll
      for (int i = 0; i < kGjTile; i++)
#pragma unroll
        for (int q = 0; q < 4; q++) a[i][q] = B.Ainv[(i * 4 + q) * 256 + tid];
    }
    float bn = 0.0f;
    for (int i = tid; i < kGjRegN; i += 256) {
      const double b = (i < n) ? -V.g[i] : 0.0;   // solve H dx = -g
      const float bh = __double2float_rn(b);
      s_bh[i] = bh;
      s_bl[i] = __double2float_rn(b - (double)bh);
      s_b[i] = bh;
      s_xh[i] = 0.0f;
      s_xl[i] = 0.0f;
      bn = fmaf(bh, bh, bn);
    }
    if (!fresh) bn = block_sum2f(bn, 0.0f, s_red).x;
    if (fresh) {
#pragma unroll
      for (int kb = 0; kb < kGjTile; kb++) {
        for (int kk = 0; kk < 16; kk++) {
          const int k = 16 * kb + kk;
          if (k < n && ok) {
            const int bf = k & 1;
            if (ty == kk) {
#pragma unroll
              for (int j = 0; j < kGjTile; j++)
                s_row[bf][tx + 16 * j] = (j & 1) ? a[kb][j >> 1].y : a[kb][j >> 1].x;
            }
            if (tx == kk) {
#pragma unroll
              for (int i = 0; i < kGjTile; i++)
                s_col[bf][ty + 16 * i] = (kb & 1) ? a[i][kb >> 1].y : a[i][kb >> 1].x;
            }
            __syncthreads();
            const float p = s_row[bf][k];
            ok = (p > 0.0f) && isfinite(p);   // the same for every thread
            const float ip = __fdividef(1.0f, p);
            float2 rc[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
              const float lo = s_row[bf][tx + 32 * q];
              const float hi = (q < 3) ? s_row[bf][tx + 32 * q + 16] : 0.0f;
              rc[q] = __fmul2_rn(make_float2(lo, hi), make_float2(ip, ip));
            }
            float cr[kGjTile];
#pragma unroll
            for (int i = 0; i < kGjTile; i++) cr[i] = s_col[bf][ty + 16 * i];
#pragma unroll
            for (int i = 0; i < kGjTile; i++)
#pragma unroll
              for (int q = 0; q < 4; q++)
                a[i][q] = __ffma2_rn(make_float2(-cr[i], -cr[i]), rc[q], a[i][q]);
            if (ty == kk) {   // pivot row: A[k][j] / p, and 1/p on the diagonal
#pragma unroll
              for (int j = 0; j < kGjTile; j++) {
                const float rj = (j & 1) ? rc[j >> 1].y : rc[j >> 1].x;
                const float v = (tx + 16 * j == k) ? ip : rj;
                if (j & 1) a[kb][j >> 1].y = v; else a[kb][j >> 1].x = v;
              }
            }
            if (tx == kk) {   // pivot column: -A[i][k] / p off the diagonal
#pragma unroll
              for (int i = 0; i < kGjTile; i++) {
                if (ty + 16 * i != k) {
                  const float v = -cr[i] * ip;
                  if (kb & 1) a[i][kb >> 1].y = v; else a[i][kb >> 1].x = v;
                }
              }
            }
          }
        }
      }
      if (tid == 0) {
        st->gj_inverses += 1;
        st->inv_valid = 0;
      }
      if (!ok) break;   // the FP64 Cholesky
      if (B.Ainv) {
#pragma unroll
        for (int i = 0; i < kGjTile; i++)
#pragma unroll
          for (int q = 0; q < 4; q++) B.Ainv[(i * 4 + q) * 256 + tid] = a[i][q];
      }
    }
    __syncthreads();
    // x0 = A (-g) and corrections dx += A r: the Newton direction needs a
    // small relative error, not FP64 accuracy (the stop test, Armijo and KKT
    // use the FP64 gradient and Psi).  A fresh inverse gets two corrections
    // and must halve the residual.  A kept one gets up to kGjReuseIters; it
    // must halve the residual at every step, and is given up as soon as its
    // rate cannot bring the residual to 1e-9 of -g within the steps left.
    const int max_it = fresh ? 3 : kGjReuseIters;
    float rn_prev = bn, rn0 = 0.0f;
    bool conv = false;
    for (int it = 0; it < max_it; it++) {
      // t = A s_b : partial rows over this thread's columns, reduced over tx
      float tv[kGjTile];
#pragma unroll
      for (int i = 0; i < kGjTile; i++) {
        float2 t2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const float lo = s_b[tx + 32 * q];
          const float hi = (q < 3) ? s_b[tx + 32 * q + 16] : 0.0f;
          t2 = __ffma2_rn(a[i][q], make_float2(lo, hi), t2);
        }
        tv[i] = t2.x + t2.y;
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < kGjTile; i++) tv[i] += __shfl_xor_sync(MEB_FULLMASK, tv[i], o);
      float dn = 0.0f, xn = 0.0f;
      if (tx == 0) {
#pragma unroll
        for (int i = 0; i < kGjTile; i++) {
          const int row = ty + 16 * i;
          if (row < n) {
            float h, e;
            two_sum(s_xh[row], tv[i], h, e);
            const float l = s_xl[row] + e;
            const float h2 = h + l;               // renormalise the pair
            s_xl[row] = l - (h2 - h);
            s_xh[row] = h2;
            dn = fmaf(tv[i], tv[i], dn);
            xn = fmaf(h2, h2, xn);
          }
        }
      }
      const float2 dx2 = block_sum2f(dn, xn, s_red);   // (barriers: s_xh, s_xl visible)
      if (dx2.x <= 1e-16f * dx2.y) { conv = true; break; }
      if (fresh && it == max_it - 1) { conv = true; break; }
      if (it == max_it - 1) break;
      // r = -g - H x in double-float, rows reduced over tx
      float sa[kGjTile], la[kGjTile];
#pragma unroll
      for (int i = 0; i < kGjTile; i++) {
        const int row = ty + 16 * i;
        sa[i] = 0.0f;
        la[i] = 0.0f;
#pragma unroll
        for (int j = 0; j < kGjTile; j++) {
          const int col = tx + 16 * j;
          if (row < n && col < n)
            df_mac(B.Hhi[(int64_t)row * n + col], B.Hlo[(int64_t)row * n + col], s_xh[col],
                   s_xl[col], sa[i], la[i]);
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < kGjTile; i++) {
          const float so = __shfl_xor_sync(MEB_FULLMASK, sa[i], o);
          const float lo = __shfl_xor_sync(MEB_FULLMASK, la[i], o);
          float t, err;
          two_sum(sa[i], so, t, err);
          sa[i] = t;
          la[i] += lo + err;
        }
      float rn = 0.0f;
      if (tx == 0) {
#pragma unroll
        for (int i = 0; i < kGjTile; i++) {
          const int row = ty + 16 * i;
          if (row < n) {
            float h, e;
            two_sum(s_bh[row], -sa[i], h, e);   // exact leading difference
            const float r = h + ((e + s_bl[row]) - la[i]);
            s_b[row] = r;
            rn = fmaf(r, r, rn);
          }
        }
      }
      const float rr = block_sum2f(rn, 0.0f, s_red).x;   // (barriers: s_b visible)
      if (fresh) {
        // the second residual at most a quarter of the first (squared norms)
        if (it == 0) rn0 = rr;
        else if (!(rr <= 0.25f * rn0)) break;
      } else {
        if (!isfinite(rr)) break;
        const float rel = rr / bn, q = rr / rn_prev;
        if (!(rel > 1e-18f)) { conv = true; break; }
        if (!(q <= 0.25f)) break;
        const int left = max_it - 1 - it;
        if ((float)left * __logf(q) > __logf(1e-18f / rel)) break;
        rn_prev = rr;
      }
    }
    if (conv) {
      solved = true;
      if (tid == 0) {
        if (!fresh) st->gj_reuses += 1;
        st->inv_valid = B.Ainv ? 1 : 0;
        st->kept_sigma = st->sigma;
      }
    } else if (fresh) {
      ok = false;   // the FP64 Cholesky
    } else {
      fresh = true;   // the kept inverse did not contract: a new one
    }
    __syncthreads();
  }
  if (!ok || !solved) {
    // the FP64 Cholesky in the same launch (dynamic shared memory n(n+1)/2 doubles)
    if (tid == 0) st->inv_valid = 0;
    __syncthreads();
    newton_chol_body(B, d, dyn_Lp);
    return;
  }
  for (int i = tid; i < kGjRegN; i += 256) s_x[i] = (double)s_xh[i] + (double)s_xl[i];
  __syncthreads();
  newton_accept(st, V, d, s_x, sh);
}

// Small dense systems (n <= 32, at most 32 support rows): the block of the
// solve assembles H itself, so the SYRK launches are skipped.  Each entry sums
// the support rows in order, as the one-group SYRK does (the batched solver's
// H is the same either way); one thread per entry, so the support is kept
// short.
constexpr int kFusedSyrkRows = 32;
__device__ __forceinline__ bool syrk_in_solve(const DevState* st, int d) {
  return d + 1 <= kGjWarpN && !st->force_fp64_solve && st->nS <= kFusedSyrkRows;
}

// H = tau/sigma I + sigma (n_I I + 1/2 [[n_M, sum w^T], [sum w, sum(1+t) I - SY]])
// with SY = sum_M t w w^T summed over the support rows in order (block-wide).
__device__ __forceinline__ void h_assemble_block(const Buffers& B, int d) {
  const DevState* st = B.st;
  const DevVecs& V = B.vec;
  const int n1 = d + 1, nS = st->nS;
  const double sigma = st->sigma, tos = st->tos;
  const double nI = st->last[P_NI], nM = st->last[P_NM], s1t = V.st1[0];
  for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x) {
    const int i = e / n1, l = e % n1;
    if (l > i) continue;   // the thread of (i, l) writes (i, l) and (l, i)
    double h;
    if (i == 0) {
      h = tos + sigma * (nI + 0.5 * nM);
    } else if (l == 0) {
      h = sigma * 0.5 * V.sw[i - 1];
    } else {
      const int j = i - 1, k = l - 1;
      double sy = 0.0;
      for (int r = 0; r < nS; r++) {
        if (B.S_case[r] != CASE_M) continue;
        const double bv = B.W[(int64_t)r * d + k] * B.S_t[r];
        sy = fma(B.W[(int64_t)r * d + j], bv, sy);
      }
      h = -0.5 * sigma * sy;
      if (i == l) h += tos + sigma * (nI + 0.5 * s1t);
    }
    B.H[(int64_t)i * n1 + l] = h;
    B.H[(int64_t)l * n1 + i] = h;
    const float hi = __double2float_rn(h);
    const float lo = __double2float_rn(h - (double)hi);
    B.Hhi[(int64_t)i * n1 + l] = hi;
    B.Hhi[(int64_t)l * n1 + i] = hi;
    B.Hlo[(int64_t)i * n1 + l] = lo;
    B.Hlo[(int64_t)l * n1 + i] = lo;
  }
}

// The dense Newton solve for n = d + 1 <= 112 (one thread block): one warp for
// n <= 32 (with H assembled here when the support is small), the 256-thread
// register sweep otherwise.
__device__ __forceinline__ void newton_gj_small_body(const Buffers& B, int d) {
  if (d + 1 <= kGjWarpN && !B.st->force_fp64_solve) {
    if (syrk_in_solve(B.st, d)) {
      h_assemble_block(B, d);
      __syncthreads();
    }
    newton_gj_warp_body(B, d);
  } else {
    newton_gj_reg_body(B, d);
  }
}

// ===========================================================================
// Matrix-free Newton system (Sec. 4.1): CG with the Jacobi preconditioner,
//   Hq = tau/sigma q + sigma (n_I q + sum_M P_k q),
//   P_k q = 1/2 (q0 + w.q1 ; q0 w + (1+t) q1 - t w (w.q1)).
// k_hvp_dot: wq_k = w_k . q1 (warp per row); k_hvp_acc: -1/2 sum_k t_k wq_k w_k
// and 1/2 sum_k wq_k; hvp_finish adds the terms in q0 sum w and sum(1+t) q1.
// Matrix-free Hessian-vector products, FP64 (the evaluation entry) or FP32
// (F32: the solve's CG, when the support rows also exist in FP32, W32: the
// product only shapes the Newton direction; the stop test, Armijo and KKT
// use the FP64 gradient and Psi).
template <bool F32 = false>
__device__ __forceinline__ void hvp_dot_block(const Buffers& B, int d, const double* __restrict__ q,
                                              double* __restrict__ wq, int bid, int nb,
                                              float* s_q32 = nullptr) {
  const DevState* st = B.st;
  const int nS = st->nS;
  const int lane = threadIdx.x & 31;
  if (F32 && s_q32) {   // q1 in FP32 once per block, not once per row
    for (int j = threadIdx.x; j < d; j += blockDim.x) s_q32[j] = (float)q[1 + j];
    __syncthreads();
  }
  for (int k = (bid * 256 + threadIdx.x) >> 5; k < nS; k += (nb * 256) >> 5) {
    double t = 0.0;
    float cf = 0.0f;
    if (B.S_case[k] == CASE_M) {
      if (F32) {
        const float* w = B.W32 + (int64_t)k * d;
        float tf = 0.0f;
        if (s_q32)
          for (int j = lane; j < d; j += 32) tf = fmaf(w[j], s_q32[j], tf);
        else
          for (int j = lane; j < d; j += 32) tf = fmaf(w[j], (float)q[1 + j], tf);
        tf = warp_sum_t(tf);
        t = (double)tf;
        // the row's coefficient in the accumulation, once per row (its
        // conversions run on the FP64 pipe)
        cf = -0.5f * (float)B.S_t[k] * tf;
      } else {
        const double* w = B.W + (int64_t)k * d;
        for (int j = lane; j < d; j += 32) t = fma(w[j], q[1 + j], t);
        t = warp_sum(t);
      }
    }
    if (lane == 0) {
      wq[k] = t;
      if (F32) B.cf32[k] = cf;
    }
  }
}

__device__ __forceinline__ bool cg_gate(const DevState* st) {
  return st->status == 0 && st->action == ACT_NEWTON && !st->cg_done;
}

// Row group bid of nb; F32: column chunk `chunk` of 256 only (chunks < 0:
// every chunk), FP64: every chunk.
template <bool F32 = false>
__device__ __forceinline__ void hvp_acc_block(const Buffers& B, int d, const double* __restrict__ q,
                                              const double* __restrict__ wq,
                                              double* __restrict__ part, int bid, int nb,
                                              int chunk = -1) {
  const DevState* st = B.st;
  const int nS = st->nS;
  const int rpb = (nS + nb - 1) / nb;
  const int k0 = bid * rpb, k1 = min(nS, k0 + rpb);
  double* out = part + (int64_t)bid * (d + 1);
  double s0 = 0.0;
  const int jb = (F32 && chunk >= 0) ? 256 * chunk : 0;
  const int je = (F32 && chunk >= 0) ? min(d, jb + 256) : d;
  for (int j0 = jb; j0 < je; j0 += 256) {
    const int j = j0 + threadIdx.x;
    if (F32) {
      // eight independent accumulators (eight rows' loads in flight), summed
      // in a fixed tree; the row coefficients come from the dot kernel
      const float* cf32 = B.cf32;
      float a[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      int k = k0;
      if (j < d) {
        for (; k + 7 < k1; k += 8) {
          float wv[8];
#pragma unroll
          for (int u = 0; u < 8; u++) wv[u] = B.W32[(int64_t)(k + u) * d + j];
#pragma unroll
          for (int u = 0; u < 8; u++) a[u] = fmaf(cf32[k + u], wv[u], a[u]);
        }
        for (; k < k1; k++) a[0] = fmaf(cf32[k], B.W32[(int64_t)k * d + j], a[0]);
        out[1 + j] = (double)(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])));
      }
      if (j0 == 0) {   // 1/2 sum_M wq over the group's rows, all threads, then in a tree
        __shared__ double sh_s0[32];
        double p0 = 0.0;
        for (int kk = k0 + (int)threadIdx.x; kk < k1; kk += 256)
          if (B.S_case[kk] == CASE_M) p0 += 0.5 * wq[kk];
        s0 = block_sum<256>(p0, sh_s0);
      }
    } else {
      double acc = 0.0;
      for (int k = k0; k < k1; k++) {
        if (B.S_case[k] != CASE_M) continue;
        const double coef = -0.5 * B.S_t[k] * wq[k];   // the q0 w part is 1/2 q0 sum w
        if (j < d) acc = fma(coef, B.W[(int64_t)k * d + j], acc);
        if (j0 == 0 && threadIdx.x == 0) s0 += 0.5 * wq[k];
      }
      if (j < d) out[1 + j] = acc;
    }
  }
  if (threadIdx.x == 0 && jb == 0) out[0] = s0;
}

// At most this many row groups in the FP32 products of the multi-block CG
// (partials per entry summed by the CG update; the partial buffer holds 152).
constexpr int kHvpGroups32 = 152;

// y = tau/sigma q + sigma (n_I q + 1/2 [n_M q0 + S0 ; q0 sum w + sum(1+t) q1] + acc)
__device__ inline void hvp_finish(DevState* st, const DevVecs& V, int d, const double* q,
                           const double* part, int nblk, double* y) {
  const int n1 = d + 1;
  const double sigma = st->sigma, tos = st->tos;
  const double nI = st->last[P_NI], nM = st->last[P_NM], s1t = V.st1[0];
  for (int k = threadIdx.x; k < n1; k += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nblk; b++) a += part[(int64_t)b * n1 + k];
    double pk;
    if (k == 0) pk = nI * q[0] + 0.5 * nM * q[0] + a;
    else pk = nI * q[k] + 0.5 * q[0] * V.sw[k - 1] + 0.5 * s1t * q[k] + a;
    y[k] = tos * q[k] + sigma * pk;
  }
}

constexpr int kHvpBlocks = 152;

__device__ __forceinline__ void cg_setup_body(const Buffers& B, int d) {
  DevState* st = B.st;
  __shared__ double sh[32];
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  const double sigma = st->sigma, tos = st->tos;
  const double nI = st->last[P_NI], nM = st->last[P_NM], s1t = V.st1[0];
  double rz = 0.0, bn = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) {
    // diag(H): k = 0: tos + sigma (nI + nM/2); k > 0: tos + sigma (nI + (s1t - sum t w_k^2)/2)
    const double dg = (k == 0) ? tos + sigma * (nI + 0.5 * nM)
                               : tos + sigma * (nI + 0.5 * (s1t - V.cg_diag[k]));
    V.cg_diag[k] = dg;   // overwrite in place (k > 0 held sum t w^2)
    const double r = -V.g[k];
    V.cg_r[k] = r;
    V.dx[k] = 0.0;
    const double z = r / dg;
    V.cg_z[k] = z;
    V.cg_p[k] = z;
    rz += r * z;
    bn += r * r;
  }
  rz = block_sum<256>(rz, sh);
  bn = block_sum<256>(bn, sh);
  if (threadIdx.x == 0) {
    st->cg_rz = rz;
    st->cg_bn = sqrt(bn);
    double gn = sqrt(bn);
    st->cg_rtol = gn < 0.01 ? sqrt(gn) : 0.1;
    // FP32 products resolve a relative residual of about 1e-7, not below
    if (B.W32 && st->cg_rtol < 1e-6) st->cg_rtol = 1e-6;
    st->cg_it = 0;
    st->cg_done = (bn == 0.0);
  }
}

// One CG iteration after the HVP partials of p are in place.
__device__ __forceinline__ void cg_update_body(const Buffers& B, int d, int nblk) {
  DevState* st = B.st;
  __shared__ double sh[32];
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  hvp_finish(st, V, d, V.cg_p, B.hpart, nblk, V.cg_ap);
  __syncthreads();
  double pap = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) pap += V.cg_p[k] * V.cg_ap[k];
  pap = block_sum<256>(pap, sh);
  const double alpha = st->cg_rz / pap;
  double rr = 0.0, rz1 = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) {
    V.dx[k] += alpha * V.cg_p[k];
    const double r = V.cg_r[k] - alpha * V.cg_ap[k];
    V.cg_r[k] = r;
    const double z = r / V.cg_diag[k];
    V.cg_z[k] = z;
    rr += r * r;
    rz1 += r * z;
  }
  rr = block_sum<256>(rr, sh);
  rz1 = block_sum<256>(rz1, sh);
  const double beta = rz1 / st->cg_rz;
  for (int k = threadIdx.x; k < n1; k += 256) V.cg_p[k] = V.cg_z[k] + beta * V.cg_p[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    st->cg_rz = rz1;
    st->cg_it += 1;
    st->tot_cg += 1;
    if (sqrt(rr) <= st->cg_rtol * st->cg_bn || st->cg_it >= st->max_cg) st->cg_done = 1;
  }
}

__device__ __forceinline__ void cg_finish_body(const Buffers& B, int d) {
  DevState* st = B.st;
  __shared__ double sh[32];
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  double gd = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) {
    gd += V.g[k] * V.dx[k];
    V.xt[k] = V.x[k] + V.dx[k];
  }
  gd = block_sum<256>(gd, sh);
  if (threadIdx.x == 0) {
    st->gdx = gd;
    st->eta = 1.0;
    st->phase = 1;
    st->bt = 0;
    st->action = ACT_TRIAL;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

// ===========================================================================
// Multiplier update (Algorithm 1): (u, v)^{k+1} = sigma_k Pi(z_k) on the
// support of the accepted point, written to the other buffer, with the
// ball->slot map; the last block flips the buffer parity.
template <bool LOWP = false>
__device__ __forceinline__ void mult_rows_block(const double* __restrict__ C, const Buffers& B,
                                                int d, int bid, int nb) {
  const DevState* st = B.st;
  const int nS = st->nS;
  const int cur = st->sup_cur, nxt = cur ^ 1, nsup = st->nsup;
  const int* sidx = B.sup_idx[cur];
  const double* sv = B.sup_v[cur];
  double* nv = B.sup_v[nxt];
  const double sigma = st->sigma_prev;   // sigma_k of the finished outer step
  const double inv_sigma = 1.0 / sigma;
  const double inv_s = st->inv_s;
  const double* ct = B.vec.ct;        // == s * x (the accepted point)
  const int lane = threadIdx.x & 31;
  for (int k = (bid * 256 + threadIdx.x) >> 5; k < nS; k += (nb * 256) >> 5) {
    const int idx = B.S_idx[k];
    const int sl0 = B.slot[idx];
    const int sl = ((unsigned)sl0 < (unsigned)nsup && sidx[sl0] == idx) ? sl0 : -1;
    const double a = B.S_a[k], n = B.S_n[k];
    const double f = (B.S_case[k] == CASE_I) ? 1.0 : 0.5 * (a + n) / n;
    // with ||v^+||^2 summed as the rows will sum it (lane-strided FMAs, warp tree)
    double vv = 0.0;
    if (LOWP) {
      for (int j = lane; j < d; j += 32) {
        double b = (double)((x32_at(B.X32, st->m_pad, idx, j) - B.vec.y32[j]) * (float)inv_s);
        if (sl >= 0) b = fma(sv[(int64_t)sl * d + j], inv_sigma, b);
        const double v = sigma * f * b;
        nv[(int64_t)k * d + j] = v;
        vv = fma(v, v, vv);
      }
    } else {
      // in units of s: b' = (c_i - c) + v (s / sigma) = s b exactly, and
      // sigma f b = b' (sigma f / s): the same numbers, one multiplication fewer
      const double s_is = inv_sigma * st->s, sfs = (sigma * f) * inv_s;
      for (int j = lane; j < d; j += 32) {
        double b2 = C[(int64_t)idx * d + j] - ct[j];
        if (sl >= 0) b2 = fma(sv[(int64_t)sl * d + j], s_is, b2);
        const double v = b2 * sfs;
        nv[(int64_t)k * d + j] = v;
        vv = fma(v, v, vv);
      }
    }
    vv = warp_sum_t(vv);
    __syncwarp();   // every lane has read the old slot of ball idx
    if (lane == 0) {
      B.sup_vv[nxt][k] = vv;
      B.sup_idx[nxt][k] = idx;
      B.sup_u[nxt][k] = B.S_u[k];
      // the new slot: each ball is in S once, so no other warp reads or
      // writes slot[idx]; balls that left the support keep stale slots that
      // fail the check against the new buffer
      B.slot[idx] = k;
    }
  }
}

// After every multiplier row is written: switch to the new buffers.
__device__ __forceinline__ void mult_flip(DevState* st) {
  st->sup_cur ^= 1;
  st->nsup = st->nS;
  st->action = ACT_NONE;
}

// ===========================================================================
// Solve initialisation (state fields set by the host beforehand): x = xt =
// xk = ab = (r0, c0)/s, trial shadow.
__device__ __forceinline__ void state_init_body(const Buffers& B, int d) {
  __shared__ double sh[32];
  DevState* st = B.st;
  const DevVecs& V = B.vec;
  const double inv_s = st->inv_s;
  for (int k = threadIdx.x; k <= d; k += blockDim.x) {
    const double v = (k == 0) ? st->rt_abs * inv_s : V.c0[k - 1] * inv_s;
    V.x[k] = v; V.xt[k] = v; V.xk[k] = v; V.ab[k] = v;
    V.g[k] = 0.0; V.dx[k] = 0.0;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

// Final centre and ALM radius (unscaled) from the accepted point.
__device__ __forceinline__ void final_point_body(const Buffers& B, int d,
                                                 double* __restrict__ c_out,
                                                 double* __restrict__ r_alm) {
  const DevState* st = B.st;
  const double s = st->s;
  for (int j = threadIdx.x; j < d; j += blockDim.x) c_out[j] = B.vec.x[1 + j] * s;
  if (threadIdx.x == 0) *r_alm = B.vec.x[0] * s;
}

}  // namespace meb
