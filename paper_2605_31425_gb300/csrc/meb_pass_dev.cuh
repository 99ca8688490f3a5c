// Device side of the streaming passes (the bodies of the kernels in
// meb_pass.cu, one pass block at a time): the FP32 and FP16 shadows, the
// screen and the FP64 rows of Algorithm 2's per-ball map, the support-row
// reduction, and the certified feasibility pass of Sec. 4.2.  Each body takes
// its block index (and the block count where it matters) so that the same
// code runs as one block of a multi-block launch or as one step of a single
// block walking a whole pass (the batched solver).
#pragma once
#include <cuda_fp16.h>

#include <type_traits>

#include "meb_control.cuh"
#include "meb_tma.cuh"

namespace meb {


// ===========================================================================
// Shadow: X32[g][i] = fl32(trunc32(c_i[4g..4g+3]) - o) (0 beyond d), with
// o = trunc32(c_0) (the first centre), R32[i] = trunc32(r_i) and E32[i] the
// absolute part of the shadow error (meb_common.cuh); FP32 and integer
// operations only.  A block takes 64 consecutive balls, in chunks of 128
// columns: warp w reads rows w, w + 8, ... coalesced (lanes over columns, 16
// loads in flight per lane), and the tile is written transposed through
// shared memory.  The same sweep checks that every centre and radius is
// finite (and r_i >= 0) and leaves block partials of the shadow column sums
// for the mean centre.
constexpr int kShadowNT = 256;
constexpr int kShadowBalls = 64;
constexpr int kShadowCols = 128;

// One block of the shadow sweep (balls [64 bid, 64 bid + 64)).
__device__ __forceinline__ void shadow_block(int bid, const double* __restrict__ C,
                                             const double* __restrict__ R, int64_t m, int d,
                                             int64_t m_pad, float4* __restrict__ X32,
                                             float* __restrict__ R32, float* __restrict__ E32,
                                             double* __restrict__ colpart, int* __restrict__ bad) {
  __shared__ float tile[kShadowBalls][kShadowCols + 1];
  __shared__ float s_o[kShadowCols];
  __shared__ float s_cs[kShadowNT / 32][kShadowCols];   // per-warp column sums
  const int64_t i0 = (int64_t)bid * kShadowBalls;
  const int nb = (int)imin64(kShadowBalls, m - i0);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int badf = 0;
  float cn[kShadowBalls / 8];   // rows w + 8k: sums of trunc32(c)^2
#pragma unroll
  for (int k = 0; k < kShadowBalls / 8; k++) cn[k] = 0.0f;
  for (int j0 = 0; j0 < d; j0 += kShadowCols) {
    const int nc = min(kShadowCols, d - j0);
    for (int j = threadIdx.x; j < nc; j += kShadowNT) s_o[j] = f64_to_f32_trunc(C[j0 + j]);
    __syncthreads();
    float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // this lane's columns over the warp's rows
#pragma unroll
    for (int h = 0; h < 4; h++) {   // four steps of 2 rows per warp
      double v[2][4];
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const int r = w + 8 * (2 * h + k);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int cc = lane + 32 * q;
          v[k][q] = (r < nb && cc < nc) ? C[(i0 + r) * (int64_t)d + j0 + cc] : 0.0;
        }
      }
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const int r = w + 8 * (2 * h + k);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int cc = lane + 32 * q;
          const unsigned long long bits = (unsigned long long)__double_as_longlong(v[k][q]);
          badf |= ((bits >> 52) & 0x7ff) == 0x7ff;
          const float tc = f64_to_f32_trunc(v[k][q]);
          cn[2 * h + k] = fmaf(tc, tc, cn[2 * h + k]);
          if (r < nb && cc < nc) {
            const float x = tc - s_o[cc];
            tile[r][cc] = x;
            cs[q] += x;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (lane + 32 * q < nc) s_cs[w][lane + 32 * q] = cs[q];
    __syncthreads();
    // transposed write: group g of 4 columns for 64 balls; column sums
    const int ng = (nc + 3) / 4;
    for (int e = threadIdx.x; e < ng * kShadowBalls; e += kShadowNT) {
      const int g = e / kShadowBalls, r = e - g * kShadowBalls;
      if (r < nb) {
        float x[4];
#pragma unroll
        for (int k = 0; k < 4; k++) x[k] = (4 * g + k < nc) ? tile[r][4 * g + k] : 0.0f;
        X32[(int64_t)(j0 / 4 + g) * m_pad + i0 + r] = make_float4(x[0], x[1], x[2], x[3]);
      }
    }
    for (int cc = threadIdx.x; cc < nc; cc += kShadowNT) {
      float t = 0.0f;   // FP32 within the block (the mean is only a starting point)
#pragma unroll
      for (int k = 0; k < kShadowNT / 32; k++) t += s_cs[k][cc];
      colpart[(int64_t)bid * d + j0 + cc] = (double)t;
    }
    __syncthreads();
  }
  // E_i from the row sums of squares (lanes hold column subsets)
#pragma unroll
  for (int k = 0; k < kShadowBalls / 8; k++) {
    float t = cn[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(MEB_FULLMASK, t, o);
    const int r = w + 8 * k;
    if (lane == 0 && r < nb) E32[i0 + r] = shadow_abs_err(t, d);
  }
  for (int r = threadIdx.x; r < nb; r += kShadowNT) {
    const double v = R[i0 + r];
    badf |= !(v >= 0.0) || !isfinite(v);
    R32[i0 + r] = f64_to_f32_trunc(v);
  }
  if (__syncthreads_or(badf) && threadIdx.x == 0) atomicOr(bad, 1);
}

// Origin o = trunc32(c_0) of the shadows, and the starting centre
// c0 = c_0 + (1/m) sum_i x32_i (a mean to FP32 accuracy; exactly c_0 when
// every centre equals c_0): block j sums column j over the block partials in
// a fixed tree order.
__device__ __forceinline__ void shadow_mean_block(int j, const double* __restrict__ C,
                                                  const double* __restrict__ colpart, int nb, int d,
                                                  int64_t m, double* __restrict__ o,
                                                  double* __restrict__ c0) {
  __shared__ double sh[32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) t += colpart[(int64_t)b * d + j];
  t = block_sum<256>(t, sh);
  if (threadIdx.x == 0) {
    o[j] = (double)f64_to_f32_trunc(C[j]);
    c0[j] = C[j] + t / (double)m;
  }
}

// FP16 copy of the shadow in scaled units, x16 = fl16(x32 / s) (round to
// nearest), built once s is known: rows of 8 halves (groups 2k and 2k+1 of
// the FP32 shadow; zeros past d), layout [ceil(d4/2)][m_pad], and per ball
// the error bound eps_i of meb_common.cuh (from N = sum x16^2 by an FP32
// fmaf chain, and E_i).  The screens then read 8 bytes per group of 4 and one
// bound per ball.
// One thread per ball: a warp's reads and writes are 32 consecutive balls of
// one row.
__device__ __forceinline__ void shadow16_block(int bid, const float4* __restrict__ X32,
                                               const float* __restrict__ E32, int64_t m_pad, int d4,
                                               float inv_s, uint4* __restrict__ X16,
                                               float* __restrict__ EPS) {
  const int64_t i = (int64_t)bid * blockDim.x + threadIdx.x;
  if (i >= m_pad) return;
  const int d8 = (d4 + 1) / 2;
  float n = 0.0f;
#pragma unroll 2
  for (int k = 0; k < d8; k++) {
    const float4 v = X32[(int64_t)(2 * k) * m_pad + i];
    const float4 u = (2 * k + 1 < d4) ? X32[(int64_t)(2 * k + 1) * m_pad + i]
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    __half2 h[4];
    h[0] = __floats2half2_rn(v.x * inv_s, v.y * inv_s);
    h[1] = __floats2half2_rn(v.z * inv_s, v.w * inv_s);
    h[2] = __floats2half2_rn(u.x * inv_s, u.y * inv_s);
    h[3] = __floats2half2_rn(u.z * inv_s, u.w * inv_s);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const float2 f = __half22float2(h[q]);
      n = fmaf(f.x, f.x, n);
      n = fmaf(f.y, f.y, n);
    }
    uint4 o;
    o.x = *reinterpret_cast<const unsigned*>(&h[0]);
    o.y = *reinterpret_cast<const unsigned*>(&h[1]);
    o.z = *reinterpret_cast<const unsigned*>(&h[2]);
    o.w = *reinterpret_cast<const unsigned*>(&h[3]);
    X16[(int64_t)k * m_pad + i] = o;
  }
  EPS[i] = half_err(n, E32[i], inv_s, 8 * d8);
}

// ===========================================================================
// The pass, in two kernels over the same block -> tiles map (block b takes the
// tiles [b*T, (b+1)*T) of 256 balls):
//  k_screen : one ball per thread; FP32 certificate from the shadows; the
//             balls it cannot certify (and the balls holding multipliers) are
//             appended, in ball order, to block b's list.
//  k_rows64 : block b evaluates its list in FP64 from the original rows, one
//             warp per ball: projection, multiplier, the per-ball parts of Psi,
//             grad, the stop test and KKT; block partials and the ordered
//             candidates of the support (cases I, M).
struct PassArgs {
  const double* C;
  const double* R;
  int64_t m, m_pad;
  int d, d4, tiles_per_block;
  int log_slot;
  long long wait_cycles;  // bound of the bulk-copy screen's waits (0: one non-blocking test)
  const float4* X32;
  const uint4* X16;     // FP16 shadow scaled by 1/s (8 halves per row), or null
  const float* EPS16;   // per ball: FP16 shadow error bound eps_i (scaled units)
  const float* E32;     // per ball: absolute FP32 shadow error E_i
  const float* R32;
  const int* slot;
  const int* sup_idx0; const int* sup_idx1;
  const double* sup_u0; const double* sup_u1;
  const double* sup_v0; const double* sup_v1;
  const double* sup_vv0; const double* sup_vv1;
  DevState* st;
  const double* ct;
  const float* y32;
  int* unc_cnt;
  int* unc_idx;
  int* unc_slot;
  float* vlb_part;      // per block: sum of max(0, certified lower bound of the violation)^2
  int* part_flag;
  double* part;
  int* part_cnt;
  int* cand_cnt;
  int* cand_idx;
  unsigned char* cand_case;
  double* cand_a; double* cand_n; double* cand_u;
};

// Shadow rows of the screen (one 16-byte load per ball and row): HALF reads
// the FP16 shadow, 8 halves = 2 groups of 4 coordinates per row, in units
// scaled by 1/s; otherwise the FP32 shadow, 1 group per row, unscaled.
template <bool HALF> struct ScreenRaw { using T = float4; static constexpr int kGroups = 1; };
template <> struct ScreenRaw<true> { using T = uint4; static constexpr int kGroups = 2; };
constexpr int kScreenBatch = 4;   // rows per register batch (two batches in flight)

__device__ __forceinline__ float2 h2f(unsigned u) {
  return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

// rows g .. g+kScreenBatch-1 of a ball (p points at its row g, row stride
// m_pad); FULL: all of them exist, else only rows < nrows are read
template <bool HALF, bool FULL>
__device__ __forceinline__ void load_batch(typename ScreenRaw<HALF>::T* r,
                                           const typename ScreenRaw<HALF>::T* __restrict__ p,
                                           int64_t m_pad, int g, int nrows) {
#pragma unroll
  for (int q = 0; q < kScreenBatch; q++) {
    if (FULL || g + q < nrows) r[q] = *p;
    p += m_pad;
  }
}

// S += ||x - y||^2 over coordinate pairs with s_ny = -y (zero past d), in
// packed FP32x2 adds and fmas (each rounds to nearest, as the scalar ones).
__device__ __forceinline__ void acc_pair(float2 x, float2 ny, float2& S) {
  const float2 t = __fadd2_rn(x, ny);
  S = __ffma2_rn(t, t, S);
}

// Sums over the batch; for the FP32 shadow also N += ||x||^2 (the FP16
// shadow's N is precomputed per ball).
template <bool HALF, bool FULL>
__device__ __forceinline__ void sum_batch(const typename ScreenRaw<HALF>::T* r,
                                          const float4* s_ny, int g, int nrows, float2& Sa,
                                          float2& Sb, float2& Na, float2& Nb) {
#pragma unroll
  for (int q = 0; q < kScreenBatch; q++) {
    if (FULL || g + q < nrows) {
      if constexpr (HALF) {
        const uint4 h = r[q];
        const float4 y0 = s_ny[2 * (g + q)], y1 = s_ny[2 * (g + q) + 1];
        acc_pair(h2f(h.x), make_float2(y0.x, y0.y), Sa);
        acc_pair(h2f(h.y), make_float2(y0.z, y0.w), Sb);
        acc_pair(h2f(h.z), make_float2(y1.x, y1.y), Sa);
        acc_pair(h2f(h.w), make_float2(y1.z, y1.w), Sb);
      } else {
        const float4 v = r[q];
        const float4 y = s_ny[g + q];
        const float2 xl = make_float2(v.x, v.y), xh = make_float2(v.z, v.w);
        acc_pair(xl, make_float2(y.x, y.y), Sa);
        acc_pair(xh, make_float2(y.z, y.w), Sb);
        Na = __ffma2_rn(xl, xl, Na);
        Nb = __ffma2_rn(xh, xh, Nb);
      }
    }
  }
}

// The screen of pass block `bid` (its tiles [bid T, (bid + 1) T) of 256 balls).
template <bool HALF>
__device__ __forceinline__ void screen_block(const PassArgs& A, int bid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DevState* st = A.st;
  const int d4 = A.d4;
  float4* s_y = reinterpret_cast<float4*>(smem_raw);
  __shared__ int s_wc[kPassWarps];
  __shared__ float s_v2[kPassWarps];
  // units of the FP16 shadow: multiplying by the power of two 1/s_h is exact
  const float sc = HALF ? (float)st->sh_inv_s : 1.0f;
  const float4* y4 = reinterpret_cast<const float4*>(A.y32);
  constexpr int GR = ScreenRaw<HALF>::kGroups;
  constexpr int NB = kScreenBatch;
  const int nrows = (d4 + GR - 1) / GR;       // shadow rows per ball
  for (int g = threadIdx.x; g < nrows * GR; g += kPassThreads) {
    const float4 y = g < d4 ? y4[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    s_y[g] = make_float4(-y.x * sc, -y.y * sc, -y.z * sc, -y.w * sc);   // -y, scaled
  }
  const int cur = st->sup_cur;
  const int nsup = st->nsup;
  const int* sidx = cur ? A.sup_idx1 : A.sup_idx0;
  const float rq = st->rq32 * sc, yn = st->yn32 * sc;
  const float unsc = HALF ? (float)st->sh_s : 1.0f;
  float v2sum = 0.0f;
  const int k4 = 4 * GR * nrows;   // terms of each sum (padding terms are exact zeros)
  __syncthreads();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t ntiles = (A.m + kPassThreads - 1) / kPassThreads;
  const int64_t t0 = (int64_t)bid * A.tiles_per_block;
  const int64_t t1 = imin64(ntiles, t0 + A.tiles_per_block);
  const int64_t base = t0 * kPassThreads;
  int count = 0;
  for (int64_t tile = t0; tile < t1; tile++) {
    const int64_t i = tile * kPassThreads + tid;
    bool need = false;
    if (i < A.m) {
      // the shadow row is read for every ball (support balls are few): its
      // first batch and the per-ball scalars go out together
      using Raw = typename ScreenRaw<HALF>::T;
      const Raw* xp = (HALF ? reinterpret_cast<const Raw*>(A.X16)
                            : reinterpret_cast<const Raw*>(A.X32)) + i;
      Raw ra[NB], rb[NB];
      const int sl = A.slot[i];
      const float r32 = A.R32[i] * sc;
      const float ex = HALF ? A.EPS16[i] : A.E32[i];
      const int64_t step = (int64_t)NB * A.m_pad;
      float2 Sa = make_float2(0.f, 0.f), Sb = Sa, Na = Sa, Nb = Sa;
      // two register batches in flight: load the next while summing this one
      if (NB <= nrows) load_batch<HALF, true>(ra, xp, A.m_pad, 0, nrows);
      else load_batch<HALF, false>(ra, xp, A.m_pad, 0, nrows);
      for (int g = 0;;) {
        xp += step;
        if (g + 2 * NB <= nrows) load_batch<HALF, true>(rb, xp, A.m_pad, g + NB, nrows);
        else if (g + NB < nrows) load_batch<HALF, false>(rb, xp, A.m_pad, g + NB, nrows);
        if (g + NB <= nrows) sum_batch<HALF, true>(ra, s_y, g, nrows, Sa, Sb, Na, Nb);
        else sum_batch<HALF, false>(ra, s_y, g, nrows, Sa, Sb, Na, Nb);
        g += NB;
        if (g >= nrows) break;
        xp += step;
        if (g + 2 * NB <= nrows) load_batch<HALF, true>(ra, xp, A.m_pad, g + NB, nrows);
        else if (g + NB < nrows) load_batch<HALF, false>(ra, xp, A.m_pad, g + NB, nrows);
        if (g + NB <= nrows) sum_batch<HALF, true>(rb, s_y, g, nrows, Sa, Sb, Na, Nb);
        else sum_batch<HALF, false>(rb, s_y, g, nrows, Sa, Sb, Na, Nb);
        g += NB;
        if (g >= nrows) break;
      }
      const float S = (Sa.x + Sa.y) + (Sb.x + Sb.y);
      const float N = (Na.x + Na.y) + (Nb.x + Nb.y);   // FP32 shadow only
      if ((unsigned)sl < (unsigned)nsup && sidx[sl] == (int)i) {
        need = true;   // the ball holds a multiplier
      } else {
        // certify ||c_i - c|| <= r - r_i from the shadows
        const float ub = HALF ? dist_ub16(S, ex, yn, k4) : dist_ub(S, N, yn, ex, k4);
        const float lb = (rq - r32) - 6.0f * kU32 * (fabsf(rq) + fabsf(r32)) - 1e-30f;
        need = !(ub <= lb);
        if (need) {
          // violation ||c_i - c|| + r_i - r >= D_lb + r32 - rq - margins; with zero
          // multipliers ||Pi(z_i)||^2 >= max(0, violation / s)^2 / 2 (summed unscaled)
          const float dl = HALF ? dist_lb16(S, ex, yn, k4) : dist_lb(S, N, yn, ex, k4);
          const float v = ((dl + r32 - rq) - 3.0f * kU32 * (dl + fabsf(r32) + fabsf(rq))) * unsc;
          if (v > 0.0f) v2sum = fmaf(v, v, v2sum);
        }
      }
    }
    const unsigned msk = __ballot_sync(MEB_FULLMASK, need);
    if (lane == 0) s_wc[w] = __popc(msk);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < kPassWarps; k++) {
      off += (k < w) ? s_wc[k] : 0;
      tot += s_wc[k];
    }
    if (need) {
      const int64_t o = base + count + off + __popc(msk & ((1u << lane) - 1u));
      A.unc_idx[o] = (int)i;
    }
    count += tot;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v2sum += __shfl_xor_sync(MEB_FULLMASK, v2sum, o);
  if (lane == 0) s_v2[w] = v2sum;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
    for (int k = 0; k < kPassWarps; k++) t += s_v2[k];
    A.unc_cnt[bid] = count;
    A.vlb_part[bid] = t;
  }
}

// reuse_lists: the point is the one of the last screen and only the
// multipliers changed; its certificates (zero-multiplier balls strictly
// inside) still hold, and its lists contain every ball that had or gets a
// multiplier.  Only the FP64 rows run again.
__device__ __forceinline__ bool screen_gate(const DevState* st) {
  return !(st->status != 0 || st->action == ACT_DONE || st->reuse_lists);
}

// The FP64 rows of pass block `bid`: its list of uncertain balls.
// LOWP: the low-precision run of the mixed-precision pipeline (Sec. 4.2):
// the rows come from the FP32 shadow (x32 = c_i - o, radii r32, the query
// y32 = trunc32(c - o), fl32(r)) and every per-ball operation and per-lane sum
// is FP32; the block records stay FP64 (their sums are the controller's).
template <bool LOWP = false>
__device__ __forceinline__ void rows_block(const PassArgs& A, int bid) {
  using T = typename std::conditional<LOWP, float, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DevState* st = A.st;
  const int n_b = A.unc_cnt[bid];
  if (n_b == 0) {
    if (threadIdx.x == 0) {
      A.part_flag[bid] = 0;
      A.cand_cnt[bid] = 0;
    }
    return;
  }
  const int d = A.d;
  double* s_ct = reinterpret_cast<double*>(smem_raw);   // d (FP64 rows)
  float* s_yf = reinterpret_cast<float*>(smem_raw);     // d (LOWP: y32)
  __shared__ unsigned char s_cf[kPassThreads];
  __shared__ unsigned char s_cc[kPassThreads];
  __shared__ double s_ca[kPassThreads], s_cn[kPassThreads], s_cu[kPassThreads];
  __shared__ int s_wc[kPassWarps];
  __shared__ double s_wp[kPassWarps][P_NREC];
  __shared__ int s_wn[kPassWarps][P_NCNT];
  for (int j = threadIdx.x; j < d; j += kPassThreads) {
    if (LOWP) s_yf[j] = A.y32[j];
    else s_ct[j] = A.ct[j];
  }
  const int cur = st->sup_cur;
  const int nsup = st->nsup;
  const int* sidx = cur ? A.sup_idx1 : A.sup_idx0;
  const double* su = cur ? A.sup_u1 : A.sup_u0;
  const double* sv = cur ? A.sup_v1 : A.sup_v0;
  const double* svv = cur ? A.sup_vv1 : A.sup_vv0;
  const T inv_s = (T)st->inv_s, sigma = (T)st->sigma, inv_sigma = (T)st->inv_sigma;
  const T rt = LOWP ? (T)st->rq32 : (T)st->rt_abs;
  const float* R32 = A.R32;
  __syncthreads();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)bid * A.tiles_per_block * kPassThreads;
  T acc[P_NREC];
#pragma unroll
  for (int k = 0; k < P_NREC; k++) acc[k] = (T)0;
  int cnt[P_NCNT] = {0, 0, 0};
  int ccount = 0;
  for (int c0 = 0; c0 < n_b; c0 += kPassThreads) {
    const int tot = min(kPassThreads, n_b - c0);
    // warp w takes the 32 chunk entries 32w .. 32w+31; lane q ends with entry q's sums
    const int e0 = 32 * w;
    T mnn = 0, mpp = 0, mdv = 0, mvv = 0;
    const int my = e0 + lane;
    const bool valid = my < tot;
    const int64_t myii = valid ? (int64_t)A.unc_idx[base + c0 + my] : 0;
    int mysl = -1;
    if (valid) {
      const int sl0 = A.slot[myii];
      if ((unsigned)sl0 < (unsigned)nsup && sidx[sl0] == (int)myii) mysl = sl0;
    }
    for (int q = 0; q < 32 && e0 + q < tot; q++) {
      const int64_t ii = __shfl_sync(MEB_FULLMASK, myii, q);
      const int sl = __shfl_sync(MEB_FULLMASK, mysl, q);
      const double* crow = A.C + ii * (int64_t)d;
      T nn = 0, pp = 0, dv = 0, vv = 0;
      if (LOWP) {
        if (sl >= 0) {
          const double* vrow = sv + (int64_t)sl * d;
          for (int j = lane; j < d; j += 32) {
            const T dl = (T)((x32_at(A.X32, A.m_pad, ii, j) - s_yf[j]) * (float)inv_s);
            const T v = (T)vrow[j];
            const T b = fma(v, inv_sigma, dl);
            nn = fma(b, b, nn);
            pp = fma(dl, dl, pp);
            dv = fma(dl, v, dv);
            vv = fma(v, v, vv);
          }
          nn = warp_sum_t(nn); pp = warp_sum_t(pp); dv = warp_sum_t(dv); vv = warp_sum_t(vv);
        } else {
          for (int j = lane; j < d; j += 32) {
            const T dl = (T)((x32_at(A.X32, A.m_pad, ii, j) - s_yf[j]) * (float)inv_s);
            nn = fma(dl, dl, nn);
          }
          nn = warp_sum_t(nn);
          pp = nn;
        }
      } else {
        // in units of s: e = c_i - c (rounded once), dl = e / s and b = dl + v / sigma
        // are exact power-of-two scalings of e and b' = e + v (s / sigma), and so are
        // the sums: one multiplication per coordinate fewer, the same results
        const double s_is = (double)inv_sigma * st->s;
        // ||v||^2 of a support row was summed, in the same order, when the
        // multiplier was written
        double nn2 = 0.0, pp2 = 0.0, dv2 = 0.0, vv2 = 0.0;
        if (sl >= 0) {
          const double* vrow = sv + (int64_t)sl * d;
          for (int j = lane; j < d; j += 32) {
            const double e = crow[j] - s_ct[j];
            const double v = vrow[j];
            const double b2 = fma(v, s_is, e);
            nn2 = fma(b2, b2, nn2);
            pp2 = fma(e, e, pp2);
            dv2 = fma(e, v, dv2);
          }
          nn2 = warp_sum_t(nn2); pp2 = warp_sum_t(pp2); dv2 = warp_sum_t(dv2);
          vv2 = svv[sl];
        } else {
          for (int j = lane; j < d; j += 32) {
            const double e = crow[j] - s_ct[j];
            nn2 = fma(e, e, nn2);
          }
          nn2 = warp_sum_t(nn2);
          pp2 = nn2;
        }
        const double is = (double)inv_s;
        nn = (T)((nn2 * is) * is);
        pp = (T)((pp2 * is) * is);
        dv = (T)(dv2 * is);
        vv = (T)vv2;
      }
      if (lane == q) { mnn = nn; mpp = pp; mdv = dv; mvv = vv; }
    }
    if (valid) {
      const int sl = mysl;
      const int64_t ii = myii;
      const T nn = mnn, pp = mpp, dv = mdv, vv = mvv;
      const T uo = (sl >= 0) ? (T)su[sl] : (T)0;
      const T ri = LOWP ? (T)R32[ii] : (T)A.R[ii];
      const T a = fma(uo, inv_sigma, (ri - rt) * inv_s);
      const T n = sqrt(nn);
      int cs;
      T pa, f, pi2;
      if (n <= a) { cs = CASE_I; pa = a; f = 1; pi2 = a * a + nn; }
      else if (n <= -a) { cs = CASE_Z; pa = 0; f = 0; pi2 = 0; }
      else { cs = CASE_M; pa = (T)0.5 * (a + n); f = pa / n; pi2 = (T)2 * pa * pa; }
      const T up = sigma * pa;
      // b.v = dl.v + ||v||^2/sigma;  ||v^+ - v||^2 = sigma^2 f^2 nn - 2 sigma f (b.v) + vv
      const T bv = dv + vv * inv_sigma;
      const T sf = sigma * f;
      T dvv = sf * sf * nn - (T)2 * sf * bv + vv;
      if (dvv < (T)0) dvv = 0;
      acc[P_PI2] += pi2;
      acc[P_SU] += up;
      acc[P_DUV2] += (up - uo) * (up - uo) + dvv;
      acc[P_UV2] += uo * uo + vv;
      const T ap = (rt - ri) * inv_s;   // (r - r_i)/s
      acc[P_KP] = fmax(acc[P_KP], (T)soc_dist_an((double)ap, sqrt((double)pp)));
      acc[P_KD] = fmax(acc[P_KD], (T)soc_dist_an((double)up, (double)(sf * n)));
      // (r - r_i) u^+ + (c - c_i).v^+ = ap u^+ - sigma f (dl.b), dl.b = pp + dv/sigma
      acc[P_KC] = fmax(acc[P_KC], fabs(ap * up - sf * (pp + dv * inv_sigma)));
      if (cs != CASE_Z) acc[P_ZMAG] += fabs(a) + n;
      cnt[0] += (cs == CASE_I);
      cnt[1] += (cs == CASE_M);
      cnt[2] += 1;
      s_cf[my] = (cs != CASE_Z);
      s_cc[my] = (unsigned char)cs;
      s_ca[my] = a;
      s_cn[my] = n;
      s_cu[my] = up;
    }
    __syncthreads();
    // ordered compaction of the candidates (cases I, M) of this chunk
    const bool cf = (tid < tot) && s_cf[tid];
    const unsigned cm = __ballot_sync(MEB_FULLMASK, cf);
    if (lane == 0) s_wc[w] = __popc(cm);
    __syncthreads();
    int cpos = 0, ctot = 0;
#pragma unroll
    for (int k = 0; k < kPassWarps; k++) {
      cpos += (k < w) ? s_wc[k] : 0;
      ctot += s_wc[k];
    }
    if (cf) {
      const int64_t o = base + ccount + cpos + __popc(cm & ((1u << lane) - 1u));
      A.cand_idx[o] = A.unc_idx[base + c0 + tid];
      A.cand_case[o] = s_cc[tid];
      A.cand_a[o] = s_ca[tid];
      A.cand_n[o] = s_cn[tid];
      A.cand_u[o] = s_cu[tid];
    }
    ccount += ctot;
    __syncthreads();
  }
  // block partial: per-lane accumulators -> warp (fixed trees) -> warps in
  // order.  Warps that took no entry hold zeros and skip the exchanges.
  if (32 * w < n_b) {
    const double v8[8] = {(double)acc[0], (double)acc[1], (double)acc[2], (double)acc[3],
                          (double)acc[4], 0.0, 0.0, 0.0};
    const double sv = warp_sum8_transposed(v8);
    if ((lane & 3) == 0 && (lane >> 2) < P_NSUM) s_wp[w][lane >> 2] = sv;
#pragma unroll
    for (int k = P_NSUM; k < P_NREC; k++) {
      const double mx = warp_max_nonneg((double)acc[k]);
      if (lane == 0) s_wp[w][k] = mx;
    }
#pragma unroll
    for (int k = 0; k < P_NCNT; k++) {
      const int c = (int)__reduce_add_sync(MEB_FULLMASK, (unsigned)cnt[k]);
      if (lane == 0) s_wn[w][k] = c;
    }
  } else if (lane < P_NREC) {
    s_wp[w][lane] = 0.0;
    if (lane < P_NCNT) s_wn[w][lane] = 0;
  }
  __syncthreads();
  if (tid < P_NSUM) {
    double t = 0.0;
    for (int k = 0; k < kPassWarps; k++) t += s_wp[k][tid];
    A.part[(int64_t)bid * P_NREC + tid] = t;
  } else if (tid < P_NREC) {
    long long t = 0;
    for (int k = 0; k < kPassWarps; k++) {
      const long long b = __double_as_longlong(s_wp[k][tid]);
      t = b > t ? b : t;
    }
    A.part[(int64_t)bid * P_NREC + tid] = __longlong_as_double(t);
  } else if (tid >= 32 && tid < 32 + P_NCNT) {
    int t = 0;
    for (int k = 0; k < kPassWarps; k++) t += s_wn[k][tid - 32];
    A.part_cnt[(int64_t)bid * P_NCNT + tid - 32] = t;
  }
  if (tid == 0) {
    A.part_flag[bid] = 1;
    A.cand_cnt[bid] = ccount;
  }
}

__device__ __forceinline__ bool rows_gate(const DevState* st) {
  return !(st->status != 0 || st->action == ACT_DONE || st->action == ACT_TRIAL_EARLY);
}

// ---------------------------------------------------------------------------
// FP16 screen through a bulk-copy pipeline (MEB_OPT_SCREEN = MEB_SCREEN_FP16_BULK).  One block per
// SM keeps `nst` tiles in flight: a tile's shadow rows (16 B per ball and row), error
// bounds, FP32 radii and slots are copied by the TMA engine into a shared
// memory stage and signal its mbarrier; the block sums each ball from shared
// memory, certifies and compacts as k_screen, and the stage is refilled with
// the tile nst ahead once every thread has passed the tile's last barrier.
// Same certificates as k_screen<true> (same sums in the same order).  It
// measured slower than the register-batched screen on GB300 (one block of
// 8 warps per SM leaves each tile's compute and compaction exposed), so it is
// not the default.
constexpr int kBulkSmemBudget = 200 * 1024;
constexpr int kBulkMaxStages = 4;

// stage: [nrows][256] uint4 | eps[256] | r32[256] | slot[256]
__host__ __device__ inline int bulk_stage_bytes(int nrows) { return nrows * 4096 + 3 * 1024; }

// ---------------------------------------------------------------------------
// The plain FP64 pass (screen variant 3): no shadow is read and nothing is
// certified; every ball of the block's tiles is listed, in order, for the
// FP64 rows.  The lower bound of the early rejection is the trivial 0
// (sum ||Pi||^2 >= 0), so that test stays valid.
__device__ __forceinline__ void screen_all_block(const PassArgs& A, int bid) {
  const int64_t ntiles = (A.m + kPassThreads - 1) / kPassThreads;
  const int64_t t0 = (int64_t)bid * A.tiles_per_block;
  const int64_t t1 = imin64(ntiles, t0 + A.tiles_per_block);
  const int64_t base = t0 * kPassThreads;
  const int64_t end = imin64(A.m, t1 * kPassThreads);
  const int n = end > base ? (int)(end - base) : 0;
  for (int k = threadIdx.x; k < n; k += kPassThreads) A.unc_idx[base + k] = (int)(base + k);
  if (threadIdx.x == 0) {
    A.unc_cnt[bid] = n;
    A.vlb_part[bid] = 0.0f;
  }
}

// ===========================================================================
// Support rows: b_k = (c_k - c)/s + v_k/sigma recomputed in FP64;
//   sum v^+ = sigma f_k b_k (all S), sum w_k (case M), sum t_k w_k^2 (case M),
//   sum (1 + t_k) (case M);  W rows w_k = b_k / n_k (M) or b_k (I).
// Block b takes rows [b*rpb, (b+1)*rpb) in order; thread j owns columns j, j+256, ...
constexpr int kSvecStage = 64;   // support rows staged per round in shared memory

// Blocks of the support-row reduction that hold rows: rows per block
// max(8, ceil(nS / nsvb)) for nsvb blocks at most.
__host__ __device__ __forceinline__ int svec_rows_per_block(int nS, int nsvb) {
  int rpb = (nS + nsvb - 1) / nsvb;
  return rpb < 8 ? 8 : rpb;
}

// Support-row block `bid` of at most nsvb (blocks past the rows return).
template <bool LOWP = false>
__device__ __forceinline__ void svec_block(const double* __restrict__ C, const Buffers& B, int d,
                                           int npb, int64_t seg, int bid, int nsvb) {
  DevState* st = B.st;
  const int nS = st->nS;
  const int rpb = svec_rows_per_block(nS, nsvb);
  const int nblk = (nS + rpb - 1) / rpb;
  if (bid == 0 && threadIdx.x == 0) { st->svec_nb = nblk; st->svec_rpb = rpb; }
  if (bid >= nblk) return;
  __shared__ int s_idx[kSvecStage], s_sl[kSvecStage];
  __shared__ int s_off[kMaxPassBlocks + 1];   // candidate segment starts of the pass blocks
  __shared__ unsigned char s_cs[kSvecStage];
  __shared__ double s_sf[kSvecStage], s_in[kSvecStage], s_t[kSvecStage];
  __shared__ float s_t32[kSvecStage];
  __shared__ double s_red[3 * 256];
  __shared__ double sh[32];
  const int k0 = bid * rpb, k1 = min(nS, k0 + rpb);
  const int cur = st->sup_cur, nsup = st->nsup;
  const int* sidx = cur ? B.sup_idx[1] : B.sup_idx[0];
  const double* sv = cur ? B.sup_v[1] : B.sup_v[0];
  const double inv_s = st->inv_s, sigma = st->sigma, inv_sigma = st->inv_sigma;
  const double* ct = B.vec.ct;
  double* out = B.svec_part + (int64_t)bid * (3 * d + 1);
  // G row groups of 32 * ceil(d / 32) threads each take every G-th row (all
  // SMSPs of the SM share the FP64 work); threads past G groups idle
  const int span = 32 * ((d + 31) / 32);
  const int G = span >= 256 ? 1 : 256 / span;
  const int grp = (int)threadIdx.x / (span >= 256 ? 256 : span);
  const int jl = (int)threadIdx.x - grp * (span >= 256 ? 256 : span);
  for (int b = threadIdx.x; b <= npb; b += 256) s_off[b] = B.cand_off[b];
  double s1t = 0.0;
  // stage rows r0 .. r0+nr-1: index, slot (checked), case and the row scalars.
  // Row k of S is entry k - s_off[b] of pass block b's candidate segment
  // (b the last block with s_off[b] <= k); the first column round also writes
  // the ordered support list S for the Newton and multiplier kernels.
  auto stage = [&](int r0, int nr, bool first) {
    if ((int)threadIdx.x < nr) {
      const int k = r0 + threadIdx.x;
      int lo = 0, hi = npb;   // s_off[lo] <= k < s_off[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= k) lo = mid; else hi = mid;
      }
      const int64_t src = (int64_t)lo * seg + (k - s_off[lo]);
      const int idx = B.cand_idx[src];
      const int cs = B.cand_case[src];
      const double a = B.cand_a[src], n = B.cand_n[src];
      if (first) {
        B.S_idx[k] = idx;
        B.S_case[k] = (unsigned char)cs;
        B.S_a[k] = a;
        B.S_n[k] = n;
        B.S_u[k] = B.cand_u[src];
      }
      const int sl0 = B.slot[idx];
      const int sl = ((unsigned)sl0 < (unsigned)nsup && sidx[sl0] == idx) ? sl0 : -1;
      s_idx[threadIdx.x] = idx;
      s_sl[threadIdx.x] = sl;
      s_cs[threadIdx.x] = (unsigned char)cs;
      if (cs == CASE_M) {
        const double in = 1.0 / n;
        const double t = a * in;
        s_in[threadIdx.x] = in;
        s_t[threadIdx.x] = t;
        s_t32[threadIdx.x] = (float)t;
        s_sf[threadIdx.x] = sigma * (0.5 * (a + n) * in);
        if (first) {
          B.S_t[k] = t;
          s1t += 1.0 + t;
        }
      } else {
        s_in[threadIdx.x] = 1.0;
        s_t[threadIdx.x] = 0.0;
        s_t32[threadIdx.x] = 0.0f;
        s_sf[threadIdx.x] = sigma;
        if (first) B.S_t[k] = 0.0;
      }
    }
  };
  if (!LOWP && G == 1 && d >= 512) {
    // wide rows: each thread takes NC columns 256 apart (more loads in flight
    // per thread, the rows staged once for NC columns); every column's sums
    // run over the rows in the same order as with one column per thread
    auto cols = [&](auto ncv) {
      constexpr int NC = decltype(ncv)::value;
      const double s_is = inv_sigma * st->s;
      float* W32 = B.W32;
      for (int j0 = 0; j0 < d; j0 += 256 * NC) {
        double av[NC], aw[NC], atw[NC];
        float atw32[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) {
          av[c] = 0.0; aw[c] = 0.0; atw[c] = 0.0; atw32[c] = 0.0f;
        }
        for (int r0 = k0; r0 < k1; r0 += kSvecStage) {
          const int nr = min(kSvecStage, k1 - r0);
          __syncthreads();
          stage(r0, nr, j0 == 0);
          __syncthreads();
          for (int r = 0; r < nr; r++) {
            const int64_t idx = s_idx[r];
            const int sl = s_sl[r];
            const int64_t k = r0 + r;
            const bool isM = s_cs[r] == CASE_M;
            const double sf = s_sf[r], ins = s_in[r] * inv_s, tt = s_t[r];
            const float t32 = s_t32[r];
#pragma unroll
            for (int c = 0; c < NC; c++) {
              const int j = j0 + 256 * c + jl;
              if (j < d) {
                double b2 = C[idx * d + j] - ct[j];
                if (sl >= 0) b2 = fma(sv[(int64_t)sl * d + j], s_is, b2);
                av[c] = fma(sf, b2, av[c]);
                if (isM) {
                  const double wv = b2 * ins;
                  aw[c] += wv;
                  B.W[k * d + j] = wv;
                  if (W32) {
                    const float w32 = f64_to_f32_trunc(wv);
                    atw32[c] = fmaf(t32 * w32, w32, atw32[c]);
                    W32[k * d + j] = w32;
                  } else {
                    atw[c] = fma(tt * wv, wv, atw[c]);
                  }
                } else {
                  const double b = b2 * inv_s;
                  B.W[k * d + j] = b;
                  if (W32) W32[k * d + j] = f64_to_f32_trunc(b);
                }
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < NC; c++) {
          const int j = j0 + 256 * c + jl;
          if (j < d) {
            out[j] = av[c] * inv_s;
            out[d + j] = aw[c];
            out[2 * d + j] = W32 ? (double)atw32[c] : atw[c];
          }
        }
      }
    };
    if (d >= 1024) cols(std::integral_constant<int, 4>());
    else cols(std::integral_constant<int, 2>());
    s1t = block_sum<256>(s1t, sh);
    if (threadIdx.x == 0) out[3 * d] = s1t;
    return;
  }
  for (int j0 = 0; j0 < d; j0 += 256) {
    const int j = j0 + jl;
    const bool act = grp < G && j < d;
    double av = 0.0, aw = 0.0, atw = 0.0;
    float atw32 = 0.0f;
    for (int r0 = k0; r0 < k1; r0 += kSvecStage) {
      const int nr = min(kSvecStage, k1 - r0);
      __syncthreads();
      // stage the rows: index, slot (checked), case and the row scalars.
      // Row k of S is entry k - s_off[b] of pass block b's candidate segment
      // (b the last block with s_off[b] <= k); the first j-round also writes
      // the ordered support list S for the Newton and multiplier kernels.
      stage(r0, nr, j0 == 0);
      __syncthreads();
      if (act && LOWP) {
        for (int r = grp; r < nr; r += G) {
          const int64_t idx = s_idx[r];
          const int sl = s_sl[r];
          double b = (double)((x32_at(B.X32, st->m_pad, idx, j) - B.vec.y32[j]) * (float)inv_s);
          if (sl >= 0) b = fma(sv[(int64_t)sl * d + j], inv_sigma, b);
          av = fma(s_sf[r], b, av);
          const int64_t k = r0 + r;
          if (s_cs[r] == CASE_M) {
            const double wv = b * s_in[r];
            aw += wv;
            atw = fma(s_t[r] * wv, wv, atw);
            B.W[k * d + j] = wv;
            if (B.W32) B.W32[k * d + j] = (float)wv;
          } else {
            B.W[k * d + j] = b;
            if (B.W32) B.W32[k * d + j] = (float)b;
          }
        }
      } else if (act) {
        // in units of s (as in the rows): b' = (c_k - c) + v (s / sigma) = s b
        // exactly, so w = b / n = b' (1 / (n s)) and sum sf b = (sum sf b') / s
        // are the same numbers with one multiplication per coordinate fewer
        // With FP32 rows for the matrix-free products, those rows and the
        // Jacobi preconditioner's sum t w^2 (both only shape the Newton
        // direction) are formed off the FP64 pipe: the rows by integer
        // truncation, the sum in FP32.
        const double s_is = inv_sigma * st->s;
        float* W32 = B.W32;
        for (int r = grp; r < nr; r += G) {
          const int64_t idx = s_idx[r];
          const int sl = s_sl[r];
          double b2 = C[idx * d + j] - ct[j];
          if (sl >= 0) b2 = fma(sv[(int64_t)sl * d + j], s_is, b2);
          av = fma(s_sf[r], b2, av);
          const int64_t k = r0 + r;
          if (s_cs[r] == CASE_M) {
            const double wv = b2 * (s_in[r] * inv_s);
            aw += wv;
            B.W[k * d + j] = wv;
            if (W32) {
              const float w32 = f64_to_f32_trunc(wv);
              atw32 = fmaf(s_t32[r] * w32, w32, atw32);
              W32[k * d + j] = w32;
            } else {
              atw = fma(s_t[r] * wv, wv, atw);
            }
          } else {
            const double b = b2 * inv_s;
            B.W[k * d + j] = b;
            if (W32) W32[k * d + j] = f64_to_f32_trunc(b);
          }
        }
      }
    }
    if (!LOWP && B.W32) atw = (double)atw32;
    // the groups' sums, in group order
    __syncthreads();
    if (act) {
      s_red[3 * threadIdx.x] = av;
      s_red[3 * threadIdx.x + 1] = aw;
      s_red[3 * threadIdx.x + 2] = atw;
    }
    __syncthreads();
    if (grp == 0 && j < d) {
      const int gs = span >= 256 ? 256 : span;
      for (int g = 1; g < G; g++) {
        const int tt = g * gs + jl;
        av += s_red[3 * tt];
        aw += s_red[3 * tt + 1];
        atw += s_red[3 * tt + 2];
      }
      out[j] = LOWP ? av : av * inv_s;
      out[d + j] = aw;
      out[2 * d + j] = atw;
    }
  }
  s1t = block_sum<256>(s1t, sh);
  if (threadIdx.x == 0) out[3 * d] = s1t;
}

// ===========================================================================
// Certified feasibility pass (Sec. 4.2).  For every ball, e_i = r_i + ||c - c_i||
// (FP64, by definition) and
//   mode 0: val_i = e_i - r;  max val (lowest index on ties), list {val_i > eps}
//   mode 1: val_i = (r - r_i) - ||c - c_i|| (slack);  list {val_i <= eps}
//   mode 2: the maximum of mode 0 only
// Sweep A bounds e_i from the shadows (FP32, rigorous) and keeps the block
// maxima of the lower bounds; sweep B evaluates in FP64 exactly the balls that
// could be the maximum or whose list membership the bounds do not decide.
constexpr int kFeasNT = 256;

struct FeasArgs {
  const double* C; const double* R;
  int64_t m, m_pad;
  int d, d4;
  const float4* X32; const float* R32; const float* E32;
  const double* c;      // query centre (unscaled)
  const float* y32;     // trunc32(c - o), 4*d4 floats
  const float* ynp;     // device: upper bound on ||y32||
  double r, eps;
  int mode;
  int want_max;
  int all64;            // no bounds: every ball evaluated in FP64 (the plain FP64 pass)
  float* eub;           // [m] upper bound on e_i
  float* elb;           // [m] lower bound on e_i
  float* blb;           // [nb] block max of the lower bounds
  double* bmax; int64_t* barg; int* bcnt; int64_t* blist;
  const float* L;       // device: max over blocks of blb
};

__device__ __forceinline__ void feas_a_block(const FeasArgs& A, int bid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_y = reinterpret_cast<float4*>(smem_raw);
  __shared__ float s_m[kFeasNT / 32];
  const float4* y4 = reinterpret_cast<const float4*>(A.y32);
  for (int g = threadIdx.x; g < A.d4; g += kFeasNT) s_y[g] = y4[g];
  __syncthreads();
  const int64_t i = (int64_t)bid * kFeasNT + threadIdx.x;
  float lbv = -INFINITY;
  if (i < A.m) {
    const float4* xp = A.X32 + i;
    float S = 0.f, N = 0.f;
    for (int g = 0; g < A.d4; g++) {
      const float4 xa = xp[(int64_t)g * A.m_pad];
      const float4 ya = s_y[g];
      float t;
      t = xa.x - ya.x; S = fmaf(t, t, S); N = fmaf(xa.x, xa.x, N);
      t = xa.y - ya.y; S = fmaf(t, t, S); N = fmaf(xa.y, xa.y, N);
      t = xa.z - ya.z; S = fmaf(t, t, S); N = fmaf(xa.z, xa.z, N);
      t = xa.w - ya.w; S = fmaf(t, t, S); N = fmaf(xa.w, xa.w, N);
    }
    const int k4 = 4 * A.d4;
    const float yn = *A.ynp;
    const float r32 = A.R32[i];   // r32 <= r_i <= r32 (1 + 2^-23)/(1 - 2^-23)
    const float E = A.E32[i];
    const float eu = (r32 * (1.0f + 5.0f * kU32) + dist_ub(S, N, yn, E, k4)) * (1.0f + 2.0f * kU32);
    const float el = (r32 + dist_lb(S, N, yn, E, k4)) * (1.0f - 2.0f * kU32);
    A.eub[i] = eu;
    A.elb[i] = el;
    lbv = el;
  }
  float t = lbv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(MEB_FULLMASK, t, o));
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = s_m[0];
    for (int k = 1; k < kFeasNT / 32; k++) v = fmaxf(v, s_m[k]);
    A.blb[bid] = v;
  }
}

__device__ __forceinline__ void feas_L_body(const float* __restrict__ blb, int nb,
                                            float* __restrict__ L) {
  __shared__ float sm[256];
  float v = -INFINITY;
  for (int b = threadIdx.x; b < nb; b += 256) v = fmaxf(v, blb[b]);
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *L = sm[0];
}

__device__ __forceinline__ void feas_b_block(const FeasArgs& A, int bid) {
  extern __shared__ double s_c[];
  __shared__ int s_list[kFeasNT];
  __shared__ unsigned char s_in[kFeasNT];     // list membership
  __shared__ double s_v[kFeasNT];
  __shared__ int64_t s_i[kFeasNT];
  __shared__ int s_wc[kFeasNT / 32];
  for (int j = threadIdx.x; j < A.d; j += kFeasNT) s_c[j] = A.c[j];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t i = (int64_t)bid * kFeasNT + tid;
  const double L = (A.want_max && !A.all64) ? (double)*A.L : INFINITY;
  // decide from the bounds; 'need' = evaluate in FP64
  bool need = false;
  unsigned char in = 0;
  if (i < A.m && A.all64) {
    need = true;
  } else if (i < A.m) {
    const double eu = (double)A.eub[i], el = (double)A.elb[i];
    const double ae = isinf(A.eps) ? 0.0 : fabs(A.eps);
    const double tolr = 4.0 * DBL_EPSILON * (fabs(eu) + fabs(A.r) + ae);
    if (A.want_max && eu >= L) need = true;
    if (A.mode == 0) {
      if (el - A.r > A.eps + tolr) in = 1;
      else if (!(eu - A.r <= A.eps - tolr)) need = true;
    } else if (A.mode == 1) {
      // slack in [r - eu, r - el]
      if ((A.r - el) <= A.eps - tolr) in = 1;
      else if (!((A.r - eu) > A.eps + tolr)) need = true;
    }   // mode 2: maximum only
  }
  s_in[tid] = in;
  const unsigned msk = __ballot_sync(MEB_FULLMASK, need);
  if (lane == 0) s_wc[w] = __popc(msk);
  __syncthreads();
  int off = 0, tot = 0;
  for (int k = 0; k < kFeasNT / 32; k++) {
    off += (k < w) ? s_wc[k] : 0;
    tot += s_wc[k];
  }
  if (need) s_list[off + __popc(msk & ((1u << lane) - 1u))] = tid;
  s_v[tid] = -INFINITY;
  s_i[tid] = INT64_MAX;
  __syncthreads();
  // FP64 rows, warp per ball
  for (int k = w; k < tot; k += kFeasNT / 32) {
    const int loc = s_list[k];
    const int64_t ii = (int64_t)bid * kFeasNT + loc;
    const double* row = A.C + ii * (int64_t)A.d;
    double acc = 0.0;
    for (int j = lane; j < A.d; j += 32) {
      const double t = s_c[j] - row[j];
      acc = fma(t, t, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      const double n = sqrt(acc);
      if (A.mode != 1) {
        const double val = (A.R[ii] + n) - A.r;
        s_in[loc] = (A.mode == 0) && (val > A.eps);
        s_v[loc] = val;
        s_i[loc] = ii;
      } else {
        const double val = (A.r - A.R[ii]) - n;
        s_in[loc] = val <= A.eps;
      }
    }
  }
  __syncthreads();
  // block max (lowest index on ties) among the FP64-evaluated balls
  for (int o = kFeasNT / 2; o > 0; o >>= 1) {
    if (tid < o) {
      const double v2 = s_v[tid + o];
      const int64_t i2 = s_i[tid + o];
      if (v2 > s_v[tid] || (v2 == s_v[tid] && i2 < s_i[tid])) { s_v[tid] = v2; s_i[tid] = i2; }
    }
    __syncthreads();
  }
  // ordered list of members of this tile
  const bool fl = (i < A.m) && s_in[tid];
  const unsigned lm = __ballot_sync(MEB_FULLMASK, fl);
  __syncthreads();
  if (lane == 0) s_wc[w] = __popc(lm);
  __syncthreads();
  int loff = 0, ltot = 0;
  for (int k = 0; k < kFeasNT / 32; k++) {
    loff += (k < w) ? s_wc[k] : 0;
    ltot += s_wc[k];
  }
  if (fl) A.blist[(int64_t)bid * kFeasNT + loff + __popc(lm & ((1u << lane) - 1u))] = i;
  if (tid == 0) {
    A.bmax[bid] = s_v[0];
    A.barg[bid] = s_i[0];
    A.bcnt[bid] = ltot;
  }
}

// One block: max over blocks (lowest index on ties), total count.
__device__ __forceinline__ void feas_final_body(const double* __restrict__ bmax,
                                                const int64_t* __restrict__ barg,
                                                const int* __restrict__ bcnt, int nb,
                                                double* out_max, int64_t* out_arg,
                                                int64_t* out_cnt) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  __shared__ long long sc[256];
  double best = -INFINITY;
  int64_t bi = INT64_MAX;
  long long cnt = 0;
  for (int b = threadIdx.x; b < nb; b += 256) {
    const double v = bmax[b];
    const int64_t ix = barg[b];
    if (v > best || (v == best && ix < bi)) { best = v; bi = ix; }
    cnt += bcnt[b];
  }
  sv[threadIdx.x] = best; si[threadIdx.x] = bi; sc[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = sv[threadIdx.x + o];
      const int64_t i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2; si[threadIdx.x] = i2;
      }
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (out_max) *out_max = sv[0];
    if (out_arg) *out_arg = si[0];
    if (out_cnt) *out_cnt = sc[0];
  }
}

// Ordered gather of per-tile lists (tile t holds cnt[t] entries at t*T).
__device__ __forceinline__ void gather_lists_block(int bid, const int* __restrict__ cnt,
                                                   const int64_t* __restrict__ lists, int nb,
                                                   int T, int64_t* __restrict__ out,
                                                   int64_t cap) {
  __shared__ long long sh[256];
  const int b0 = bid * 256;
  long long pre = 0;
  for (int t = threadIdx.x; t < b0; t += 256) pre += cnt[t];
  sh[threadIdx.x] = pre;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const long long base = sh[0];
  __syncthreads();
  const int t = b0 + threadIdx.x;
  const long long my = (t < nb) ? cnt[t] : 0;
  sh[threadIdx.x] = my;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const long long v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < 256; k += 8) {
    const int tt = b0 + k;
    if (tt >= nb) break;
    const long long n = cnt[tt];
    const long long st0 = base + sh[k] - n;
    for (long long e = lane; e < n; e += 32) {
      const long long pos = st0 + e;
      if (pos < cap) out[pos] = lists[(int64_t)tt * T + e];
    }
  }
}

// Query shadow for the feasibility pass: y32 = trunc32(c - o), yn >= ||y32||;
// a non-finite query centre sets *bad (when given).
__device__ __forceinline__ void query_shadow_body(const double* __restrict__ c,
                                                  const double* __restrict__ o, int d,
                                                  float* __restrict__ y32, float* __restrict__ yn,
                                                  int* bad) {
  __shared__ double sh[32];
  const int d4 = (d + 3) / 4;
  double q = 0.0;
  int nf = 0;
  for (int j = threadIdx.x; j < 4 * d4; j += blockDim.x) {
    float y = 0.0f;
    if (j < d) {
      const double cj = c[j];
      nf |= !isfinite(cj);
      y = f64_to_f32_trunc(cj - o[j]);
    }
    y32[j] = y;
    q += (double)y * (double)y;
  }
  if (__syncthreads_or(nf) && threadIdx.x == 0 && bad) atomicOr(bad, 1);
  q = block_sum<256>(q, sh);
  if (threadIdx.x == 0) *yn = __double2float_ru(sqrt(q) * (1.0 + 1e-12));
}

}  // namespace meb
