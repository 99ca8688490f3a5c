// libmeb kernels: the per-ball map-reduce of the ripALM minimum-enclosing-ball
// method (arxiv 2605.31425) for sm_103a.
//
// Notation (Sec. 2 and Sec. 4 of the paper): for ball i with centre c_i and
// radius r_i, at the point x = (r, c) and multipliers (u_i, v_i),
//   z_i = (a_i, b_i) = (r_i - r, c_i - c) + (u_i, v_i)/sigma,
//   (u_i^+, v_i^+) = sigma * Pi_Q(z_i)        (projection onto Q_{d+1}),
// with the three cases of the closed-form projection:
//   I: ||b|| <= a (Pi = z),  Z: ||b|| <= -a (Pi = 0),  M: otherwise.
// All quantities are on the scaled problem (data divided by a power of two s);
// the kernels read the unscaled FP64 input and multiply differences by 1/s,
// which is exact.
//
// Design for GB300: FP64 arithmetic runs at about 2 lanes/clk/SM on this part,
// so the full pass over all balls streams an FP32 shadow of the centres
// (ball-interleaved float4, 4*ceil(d/4) bytes per ball) and certifies with a
// rigorous FP32 error bound that a ball with zero multipliers is strictly
// inside the current ball (case Z, contributes exactly nothing).  Every ball
// that is not certified, and every ball holding a multiplier, is evaluated in
// FP64 from the original row.  All reductions are deterministic: fixed
// block-to-ball maps, in-order per-thread sums and fixed-order trees.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "meb_internal.cuh"

namespace meb {

#define FULLMASK 0xffffffffu

static inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULLMASK, v, o));
  return v;
}

// Block-wide sum in a fixed tree order; all threads get the result.
template <int NT>
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < NT / 32 ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

template <int NT>
__device__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < NT / 32 ? sh[lane] : -INFINITY;
    t = warp_max(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Distance of (a, n) -- a point with ||b|| = n -- to Q: 0 / sqrt(a^2+n^2) / (n-a)/sqrt2.
__device__ __forceinline__ double soc_dist_an(double a, double n) {
  if (n <= a) return 0.0;
  if (n <= -a) return sqrt(a * a + n * n);
  return (n - a) * 0.70710678118654752440;
}

// ===========================================================================
// Column sums of C (for the mean centre c^0), deterministic.
// Block b handles rows [b*rpb, ...); partial[b][j].  Then one block sums the
// partials in block order and divides by m.
__global__ void k_colsum_part(const double* __restrict__ C, int64_t m, int d, int64_t rpb,
                              double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int64_t r1 = min(m, r0 + rpb);
  __shared__ double sh[256];
  if (d <= 256) {
    const int per = 256 / d;           // threads per column
    const int t = threadIdx.x;
    const int j = t % d, ro = t / d;
    double acc = 0.0;
    if (ro < per)
      for (int64_t r = r0 + ro; r < r1; r += per) acc += C[r * d + j];
    sh[t] = (ro < per) ? acc : 0.0;
    __syncthreads();
    if (t < d) {
      double s = 0.0;
      for (int k = 0; k < per; k++) s += sh[t + k * d];
      part[(int64_t)blockIdx.x * d + t] = s;
    }
  } else {
    for (int j = threadIdx.x; j < d; j += 256) {
      double acc = 0.0;
      for (int64_t r = r0; r < r1; r++) acc += C[r * d + j];
      part[(int64_t)blockIdx.x * d + j] = acc;
    }
  }
}

__global__ void k_colsum_final(const double* __restrict__ part, int nb, int d, int64_t m,
                               double* __restrict__ out) {
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[(int64_t)b * d + j];
    out[j] = s / (double)m;
  }
}

cudaError_t launch_colsum(const double* C, int64_t m, int d, double* part, double* out,
                          cudaStream_t s) {
  int nb = (int)imin64(1024, (m + 63) / 64);
  int64_t rpb = (m + nb - 1) / nb;
  nb = (int)((m + rpb - 1) / rpb);
  k_colsum_part<<<nb, 256, 0, s>>>(C, m, d, rpb, part);
  k_colsum_final<<<1, 256, 0, s>>>(part, nb, d, m, out);
  return cudaGetLastError();
}

// ===========================================================================
// Feasibility pass (Sec. 4.2): for every ball, n_i = ||c - c_i|| in FP64.
//   mode 0: val_i = (r_i + n_i) - r; max/argmax (lowest index); list {val_i > eps}
//   mode 1: val_i = (r - r_i) - n_i (slack); list {val_i <= eps}
// e_out (optional): r_i + n_i.  Groups of L lanes per ball (L = pow2 >= d, <= 32).
constexpr int kFeasNT = 256;

__global__ void __launch_bounds__(kFeasNT) k_feas(const double* __restrict__ C,
                                                   const double* __restrict__ R, int64_t m,
                                                   int d, const double* __restrict__ c, double r,
                                                   double eps, int mode, int L,
                                                   double* __restrict__ e_out,
                                                   double* __restrict__ bmax,
                                                   int64_t* __restrict__ barg,
                                                   int* __restrict__ bcnt,
                                                   int64_t* __restrict__ blist) {
  extern __shared__ double s_c[];
  __shared__ unsigned char s_flag[kFeasNT];
  __shared__ double s_v[kFeasNT];
  __shared__ int s_cnt[kFeasNT / 32];
  for (int j = threadIdx.x; j < d; j += kFeasNT) s_c[j] = c[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sub = lane % L, grp = lane / L, gpw = 32 / L;   // groups per warp
  const int64_t tile0 = (int64_t)blockIdx.x * kFeasNT;
  const int per_step = (kFeasNT / 32) * gpw;
  double best = -INFINITY;
  int64_t besti = INT64_MAX;
  for (int base = 0; base < kFeasNT; base += per_step) {
    const int loc = base + w * gpw + grp;
    const int64_t i = tile0 + loc;
    double acc = 0.0;
    if (loc < kFeasNT && i < m) {
      const double* row = C + i * (int64_t)d;
      for (int j = sub; j < d; j += L) {
        double t = s_c[j] - row[j];
        acc = fma(t, t, acc);
      }
    }
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULLMASK, acc, o);
    if (sub == 0 && loc < kFeasNT) {
      unsigned char f = 0;
      double val = -INFINITY;
      if (i < m) {
        double n = sqrt(acc);
        if (e_out) e_out[i] = R[i] + n;
        if (mode == 0) {
          val = (R[i] + n) - r;
          f = val > eps;
          if (val > best || (val == best && i < besti)) { best = val; besti = i; }
        } else {
          val = (r - R[i]) - n;
          f = val <= eps;
        }
      }
      s_flag[loc] = f;
    }
  }
  // block max with lowest index
  s_v[threadIdx.x] = best;
  __syncthreads();
  __shared__ int64_t s_i[kFeasNT];
  s_i[threadIdx.x] = besti;
  __syncthreads();
  for (int o = kFeasNT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = s_v[threadIdx.x + o];
      int64_t i2 = s_i[threadIdx.x + o];
      if (v2 > s_v[threadIdx.x] || (v2 == s_v[threadIdx.x] && i2 < s_i[threadIdx.x])) {
        s_v[threadIdx.x] = v2;
        s_i[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  // ordered compaction of the flagged balls of this tile
  const int64_t i = tile0 + threadIdx.x;
  const bool fl = (i < m) && s_flag[threadIdx.x];
  unsigned msk = __ballot_sync(FULLMASK, fl);
  if (lane == 0) s_cnt[w] = __popc(msk);
  __syncthreads();
  int off = 0, tot = 0;
  for (int k = 0; k < kFeasNT / 32; k++) {
    if (k < w) off += s_cnt[k];
    tot += s_cnt[k];
  }
  if (fl) blist[tile0 + off + __popc(msk & ((1u << lane) - 1u))] = i;
  if (threadIdx.x == 0) {
    bmax[blockIdx.x] = s_v[0];
    barg[blockIdx.x] = s_i[0];
    bcnt[blockIdx.x] = tot;
  }
}

// One block: max over blocks (lowest index on ties), total count.
__global__ void k_feas_final(const double* __restrict__ bmax, const int64_t* __restrict__ barg,
                             const int* __restrict__ bcnt, int nb, double* out_max,
                             int64_t* out_arg, int64_t* out_cnt) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  __shared__ long long sc[256];
  double best = -INFINITY;
  int64_t bi = INT64_MAX;
  long long cnt = 0;
  for (int b = threadIdx.x; b < nb; b += 256) {
    double v = bmax[b];
    int64_t ix = barg[b];
    if (v > best || (v == best && ix < bi)) { best = v; bi = ix; }
    cnt += bcnt[b];
  }
  sv[threadIdx.x] = best; si[threadIdx.x] = bi; sc[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = sv[threadIdx.x + o];
      int64_t i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2; si[threadIdx.x] = i2;
      }
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { *out_max = sv[0]; *out_arg = si[0]; *out_cnt = sc[0]; }
}

// Ordered gather of per-tile lists (tile t holds cnt[t] entries at t*T) into out[].
__global__ void k_gather_lists(const int* __restrict__ cnt, const int64_t* __restrict__ lists,
                               int nb, int T, int64_t* __restrict__ out, int64_t cap) {
  __shared__ long long sh[256];
  // blocks of 256 tiles; base = sum of counts of all earlier tiles
  const int b0 = blockIdx.x * 256;
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
  long long my = (t < nb) ? cnt[t] : 0;
  sh[threadIdx.x] = my;
  __syncthreads();
  // inclusive scan (Hillis-Steele)
  for (int o = 1; o < 256; o <<= 1) {
    long long v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  const long long excl = sh[threadIdx.x] - my;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // warp w copies tiles b0 + w, b0 + w + 8, ...
  for (int k = w; k < 256; k += 8) {
    const int tt = b0 + k;
    if (tt >= nb) break;
    const long long n = cnt[tt];
    const long long st0 = base + sh[k] - n;
    for (long long e = lane; e < n; e += 32) {
      long long pos = st0 + e;
      if (pos < cap) out[pos] = lists[(int64_t)tt * T + e];
    }
  }
  (void)excl;
}

// Sum of per-tile counts into *out (one block).
__global__ void k_count_sum(const int* __restrict__ cnt, int nb, int64_t* __restrict__ out) {
  __shared__ long long sh[256];
  long long s = 0;
  for (int b = threadIdx.x; b < nb; b += 256) s += cnt[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_feas(const double* C, const double* R, int64_t m, int d, const double* c,
                        double r, double eps, int mode, double* e_out, Buffers& B,
                        double* dmax_out, int64_t* argmax_out, int64_t* nviol_out,
                        cudaStream_t s) {
  int L = 1;
  while (L < d && L < 32) L <<= 1;
  const int nb = (int)((m + kFeasNT - 1) / kFeasNT);
  size_t sh = sizeof(double) * (size_t)d;
  if (sh > 48 * 1024) {
    cudaError_t e0 = cudaFuncSetAttribute(k_feas, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e0 != cudaSuccess) return e0;
  }
  k_feas<<<nb, kFeasNT, sh, s>>>(C, R, m, d, c, r, eps, mode, L, e_out, B.feas_part,
                                 B.feas_ipart, B.feas_cnt, B.list_tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_feas_final<<<1, 256, 0, s>>>(B.feas_part, B.feas_ipart, B.feas_cnt, nb, dmax_out,
                                 argmax_out, nviol_out);
  k_gather_lists<<<(nb + 255) / 256, 256, 0, s>>>(B.feas_cnt, B.list_tmp, nb, kFeasNT, B.viol, m);
  B.launches += 3;
  return cudaGetLastError();
}

// ===========================================================================
// FP32 shadow of the scaled, centred data (built once per solve):
//   X32[g][i] = (fl32(c_i[4g..4g+3] - o) * (1/s)),   R32[i] = fl32(r_i) * (1/s).
// fl32 is round-to-nearest; multiplying by the power of two 1/s is exact.
__global__ void k_shadow(const double* __restrict__ C, const double* __restrict__ R, int64_t m,
                         int d, int64_t m_pad, const double* __restrict__ o, float inv_s,
                         float4* __restrict__ X32, float* __restrict__ R32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (i >= m) return;
  const double* row = C + i * (int64_t)d;
  float v[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    int j = 4 * g + k;
    v[k] = (j < d) ? __double2float_rn(row[j] - o[j]) * inv_s : 0.0f;
  }
  X32[(int64_t)g * m_pad + i] = make_float4(v[0], v[1], v[2], v[3]);
  if (g == 0) R32[i] = __double2float_rn(R[i]) * inv_s;
}

cudaError_t launch_shadow(const double* C, const double* R, int64_t m, int d, int64_t m_pad,
                          const double* o, double inv_s, float4* X32, float* R32,
                          cudaStream_t s) {
  const int d4 = (d + 3) / 4;
  dim3 grid((unsigned)((m + 255) / 256), (unsigned)d4);
  k_shadow<<<grid, 256, 0, s>>>(C, R, m, d, m_pad, o, (float)inv_s, X32, R32);
  return cudaGetLastError();
}

// ===========================================================================
// The pass (Algorithm 2, step 1 + the per-ball parts of step 2): one thread
// per ball for the FP32 certificate, one warp per ball for the FP64 rows.
struct PassArgs {
  const double* C;
  const double* R;
  int64_t m, m_pad;
  int d, d4;
  const float4* X32;
  const float* R32;
  const int* slot;
  const int* sup_idx0; const int* sup_idx1;
  const double* sup_u0; const double* sup_u1;
  const double* sup_v0; const double* sup_v1;
  DevState* st;
  const double* ct;
  const float* y32;
  int* part_flag;
  double* part;
  int* cand_cnt;
  int* cand_idx;
  unsigned char* cand_case;
  double* cand_a; double* cand_n; double* cand_u;
};

__global__ void __launch_bounds__(kPassThreads) k_pass(PassArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DevState* st = A.st;
  if (st->status != 0 || st->action == ACT_DONE) return;
  const int d = A.d, d4 = A.d4;
  float4* s_y = reinterpret_cast<float4*>(smem_raw);                    // d4
  double* s_ct = reinterpret_cast<double*>(smem_raw + 16 * (size_t)d4);  // d
  __shared__ int s_list[kPassThreads];
  __shared__ int s_lslot[kPassThreads];
  __shared__ unsigned char s_cf[kPassThreads];   // candidate flag per list entry
  __shared__ unsigned char s_cc[kPassThreads];
  __shared__ double s_ca[kPassThreads], s_cn[kPassThreads], s_cu[kPassThreads];
  __shared__ int s_wc[kPassWarps];
  __shared__ double s_wp[kPassWarps][P_COUNT];

  const float4* y4 = reinterpret_cast<const float4*>(A.y32);
  for (int g = threadIdx.x; g < d4; g += kPassThreads) s_y[g] = y4[g];
  for (int j = threadIdx.x; j < d; j += kPassThreads) s_ct[j] = A.ct[j];
  const int cur = st->sup_cur;
  const int nsup = st->nsup;
  const int* sidx = cur ? A.sup_idx1 : A.sup_idx0;
  const double* su = cur ? A.sup_u1 : A.sup_u0;
  const double* sv = cur ? A.sup_v1 : A.sup_v0;
  const double inv_s = st->inv_s, sigma = st->sigma, inv_sigma = st->inv_sigma;
  const double rt = st->rt_abs;
  const float rq = st->rq32, yn = st->yn32;
  __syncthreads();

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t i = (int64_t)blockIdx.x * kPassThreads + tid;
  bool need = false;
  int myslot = -1;
  if (i < A.m) {
    const int sl = A.slot[i];
    if ((unsigned)sl < (unsigned)nsup && sidx[sl] == (int)i) myslot = sl;
    if (myslot >= 0) {
      need = true;
    } else {
      // FP32 certificate that ||c_i - c|| <= r - r_i with margin.
      const float4* xp = A.X32 + i;
      float S0 = 0.f, S1 = 0.f, N0 = 0.f, N1 = 0.f;
      int g = 0;
      for (; g + 1 < d4; g += 2) {
        float4 xa = xp[(int64_t)g * A.m_pad];
        float4 xb = xp[(int64_t)(g + 1) * A.m_pad];
        float4 ya = s_y[g], yb = s_y[g + 1];
        float t;
        t = xa.x - ya.x; S0 = fmaf(t, t, S0); N0 = fmaf(xa.x, xa.x, N0);
        t = xa.y - ya.y; S0 = fmaf(t, t, S0); N0 = fmaf(xa.y, xa.y, N0);
        t = xa.z - ya.z; S0 = fmaf(t, t, S0); N0 = fmaf(xa.z, xa.z, N0);
        t = xa.w - ya.w; S0 = fmaf(t, t, S0); N0 = fmaf(xa.w, xa.w, N0);
        t = xb.x - yb.x; S1 = fmaf(t, t, S1); N1 = fmaf(xb.x, xb.x, N1);
        t = xb.y - yb.y; S1 = fmaf(t, t, S1); N1 = fmaf(xb.y, xb.y, N1);
        t = xb.z - yb.z; S1 = fmaf(t, t, S1); N1 = fmaf(xb.z, xb.z, N1);
        t = xb.w - yb.w; S1 = fmaf(t, t, S1); N1 = fmaf(xb.w, xb.w, N1);
      }
      if (g < d4) {
        float4 xa = xp[(int64_t)g * A.m_pad];
        float4 ya = s_y[g];
        float t;
        t = xa.x - ya.x; S0 = fmaf(t, t, S0); N0 = fmaf(xa.x, xa.x, N0);
        t = xa.y - ya.y; S0 = fmaf(t, t, S0); N0 = fmaf(xa.y, xa.y, N0);
        t = xa.z - ya.z; S0 = fmaf(t, t, S0); N0 = fmaf(xa.z, xa.z, N0);
        t = xa.w - ya.w; S0 = fmaf(t, t, S0); N0 = fmaf(xa.w, xa.w, N0);
      }
      const float S = S0 + S1, N = N0 + N1;
      // Error bound (u = 2^-24, every op round-to-nearest, fmaf sums):
      //   ||x_i - y|| <= (sqrt(S) + 1.01u (sqrt(N) + yn)) * (1 + (d4*4 + 16) u)
      //   (r - r_i)/s >= (rq - r32_i) - 5u (|rq| + |r32_i|)
      const float u = 5.9604645e-08f;
      const float r32 = A.R32[i];
      const float ub = (sqrtf(S) + 1.01f * u * (sqrtf(N) + yn)) *
                           (1.0f + (float)(4 * d4 + 16) * u) + 1e-30f;
      const float lb = (rq - r32) - 5.0f * u * (fabsf(rq) + fabsf(r32)) - 1e-30f;
      need = !(ub <= lb);
    }
  }
  // ordered compaction of the balls that need FP64
  const unsigned msk = __ballot_sync(FULLMASK, need);
  if (lane == 0) s_wc[w] = __popc(msk);
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < kPassWarps; k++) {
    off += (k < w) ? s_wc[k] : 0;
    tot += s_wc[k];
  }
  if (need) {
    const int pos = off + __popc(msk & ((1u << lane) - 1u));
    s_list[pos] = tid;
    s_lslot[pos] = myslot;
  }
  __syncthreads();
  if (tot == 0) {
    if (tid == 0) {
      A.part_flag[blockIdx.x] = 0;
      A.cand_cnt[blockIdx.x] = 0;
    }
    return;
  }

  // FP64 rows: warp w takes list entries w, w + 8, ...
  double acc[P_COUNT];
#pragma unroll
  for (int k = 0; k < P_COUNT; k++) acc[k] = 0.0;
  for (int k = w; k < tot; k += kPassWarps) {
    const int64_t ii = (int64_t)blockIdx.x * kPassThreads + s_list[k];
    const int sl = s_lslot[k];
    const double* crow = A.C + ii * (int64_t)d;
    double nn = 0.0, pp = 0.0, dv = 0.0, vv = 0.0;
    if (sl >= 0) {
      const double* vrow = sv + (int64_t)sl * d;
      for (int j = lane; j < d; j += 32) {
        const double dl = (crow[j] - s_ct[j]) * inv_s;
        const double v = vrow[j];
        const double b = fma(v, inv_sigma, dl);
        nn = fma(b, b, nn);
        pp = fma(dl, dl, pp);
        dv = fma(dl, v, dv);
        vv = fma(v, v, vv);
      }
      nn = warp_sum(nn); pp = warp_sum(pp); dv = warp_sum(dv); vv = warp_sum(vv);
    } else {
      for (int j = lane; j < d; j += 32) {
        const double dl = (crow[j] - s_ct[j]) * inv_s;
        nn = fma(dl, dl, nn);
      }
      nn = warp_sum(nn);
      pp = nn;
    }
    if (lane == 0) {
      const double uo = (sl >= 0) ? su[sl] : 0.0;
      const double a = fma(uo, inv_sigma, (A.R[ii] - rt) * inv_s);
      const double n = sqrt(nn);
      int cs;
      double pa, f, pi2;
      if (n <= a) { cs = CASE_I; pa = a; f = 1.0; pi2 = a * a + nn; }
      else if (n <= -a) { cs = CASE_Z; pa = 0.0; f = 0.0; pi2 = 0.0; }
      else { cs = CASE_M; pa = 0.5 * (a + n); f = pa / n; pi2 = 2.0 * pa * pa; }
      const double up = sigma * pa;
      // b.v = dl.v + ||v||^2 / sigma ; ||v^+ - v||^2 = sigma^2 f^2 nn - 2 sigma f (b.v) + vv
      const double bv = dv + vv * inv_sigma;
      const double sf = sigma * f;
      double dvv = sf * sf * nn - 2.0 * sf * bv + vv;
      if (dvv < 0.0) dvv = 0.0;
      acc[P_PI2] += pi2;
      acc[P_SU] += up;
      acc[P_DUV2] += (up - uo) * (up - uo) + dvv;
      acc[P_UV2] += uo * uo + vv;
      // KKT terms at the evaluated point with the new multipliers
      const double ap = (rt - A.R[ii]) * inv_s;          // (r - r_i)/s
      acc[P_KP] = fmax(acc[P_KP], soc_dist_an(ap, sqrt(pp)));
      acc[P_KD] = fmax(acc[P_KD], soc_dist_an(up, sf * n));
      // (r - r_i) u^+ + (c - c_i).v^+ = ap u^+ - sigma f (dl.b),  dl.b = pp + dv/sigma
      acc[P_KC] = fmax(acc[P_KC], fabs(ap * up - sf * (pp + dv * inv_sigma)));
      if (cs != CASE_Z) acc[P_ZMAG] += fabs(a) + n;
      acc[P_NI] += (cs == CASE_I);
      acc[P_NM] += (cs == CASE_M);
      acc[P_N64] += 1.0;
      s_cf[k] = (cs != CASE_Z);
      s_cc[k] = (unsigned char)cs;
      s_ca[k] = a;
      s_cn[k] = n;
      s_cu[k] = up;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < P_COUNT; k++) s_wp[w][k] = acc[k];
  }
  __syncthreads();
  // block partial: warps in order
  if (tid < P_COUNT) {
    const bool ismax = (tid == P_KP || tid == P_KD || tid == P_KC);
    double t = 0.0;
    for (int k = 0; k < kPassWarps; k++) t = ismax ? fmax(t, s_wp[k][tid]) : t + s_wp[k][tid];
    A.part[(int64_t)blockIdx.x * P_COUNT + tid] = t;
  }
  // ordered compaction of the candidates (cases I, M) among the list entries
  int cpos = 0;
  const bool cf = (tid < tot) && s_cf[tid];
  const unsigned cm = __ballot_sync(FULLMASK, cf);
  __syncthreads();
  if (lane == 0) s_wc[w] = __popc(cm);
  __syncthreads();
  int ctot = 0;
#pragma unroll
  for (int k = 0; k < kPassWarps; k++) {
    cpos += (k < w) ? s_wc[k] : 0;
    ctot += s_wc[k];
  }
  if (cf) {
    const int64_t o = (int64_t)blockIdx.x * kPassThreads + cpos + __popc(cm & ((1u << lane) - 1u));
    A.cand_idx[o] = (int)((int64_t)blockIdx.x * kPassThreads + s_list[tid]);
    A.cand_case[o] = s_cc[tid];
    A.cand_a[o] = s_ca[tid];
    A.cand_n[o] = s_cn[tid];
    A.cand_u[o] = s_cu[tid];
  }
  if (tid == 0) {
    A.part_flag[blockIdx.x] = 1;
    A.cand_cnt[blockIdx.x] = ctot;
  }
}

// Ordered gather of the pass candidates into the support list S.
__global__ void k_compact_S(Buffers B, int nb) {
  DevState* st = B.st;
  if (st->status != 0 || st->action == ACT_DONE) return;
  __shared__ long long sh[256];
  __shared__ long long sc[256];
  const int b0 = blockIdx.x * 256;
  long long pre = 0;
  for (int t = threadIdx.x; t < b0; t += 256) pre += B.cand_cnt[t];
  sh[threadIdx.x] = pre;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const long long base = sh[0];
  __syncthreads();
  const int t = b0 + threadIdx.x;
  sc[threadIdx.x] = (t < nb) ? B.cand_cnt[t] : 0;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    long long v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
    __syncthreads();
    sc[threadIdx.x] += v;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < 256; k += 8) {
    const int tt = b0 + k;
    if (tt >= nb) break;
    const long long n = B.cand_cnt[tt];
    const long long s0 = base + sc[k] - n;
    for (long long e = lane; e < n; e += 32) {
      const int64_t src = (int64_t)tt * kPassThreads + e;
      const int64_t dst = s0 + e;
      B.S_idx[dst] = B.cand_idx[src];
      B.S_case[dst] = B.cand_case[src];
      B.S_a[dst] = B.cand_a[src];
      B.S_n[dst] = B.cand_n[src];
      B.S_u[dst] = B.cand_u[src];
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 255) st->nS = (int)(base + sc[255]);
}

// Support rows: b_k = (c_k - c)/s + v_k/sigma recomputed in FP64;
//   sum v^+ = sigma f_k b_k (all S), sum w_k (case M), sum (1 + t_k) (case M),
//   sum t_k w_k^2 (case M, for the Jacobi preconditioner);
// W rows (w_k = b_k / n_k) for the Hessian.  Block b takes rows
// [b*rpb, (b+1)*rpb) in order; thread j owns columns j, j + 256, ...
__global__ void __launch_bounds__(256) k_svec(const double* __restrict__ C, Buffers B, int d) {
  DevState* st = B.st;
  if (st->status != 0 || st->action == ACT_DONE) return;
  const int nS = st->nS;
  int rpb = (nS + kSvecBlocks - 1) / kSvecBlocks;
  if (rpb < 8) rpb = 8;
  const int nblk = (nS + rpb - 1) / rpb;
  if (blockIdx.x == 0 && threadIdx.x == 0) { st->svec_nb = nblk; st->svec_rpb = rpb; }
  if ((int)blockIdx.x >= nblk) return;
  const int k0 = blockIdx.x * rpb, k1 = min(nS, k0 + rpb);
  const int cur = st->sup_cur, nsup = st->nsup;
  const int* sidx = cur ? B.sup_idx[1] : B.sup_idx[0];
  const double* sv = cur ? B.sup_v[1] : B.sup_v[0];
  const double inv_s = st->inv_s, sigma = st->sigma, inv_sigma = st->inv_sigma;
  const double* ct = B.vec.ct;
  double* out = B.svec_part + (int64_t)blockIdx.x * (3 * d + 1);
  double s1t = 0.0;
  for (int j0 = 0; j0 < d; j0 += 256) {
    const int j = j0 + threadIdx.x;
    double av = 0.0, aw = 0.0, atw = 0.0;
    for (int k = k0; k < k1; k++) {
      const int idx = B.S_idx[k];
      const int cs = B.S_case[k];
      const double a = B.S_a[k], n = B.S_n[k];
      const int sl0 = B.slot[idx];
      const int sl = ((unsigned)sl0 < (unsigned)nsup && sidx[sl0] == idx) ? sl0 : -1;
      if (j0 == 0 && threadIdx.x == 0) {
        const double t = (cs == CASE_M) ? a / n : 0.0;
        B.S_t[k] = t;
        if (cs == CASE_M) s1t += 1.0 + t;
      }
      if (j < d) {
        double b = (C[(int64_t)idx * d + j] - ct[j]) * inv_s;
        if (sl >= 0) b = fma(sv[(int64_t)sl * d + j], inv_sigma, b);
        if (cs == CASE_I) {
          av += sigma * b;
          B.W[(int64_t)k * d + j] = b;
        } else {
          const double f = 0.5 * (a + n) / n;
          const double wv = b / n;
          const double t = a / n;
          av += sigma * f * b;
          aw += wv;
          atw += t * wv * wv;
          B.W[(int64_t)k * d + j] = wv;
        }
      }
    }
    if (j < d) {
      out[j] = av;
      out[d + j] = aw;
      out[2 * d + j] = atw;
    }
  }
  if (threadIdx.x == 0) out[3 * d] = s1t;
}

cudaError_t launch_pass(const double* C, const double* R, Buffers& B, int64_t m, int d,
                        cudaStream_t s) {
  PassArgs A;
  A.C = C; A.R = R; A.m = m;
  const int d4 = (d + 3) / 4;
  A.m_pad = ((m + 255) / 256) * 256;
  A.d = d; A.d4 = d4;
  A.X32 = B.X32; A.R32 = B.R32; A.slot = B.slot;
  A.sup_idx0 = B.sup_idx[0]; A.sup_idx1 = B.sup_idx[1];
  A.sup_u0 = B.sup_u[0]; A.sup_u1 = B.sup_u[1];
  A.sup_v0 = B.sup_v[0]; A.sup_v1 = B.sup_v[1];
  A.st = B.st; A.ct = B.vec.ct; A.y32 = B.vec.y32;
  A.part_flag = B.part_flag; A.part = B.part;
  A.cand_cnt = B.cand_cnt; A.cand_idx = B.cand_idx; A.cand_case = B.cand_case;
  A.cand_a = B.cand_a; A.cand_n = B.cand_n; A.cand_u = B.cand_u;
  const int nb = (int)((m + kPassThreads - 1) / kPassThreads);
  const size_t sh = 16 * (size_t)d4 + 8 * (size_t)d;
  if (sh > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  k_pass<<<nb, kPassThreads, sh, s>>>(A);
  B.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_pass_post(const double* C, Buffers& B, int64_t m, int d, cudaStream_t s) {
  const int nb = (int)((m + kPassThreads - 1) / kPassThreads);
  k_compact_S<<<(nb + 255) / 256, 256, 0, s>>>(B, nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_svec<<<kSvecBlocks, 256, 0, s>>>(C, B, d);
  B.launches += 2;
  return cudaGetLastError();
}

// ===========================================================================
// Controller (one block): reduces the pass, forms grad and Psi, and takes the
// decisions of Algorithms 1 and 2.  Vector work is spread over the block.

// Trial shadow: ct = s * xt[1:], rt = s * xt[0], y32 = fl32(ct - o) / s.
__device__ void set_trial(DevState* st, const DevVecs& V, int d, double* sh) {
  const double s = st->s;
  const float inv_s = (float)st->inv_s;
  double q = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double c = V.xt[1 + j] * s;
    V.ct[j] = c;
    const float y = __double2float_rn(c - V.o[j]) * inv_s;
    V.y32[j] = y;
    q += (double)y * (double)y;
  }
  const int d4 = (d + 3) / 4;
  for (int j = d + threadIdx.x; j < 4 * d4; j += blockDim.x) V.y32[j] = 0.0f;
  q = block_sum<256>(q, sh);
  if (threadIdx.x == 0) {
    st->rt_abs = V.xt[0] * s;
    st->rq32 = __double2float_rn(V.xt[0]);
    st->yn32 = __double2float_ru(sqrt(q) * (1.0 + 1e-12));
  }
  __syncthreads();
}

// Outer update (Algorithm 1): (alpha,beta) -= sigma g, KKT_max, sigma rule.
// Returns the action; thread 0 writes the state.
__device__ void do_outer(DevState* st, const DevVecs& V, int d, double* sh) {
  const int n1 = d + 1;
  const double sigma = st->sigma;
  for (int k = threadIdx.x; k < n1; k += blockDim.x) V.ab[k] -= sigma * V.g[k];
  double q = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) q += V.sv[j] * V.sv[j];
  q = block_sum<256>(q, sh);
  __shared__ int s_act;
  if (threadIdx.x == 0) {
    st->kkt[0] = fabs(1.0 - st->last[P_SU]);
    st->kkt[1] = sqrt(q);
    st->kkt[2] = st->last[P_KP];
    st->kkt[3] = st->last[P_KD];
    st->kkt[4] = st->last[P_KC];
    double km = 0.0;
    for (int k = 0; k < 5; k++) km = fmax(km, st->kkt[k]);
    st->kkt_max = km;
    st->outer += 1;
    int act;
    if (km <= st->tol) { st->status = 1; act = ACT_DONE; }
    else if (st->outer >= st->max_outer) { st->status = 2; act = ACT_DONE; }
    else {
      act = ACT_OUTER;
      const double pinf = st->last[P_KP];
      // the multiplier update uses the sigma of the finished outer step
      st->sigma_prev = sigma;
      if (pinf > st->tol && pinf > st->sigma_ratio * st->pinf_prev) {
        double sg = sigma * st->sigma_growth;
        if (sg > st->sigma_max) sg = st->sigma_max;
        st->sigma = sg;
        st->inv_sigma = 1.0 / sg;
      }
      st->pinf_prev = pinf;
      st->phase = 0;
    }
    st->action = act;
    s_act = act;
  }
  __syncthreads();
  if (s_act == ACT_OUTER) {
    for (int k = threadIdx.x; k < n1; k += blockDim.x) {
      V.xk[k] = V.x[k];
      V.xt[k] = V.x[k];
    }
    __syncthreads();
    set_trial(st, V, d, sh);
  }
}

__global__ void __launch_bounds__(256) k_control(Buffers B, int d, int nb) {
  DevState* st = B.st;
  if (st->status != 0 || st->action == ACT_DONE) return;
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  __shared__ double sh[32];
  __shared__ double s_last[P_COUNT];
  __shared__ int s_next;

  // 1. reduce the pass partials over the active blocks, in block order
  {
    double acc[P_COUNT];
#pragma unroll
    for (int k = 0; k < P_COUNT; k++) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) {
      if (!B.part_flag[b]) continue;
      const double* p = B.part + (int64_t)b * P_COUNT;
#pragma unroll
      for (int k = 0; k < P_COUNT; k++) {
        const bool ismax = (k == P_KP || k == P_KD || k == P_KC);
        acc[k] = ismax ? fmax(acc[k], p[k]) : acc[k] + p[k];
      }
    }
#pragma unroll
    for (int k = 0; k < P_COUNT; k++) {
      const bool ismax = (k == P_KP || k == P_KD || k == P_KC);
      const double r = ismax ? block_max<256>(acc[k], sh) : block_sum<256>(acc[k], sh);
      if (threadIdx.x == 0) s_last[k] = r;
    }
  }
  __syncthreads();
  // 2. support-row vectors: sum over the svec blocks in order
  const int snb = st->svec_nb;
  double s1t_part = 0.0;
  for (int j = threadIdx.x; j < d; j += 256) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < snb; k++) {
      const double* p = B.svec_part + (int64_t)k * (3 * d + 1);
      a += p[j];
      b += p[d + j];
      c += p[2 * d + j];
    }
    V.sv[j] = a;
    V.sw[j] = b;
    V.cg_diag[1 + j] = c;   // sum_M t w_j^2 (Jacobi preconditioner)
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < snb; k++) s1t_part += B.svec_part[(int64_t)k * (3 * d + 1) + 3 * d];
    V.st1[0] = s1t_part;
  }
  __syncthreads();
  // 3. gradient at the trial, Psi (without the constant term) and magnitudes
  const double sigma = st->sigma, tau = st->tau;
  const double tos = tau / sigma;
  double dx2 = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) {
    const double dk = V.xt[k] - V.xk[k];
    dx2 += dk * dk;
    const double sk = (k == 0) ? s_last[P_SU] : V.sv[k - 1];
    V.gt[k] = ((k == 0) ? 1.0 : 0.0) - sk + tos * dk;
  }
  dx2 = block_sum<256>(dx2, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < P_COUNT; k++) st->last[k] = s_last[k];
    st->tot_passes += 1;
    st->n64_total += (int64_t)s_last[P_N64];
  }
  const double psi_t = V.xt[0] + 0.5 * sigma * s_last[P_PI2] + 0.5 * tos * dx2;
  const double mag_t = fabs(V.xt[0]) + 0.5 * sigma * s_last[P_PI2] + 0.5 * tos * dx2;
  const double gmag_t = 1.0 + sigma * s_last[P_ZMAG] + tos * sqrt(dx2);

  if (st->eval_only) {
    if (threadIdx.x == 0) {
      st->psi = psi_t - s_last[P_UV2] / (2.0 * sigma);
      st->action = ACT_DONE;
      st->status = 1;
    }
    return;
  }

  // 4. decisions
  if (threadIdx.x == 0) {
    int nxt;  // 0: stop test at the accepted point, 1: backtrack, 2: outer (forced)
    if (st->phase == 1) {
      const double allow = 64.0 * DBL_EPSILON * fmax(st->psi_mag, mag_t);
      const bool ok = psi_t <= st->psi + st->mu * st->eta * st->gdx + allow;
      if (ok || st->bt >= st->max_backtrack) {
        st->psi = psi_t; st->psi_mag = mag_t; st->gmag = gmag_t;
        st->ssn_j += 1;
        st->tot_ssn += 1;
        if (!ok) nxt = 2;
        else if (st->ssn_j >= st->max_ssn) nxt = 2;
        else nxt = 0;
        st->phase = 2;   // accepted: copy xt -> x below
      } else {
        st->bt += 1;
        st->tot_bt += 1;
        st->eta *= 0.5;
        nxt = 1;
      }
    } else {
      st->psi = psi_t; st->psi_mag = mag_t; st->gmag = gmag_t;
      st->ssn_j = 0;
      st->phase = 2;
      nxt = 0;
    }
    s_next = nxt;
  }
  __syncthreads();
  const int nxt = s_next;
  if (nxt == 1) {
    const double eta = st->eta;
    for (int k = threadIdx.x; k < n1; k += 256) V.xt[k] = V.x[k] + eta * V.dx[k];
    __syncthreads();
    set_trial(st, V, d, sh);
    if (threadIdx.x == 0) { st->phase = 1; st->action = ACT_TRIAL; }
    return;
  }
  // accepted point: x <- xt, g <- gt
  for (int k = threadIdx.x; k < n1; k += 256) {
    V.x[k] = V.xt[k];
    V.g[k] = V.gt[k];
  }
  __syncthreads();
  if (nxt == 2) {
    do_outer(st, V, d, sh);
    return;
  }
  // relative-type stopping condition (Algorithm 1) on the tentative quantities
  double la = 0.0, g2 = 0.0, dk2 = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) {
    la += (V.ab[k] - V.x[k]) * V.g[k];
    g2 += V.g[k] * V.g[k];
    const double t = V.x[k] - V.xk[k];
    dk2 += t * t;
  }
  la = block_sum<256>(la, sh);
  g2 = block_sum<256>(g2, sh);
  dk2 = block_sum<256>(dk2, sh);
  const double lhs = 2.0 * sigma * fabs(la) + sigma * sigma * g2;
  const double rhs = st->rho * (s_last[P_DUV2] + tau * dk2);
  const bool stop = (lhs <= rhs) || (sqrt(g2) <= 8.0 * DBL_EPSILON * st->gmag);
  if (stop) {
    do_outer(st, V, d, sh);
    return;
  }
  if (threadIdx.x == 0) {
    st->action = ACT_NEWTON;
    st->bt = 0;
  }
}

cudaError_t launch_tick_control(Buffers& B, int64_t m, int d, cudaStream_t s) {
  const int nb = (int)((m + kPassThreads - 1) / kPassThreads);
  k_control<<<1, 256, 0, s>>>(B, d, nb);
  B.launches += 1;
  return cudaGetLastError();
}

// ===========================================================================
// Dense Newton system (d + 1 <= kMaxDenseN):
//   H = tau/sigma I + sigma (n_I I + sum_M P_k),
//   sum_M P_k = 1/2 [[n_M, sum w^T], [sum w, sum(1+t) I - sum t w w^T]].
// k_syrk: partial tiles of sum_M t_k w_k w_k^T over row groups.
constexpr int kSyrkGroups = 24;

__global__ void __launch_bounds__(256) k_syrk(Buffers B, int d, int force) {
  DevState* st = B.st;
  if (!force && (st->status != 0 || st->action != ACT_NEWTON)) return;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  const int tri = blockIdx.x, grp = blockIdx.y;
  if (tri >= ntri) return;
  // tile (ti >= tj) from the linear lower-triangle index
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= tri) ti++;
  const int tj = tri - ti * (ti + 1) / 2;
  const int nS = st->nS;
  const int rpg = (nS + kSyrkGroups - 1) / kSyrkGroups;
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

// Sum the group partials (in group order) into B.H's lower triangle block (rows/cols 1..d).
__global__ void k_syrk_reduce(Buffers B, int d, int force) {
  DevState* st = B.st;
  if (!force && (st->status != 0 || st->action != ACT_NEWTON)) return;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  const int64_t tot = (int64_t)ntri * kSyrkTile * kSyrkTile;
  const int n1 = d + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int tri = (int)(e / (kSyrkTile * kSyrkTile));
    const int loc = (int)(e % (kSyrkTile * kSyrkTile));
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= tri) ti++;
    const int tj = tri - ti * (ti + 1) / 2;
    const int j = ti * kSyrkTile + loc / kSyrkTile, l = tj * kSyrkTile + loc % kSyrkTile;
    if (j >= d || l >= d || l > j) continue;
    double s = 0.0;
    for (int g = 0; g < kSyrkGroups; g++)
      s += B.hpart[((int64_t)g * ntri + tri) * (kSyrkTile * kSyrkTile) + loc];
    B.H[(int64_t)(1 + j) * n1 + (1 + l)] = s;
  }
}

// One block: assemble H (packed lower, smem), Cholesky, solve H dx = -g,
// then set the first line-search trial x + dx.
__global__ void __launch_bounds__(256) k_newton_chol(Buffers B, int d) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_NEWTON) return;
  extern __shared__ double Lp[];   // packed lower: row i at i(i+1)/2
  __shared__ double sh[32];
  __shared__ int s_fail;
  const DevVecs& V = B.vec;
  const int n = d + 1;
  const double sigma = st->sigma, tos = st->tau / sigma;
  const double nI = st->last[P_NI], nM = st->last[P_NM];
  const double s1t = V.st1[0];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < n; i += 8) {
    const int64_t ri = (int64_t)i * (i + 1) / 2;
    for (int l = lane; l <= i; l += 32) {
      double h;
      if (i == 0) h = tos + sigma * (nI + 0.5 * nM);
      else if (l == 0) h = sigma * 0.5 * V.sw[i - 1];
      else {
        const double sy = B.H[(int64_t)i * n + l];
        h = sigma * (-0.5 * sy);
        if (i == l) h += tos + sigma * (nI + 0.5 * s1t);
      }
      Lp[ri + l] = h;
    }
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
    st->gdx = gd;
    st->eta = 1.0;
    st->phase = 1;
    st->bt = 0;
    st->action = ACT_TRIAL;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

cudaError_t launch_newton_dense(Buffers& B, int d, cudaStream_t s) {
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  k_syrk<<<dim3(ntri, kSyrkGroups), 256, 0, s>>>(B, d, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_syrk_reduce<<<64, 256, 0, s>>>(B, d, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = d + 1;
  const size_t sh = sizeof(double) * (size_t)n * (n + 1) / 2;
  if (sh > 48 * 1024) {
    e = cudaFuncSetAttribute(k_newton_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  k_newton_chol<<<1, 256, sh, s>>>(B, d);
  B.launches += 3;
  return cudaGetLastError();
}

// ===========================================================================
// Matrix-free Newton system (Sec. 4.1): CG with the Jacobi preconditioner,
//   Hq = tau/sigma q + sigma (n_I q + sum_M P_k q),
//   P_k q = 1/2 (q0 + w.q1 ; q0 w + (1+t) q1 - t w (w.q1)).
// k_hvp_dot: wq_k = w_k . q1 (warp per row); k_hvp_acc: -1/2 sum_k t_k wq_k w_k
// and 1/2 sum_k wq_k; hvp_finish adds the terms in q0 sum w and sum(1+t) q1.
__global__ void __launch_bounds__(256) k_hvp_dot(Buffers B, int d, const double* __restrict__ q,
                                                  double* __restrict__ wq, int force) {
  DevState* st = B.st;
  if (!force && (st->status != 0 || st->action != ACT_NEWTON || st->cg_done)) return;
  const int nS = st->nS;
  const int lane = threadIdx.x & 31;
  for (int k = (blockIdx.x * 256 + threadIdx.x) >> 5; k < nS; k += (gridDim.x * 256) >> 5) {
    double t = 0.0;
    if (B.S_case[k] == CASE_M) {
      const double* w = B.W + (int64_t)k * d;
      for (int j = lane; j < d; j += 32) t = fma(w[j], q[1 + j], t);
      t = warp_sum(t);
    }
    if (lane == 0) wq[k] = t;
  }
}

__global__ void __launch_bounds__(256) k_hvp_acc(Buffers B, int d, const double* __restrict__ q,
                                                  const double* __restrict__ wq,
                                                  double* __restrict__ part, int force) {
  DevState* st = B.st;
  if (!force && (st->status != 0 || st->action != ACT_NEWTON || st->cg_done)) return;
  const int nS = st->nS;
  const int rpb = (nS + gridDim.x - 1) / gridDim.x;
  const int k0 = blockIdx.x * rpb, k1 = min(nS, k0 + rpb);
  double* out = part + (int64_t)blockIdx.x * (d + 1);
  double s0 = 0.0;
  for (int j0 = 0; j0 < d; j0 += 256) {
    const int j = j0 + threadIdx.x;
    double acc = 0.0;
    for (int k = k0; k < k1; k++) {
      if (B.S_case[k] != CASE_M) continue;
      const double coef = -0.5 * B.S_t[k] * wq[k];   // the q0 w part is 1/2 q0 sum w
      if (j < d) acc = fma(coef, B.W[(int64_t)k * d + j], acc);
      if (j0 == 0 && threadIdx.x == 0) s0 += 0.5 * wq[k];
    }
    if (j < d) out[1 + j] = acc;
  }
  if (threadIdx.x == 0) out[0] = s0;
}

// y = tau/sigma q + sigma (n_I q + 1/2 [n_M q0 + S0 ; q0 sum w + sum(1+t) q1] + acc)
__device__ void hvp_finish(DevState* st, const DevVecs& V, int d, const double* q,
                           const double* part, int nblk, double* y) {
  const int n1 = d + 1;
  const double sigma = st->sigma, tos = st->tau / sigma;
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

__global__ void __launch_bounds__(256) k_cg_setup(Buffers B, int d) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_NEWTON) return;
  __shared__ double sh[32];
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  const double sigma = st->sigma, tos = st->tau / sigma;
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
    st->cg_it = 0;
    st->cg_done = (bn == 0.0);
  }
}

// One CG iteration after the HVP partials of p are in place.
__global__ void __launch_bounds__(256) k_cg_update(Buffers B, int d, int nblk) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_NEWTON || st->cg_done) return;
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

__global__ void __launch_bounds__(256) k_cg_finish(Buffers B, int d) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_NEWTON) return;
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

cudaError_t launch_cg_setup(Buffers& B, int d, cudaStream_t s) {
  k_cg_setup<<<1, 256, 0, s>>>(B, d);
  B.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_cg_iter(Buffers& B, int d, cudaStream_t s) {
  k_hvp_dot<<<kHvpBlocks * 4, 256, 0, s>>>(B, d, B.vec.cg_p, B.wq, 0);
  k_hvp_acc<<<kHvpBlocks, 256, 0, s>>>(B, d, B.vec.cg_p, B.wq, B.hpart, 0);
  k_cg_update<<<1, 256, 0, s>>>(B, d, kHvpBlocks);
  B.launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_cg_finish(Buffers& B, int d, cudaStream_t s) {
  k_cg_finish<<<1, 256, 0, s>>>(B, d);
  B.launches += 1;
  return cudaGetLastError();
}

// ===========================================================================
// Multiplier update (Algorithm 1): (u, v)^{k+1} = sigma_k Pi(z_k) on the
// support of the accepted point, written to the other buffer; then the
// ball->slot map and the buffer parity.
__global__ void __launch_bounds__(256) k_mult_rows(const double* __restrict__ C, Buffers B,
                                                   int d) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_OUTER) return;
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
  for (int k = (blockIdx.x * 256 + threadIdx.x) >> 5; k < nS; k += (gridDim.x * 256) >> 5) {
    const int idx = B.S_idx[k];
    const int sl0 = B.slot[idx];
    const int sl = ((unsigned)sl0 < (unsigned)nsup && sidx[sl0] == idx) ? sl0 : -1;
    const double a = B.S_a[k], n = B.S_n[k];
    const double f = (B.S_case[k] == CASE_I) ? 1.0 : 0.5 * (a + n) / n;
    for (int j = lane; j < d; j += 32) {
      double b = (C[(int64_t)idx * d + j] - ct[j]) * inv_s;
      if (sl >= 0) b = fma(sv[(int64_t)sl * d + j], inv_sigma, b);
      nv[(int64_t)k * d + j] = sigma * f * b;
    }
    if (lane == 0) {
      B.sup_idx[nxt][k] = idx;
      B.sup_u[nxt][k] = B.S_u[k];
    }
  }
}

__global__ void k_mult_slots(Buffers B) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_OUTER) return;
  const int nS = st->nS;
  const int nxt = st->sup_cur ^ 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nS; k += gridDim.x * blockDim.x)
    B.slot[B.sup_idx[nxt][k]] = k;
}

__global__ void k_mult_flip(Buffers B) {
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_OUTER) return;
  st->sup_cur ^= 1;
  st->nsup = st->nS;
  st->action = ACT_NONE;
}

cudaError_t launch_mult_update(const double* C, Buffers& B, int64_t m, int d, cudaStream_t s) {
  (void)m;
  k_mult_rows<<<304, 256, 0, s>>>(C, B, d);
  k_mult_slots<<<152, 256, 0, s>>>(B);
  k_mult_flip<<<1, 1, 0, s>>>(B);
  B.launches += 3;
  return cudaGetLastError();
}

// ===========================================================================
// Solve initialisation (state fields set by the host beforehand): x = xt =
// xk = ab = (r0, c0)/s, trial shadow.
__global__ void k_state_init(Buffers B, int d) {
  __shared__ double sh[32];
  DevState* st = B.st;
  const DevVecs& V = B.vec;
  const double inv_s = st->inv_s;
  for (int k = threadIdx.x; k <= d; k += blockDim.x) {
    const double v = (k == 0) ? st->rt_abs * inv_s : V.o[k - 1] * inv_s;
    V.x[k] = v; V.xt[k] = v; V.xk[k] = v; V.ab[k] = v;
    V.g[k] = 0.0; V.dx[k] = 0.0;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

cudaError_t launch_state_init(Buffers& B, int d, cudaStream_t s) {
  k_state_init<<<1, 256, 0, s>>>(B, d);
  B.launches += 1;
  return cudaGetLastError();
}

// ===========================================================================
// Evaluation entry: support from dense (U, V) rows, outputs back to dense.
__global__ void k_dense_flags(const double* __restrict__ U, const double* __restrict__ V,
                              int64_t m, int d, int* __restrict__ cnt,
                              int64_t* __restrict__ lists) {
  __shared__ int s_wc[8];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  bool nz = false;
  if (i < m) {
    nz = U[i] != 0.0;
    for (int j = 0; j < d && !nz; j++) nz = V[i * (int64_t)d + j] != 0.0;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned msk = __ballot_sync(FULLMASK, nz);
  if (lane == 0) s_wc[w] = __popc(msk);
  __syncthreads();
  int off = 0, tot = 0;
  for (int k = 0; k < 8; k++) { off += (k < w) ? s_wc[k] : 0; tot += s_wc[k]; }
  if (nz) lists[(int64_t)blockIdx.x * 256 + off + __popc(msk & ((1u << lane) - 1u))] = i;
  if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

__global__ void k_dense_support(const double* __restrict__ U, const double* __restrict__ V,
                                const int64_t* __restrict__ list, const int64_t* __restrict__ n,
                                int d, Buffers B) {
  const int64_t ns = *n;
  const int lane = threadIdx.x & 31;
  for (int64_t k = ((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5; k < ns;
       k += ((int64_t)gridDim.x * 256) >> 5) {
    const int64_t i = list[k];
    for (int j = lane; j < d; j += 32) B.sup_v[0][k * d + j] = V[i * (int64_t)d + j];
    if (lane == 0) {
      B.sup_idx[0][k] = (int)i;
      B.sup_u[0][k] = U[i];
      B.slot[i] = (int)k;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.st->sup_cur = 0;
    B.st->nsup = (int)ns;
  }
}

cudaError_t launch_support_from_dense(const double* U, const double* V, Buffers& B, int64_t m,
                                      int d, cudaStream_t s) {
  const int nb = (int)((m + 255) / 256);
  k_dense_flags<<<nb, 256, 0, s>>>(U, V, m, d, B.feas_cnt, B.list_tmp);
  k_gather_lists<<<(nb + 255) / 256, 256, 0, s>>>(B.feas_cnt, B.list_tmp, nb, 256, B.viol, m);
  k_count_sum<<<1, 256, 0, s>>>(B.feas_cnt, nb, B.count64);
  k_dense_support<<<304, 256, 0, s>>>(U, V, B.viol, B.count64, d, B);
  return cudaGetLastError();
}

// Evaluation entry: state for one pass at x with prox centre xbar, s = 1.
__global__ void k_eval_prepare(Buffers B, const double* __restrict__ x,
                               const double* __restrict__ xbar, int d) {
  __shared__ double sh[32];
  DevState* st = B.st;
  const DevVecs& V = B.vec;
  for (int k = threadIdx.x; k <= d; k += blockDim.x) {
    V.x[k] = x[k]; V.xt[k] = x[k]; V.xk[k] = xbar[k]; V.ab[k] = x[k];
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

cudaError_t launch_eval_prepare(Buffers& B, const double* x, const double* xbar, int d,
                                cudaStream_t s) {
  k_eval_prepare<<<1, 256, 0, s>>>(B, x, xbar, d);
  return cudaGetLastError();
}

// Dense outputs of the evaluation: U+ (m), V+ (m x d) from the support list.
__global__ void k_eval_scatter(Buffers B, int d, double* __restrict__ Up,
                               double* __restrict__ Vp) {
  DevState* st = B.st;
  const int nS = st->nS;
  const double sigma = st->sigma;
  const int lane = threadIdx.x & 31;
  for (int k = (blockIdx.x * 256 + threadIdx.x) >> 5; k < nS; k += (gridDim.x * 256) >> 5) {
    const int64_t i = B.S_idx[k];
    const bool isI = B.S_case[k] == CASE_I;
    const double coef = isI ? sigma : B.S_u[k];   // v+ = sigma b (I) or u+ w (M)
    for (int j = lane; j < d; j += 32) Vp[i * d + j] = coef * B.W[(int64_t)k * d + j];
    if (lane == 0) Up[i] = B.S_u[k];
  }
}

// H = tau/sigma I + sigma (n_I I + sum_M P_k), dense n1 x n1, both triangles.
__global__ void k_eval_hess(Buffers B, int d, double* __restrict__ Hout) {
  DevState* st = B.st;
  const DevVecs& V = B.vec;
  const int n = d + 1;
  const double sigma = st->sigma, tos = st->tau / sigma;
  const double nI = st->last[P_NI], nM = st->last[P_NM], s1t = V.st1[0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), l = (int)(e % n);
    if (l > i) { int t = i; i = l; l = t; }
    double h;
    if (i == 0) h = tos + sigma * (nI + 0.5 * nM);
    else if (l == 0) h = sigma * 0.5 * V.sw[i - 1];
    else {
      h = -0.5 * sigma * B.H[(int64_t)i * n + l];
      if (i == l) h += tos + sigma * (nI + 0.5 * s1t);
    }
    Hout[e] = h;
  }
}

__global__ void k_eval_hq(Buffers B, int d, const double* __restrict__ q, double* __restrict__ y) {
  hvp_finish(B.st, B.vec, d, q, B.hpart, kHvpBlocks, y);
}

cudaError_t launch_eval_outputs(const double* C, Buffers& B, int64_t m, int d, const double* q,
                                double* Uplus, double* Vplus, double* Hq, double* H,
                                cudaStream_t s) {
  (void)C;
  if (Uplus) cudaMemsetAsync(Uplus, 0, sizeof(double) * (size_t)m, s);
  if (Vplus) cudaMemsetAsync(Vplus, 0, sizeof(double) * (size_t)m * d, s);
  if (Uplus && Vplus) k_eval_scatter<<<304, 256, 0, s>>>(B, d, Uplus, Vplus);
  if (Hq) {
    k_hvp_dot<<<kHvpBlocks * 4, 256, 0, s>>>(B, d, q, B.wq, 1);
    k_hvp_acc<<<kHvpBlocks, 256, 0, s>>>(B, d, q, B.wq, B.hpart, 1);
    k_eval_hq<<<1, 256, 0, s>>>(B, d, q, Hq);
  }
  if (H) {
    const int nt = (d + kSyrkTile - 1) / kSyrkTile;
    const int ntri = nt * (nt + 1) / 2;
    k_syrk<<<dim3(ntri, kSyrkGroups), 256, 0, s>>>(B, d, 1);
    k_syrk_reduce<<<64, 256, 0, s>>>(B, d, 1);
    const int64_t n2 = (int64_t)(d + 1) * (d + 1);
    k_eval_hess<<<(int)imin64(1024, (n2 + 255) / 256), 256, 0, s>>>(B, d, H);
  }
  return cudaGetLastError();
}

// Final centre and ALM radius (unscaled) from the accepted point.
__global__ void k_final_point(Buffers B, int d, double* __restrict__ c_out,
                              double* __restrict__ r_alm) {
  DevState* st = B.st;
  const double s = st->s;
  for (int j = threadIdx.x; j < d; j += blockDim.x) c_out[j] = B.vec.x[1 + j] * s;
  if (threadIdx.x == 0) *r_alm = B.vec.x[0] * s;
}

cudaError_t launch_final_point(Buffers& B, int d, double* c_out, double* r_alm, cudaStream_t s) {
  k_final_point<<<1, 256, 0, s>>>(B, d, c_out, r_alm);
  B.launches += 1;
  return cudaGetLastError();
}

}  // namespace meb
