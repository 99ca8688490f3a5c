// Device helpers shared by the libmeb translation units: deterministic warp
// and block reductions, the distance to the second-order cone, and the FP32
// shadow conversion with its error bound.
#pragma once
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "meb_internal.cuh"

namespace meb {

#define MEB_FULLMASK 0xffffffffu

__host__ __device__ static inline int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// Programmatic dependent launch: wait for the preceding grid (a no-op when the
// kernel was launched without the attribute), then let the next grid be
// scheduled (it waits for this grid in turn).
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(MEB_FULLMASK, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(MEB_FULLMASK, v, o));
  return v;
}

// Transposed warp sum of 8 slots: after log2(32) exchange levels lane L holds
// the full warp sum of slot (L >> 2) & 7, in a fixed tree order.  9 FP64 adds
// per lane instead of 8 x 5 for eight separate warp_sum calls.
__device__ __forceinline__ double warp_sum8_transposed(const double (&v)[8]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  double w4[4], w2[2];
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const double send = b4 ? v[p] : v[p + 4];
    const double keep = b4 ? v[p + 4] : v[p];
    w4[p] = keep + __shfl_xor_sync(MEB_FULLMASK, send, 16);
  }
#pragma unroll
  for (int p = 0; p < 2; p++) {
    const double send = b3 ? w4[p] : w4[p + 2];
    const double keep = b3 ? w4[p + 2] : w4[p];
    w2[p] = keep + __shfl_xor_sync(MEB_FULLMASK, send, 8);
  }
  const double send = b2 ? w2[0] : w2[1];
  double w1 = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(MEB_FULLMASK, send, 4);
  w1 += __shfl_xor_sync(MEB_FULLMASK, w1, 2);
  w1 += __shfl_xor_sync(MEB_FULLMASK, w1, 1);
  return w1;
}

// Warp max of non-negative doubles on their bit patterns (IEEE order equals
// integer order for x >= 0): integer instructions only.
__device__ __forceinline__ double warp_max_nonneg(double v) {
  long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long t = __shfl_xor_sync(MEB_FULLMASK, b, o);
    b = t > b ? t : b;
  }
  return __longlong_as_double(b);
}

// Block-wide sum in a fixed tree order; every thread gets the result.
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

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(MEB_FULLMASK, v, o);
  return v;
}

// Element j of ball i of the FP32 shadow (layout [ceil(d/4)][m_pad] float4).
__device__ __forceinline__ float x32_at(const float4* X32, int64_t m_pad, int64_t i, int j) {
  return reinterpret_cast<const float*>(X32)[(((int64_t)(j >> 2)) * m_pad + i) * 4 + (j & 3)];
}

// Distance to Q of a point (a, b) with ||b|| = n (closed form of ||z - Pi(z)||).
__device__ __forceinline__ double soc_dist_an(double a, double n) {
  if (n <= a) return 0.0;
  if (n <= -a) return sqrt(a * a + n * n);
  return (n - a) * 0.70710678118654752440;
}

// FP64 -> FP32 by truncation of the mantissa, with integer operations only
// (the conversion instruction runs on the FP64 pipe).  |result| <= |x| and
// |x - result| < 2^-23 |x| for normal results; |x| < 2^-126 gives 0 (absolute
// error < 2^-126); |x| >= 2^128 gives +-inf (never certified).
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ff) - 1023 + 127;
  unsigned r;
  if (e <= 0) r = sign;                         // zero, subnormal, underflow
  else if (e >= 255) r = sign | 0x7f800000u;    // overflow, inf, NaN -> inf
  else r = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(r);
}

// The FP32 shadow.  The origin o is the first centre truncated to FP32 (so
// it is exact in both precisions); each element is
//   x32 = fl32(trunc32(c_ij) - o_j)
// with FP32 operations only (the FP64 pipe is not used).  With x = c_i - o,
//   |x - x32| <= 2^-24 |x32| + 2^-23 |c_ij| + 2^-126,
// so ||x_i - x32_i|| <= kShadowU ||x32_i|| + E_i, where E_i >= 2^-23 ||c_i|| +
// sqrt(d) 2^-126 is stored per ball.  The query shadow y32 = trunc32(y - o)
// is formed in FP64 (one rounding, one truncation): |y - y32| <= kShadowU |y32|.
constexpr float kU32 = 5.9604645e-08f;     // 2^-24
constexpr float kShadowU = 2.02f * 2.0f * kU32;

// E_i from cn2 = fmaf sum of trunc32(c_ij)^2 over the d elements of a row:
// ||c_i|| <= ||trunc32(c_i)|| (1 + 2^-23) + sqrt(d) 2^-126 and the sum and
// square root add at most (d + 4) 2^-24 relative (d <= 16384).
__device__ __forceinline__ float shadow_abs_err(float cn2, int d) {
  return 1.1920929e-7f * sqrtf(cn2) * (1.0f + (float)(d + 12) * kU32) + 4e-36f;
}

// Certified bounds on D = ||x - y|| from the FP32 shadows x32, y32:
//   S = sum (x32 - y32)^2, N = sum x32^2 (fmaf sums over k4 elements, k4 = 4 d4),
//   yn >= ||y32||, E = the ball's absolute shadow error.  Each of the k4
//   difference/square/sum steps is round-to-nearest.
__device__ __forceinline__ float dist_ub(float S, float N, float yn, float E, int k4) {
  return (sqrtf(S) + kShadowU * (sqrtf(N) + yn) + E) * (1.0f + (float)(k4 + 16) * kU32) + 1e-30f;
}
__device__ __forceinline__ float dist_lb(float S, float N, float yn, float E, int k4) {
  const float v = (sqrtf(S) * (1.0f - (float)(k4 + 16) * kU32)) -
                  (kShadowU * (sqrtf(N) + yn) + E) * (1.0f + (float)(k4 + 16) * kU32) - 1e-30f;
  return v > 0.0f ? v : 0.0f;
}

// Two block-wide sums at once, in a fixed tree order: a transposed first
// exchange (lanes 0..15 carry a, lanes 16..31 carry b), then one warp sums the
// warps' results.  Every thread gets both.
__device__ __forceinline__ double2 block_sum2(double a, double b) {
  __shared__ double s_b2[34];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool hi = lane & 16;
  double v = (hi ? b : a) + __shfl_xor_sync(MEB_FULLMASK, hi ? a : b, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(MEB_FULLMASK, v, o);
  __syncthreads();
  if (lane == 0) s_b2[w] = v;
  if (lane == 16) s_b2[16 + w] = v;
  __syncthreads();
  if (w == 0) {
    const int k = lane & 15;
    double t = (k < nw) ? s_b2[(lane & 16) + k] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(MEB_FULLMASK, t, o);
    if (lane == 0) s_b2[32] = t;
    if (lane == 16) s_b2[33] = t;
  }
  __syncthreads();
  const double2 r = make_double2(s_b2[32], s_b2[33]);
  __syncthreads();
  return r;
}

// Trial point for the next pass: ct = s * xt[1:] (exact), rt = s * xt[0],
// the query shadow y32 = trunc32(ct - o) with yn >= ||y32||, rq32 = fl32(rt),
// and dx2_t = ||xt - xk||^2 (the proximal term of Psi at the trial).
__device__ __forceinline__ void set_trial(DevState* st, const DevVecs& V, int d, double* sh) {
  const double s = st->s;
  const int d4 = (d + 3) / 4;
  double q = 0.0, dx2 = 0.0;
  if (threadIdx.x == 0) {
    const double dk = V.xt[0] - V.xk[0];
    dx2 = dk * dk;
  }
  for (int j = threadIdx.x; j < 4 * d4; j += blockDim.x) {
    float y = 0.0f;
    if (j < d) {
      const double xt = V.xt[1 + j];
      const double c = xt * s;
      V.ct[j] = c;
      y = f64_to_f32_trunc(c - V.o[j]);
      const double dk = xt - V.xk[1 + j];
      dx2 += dk * dk;
    }
    V.y32[j] = y;
    q += (double)y * (double)y;
  }
  const double2 r = block_sum2(q, dx2);
  if (threadIdx.x == 0) {
    st->rt_abs = V.xt[0] * s;
    st->rq32 = __double2float_rn(V.xt[0] * s);
    st->yn32 = __double2float_ru(sqrt(r.x) * (1.0 + 1e-12));
    st->dx2_t = r.y;
  }
  __syncthreads();
}

// FP16 shadow (scaled by 1/s): x16 = fl16(x32 / s) with x32 the FP32 shadow.
// Per element |x/s - x16| <= kHalfU |x16| + kHalfAbs + abs_ij / s (normal and
// subnormal halves), so ||x/s - x16_i|| <= eps_i with
//   eps_i = kHalfU ||x16_i|| + sqrt(k) kHalfAbs + E_i / s,
// stored per ball (k = 8 ceil(d/8) elements, padding included).
constexpr float kHalfU = 4.8828125e-4f + 1.001f * kShadowU;   // 2^-11 + shadow error
constexpr float kHalfAbs = 2.99e-8f;                            // 2^-25 (1 + shadow error)

// eps_i from N16 = fmaf sum of the k squared halves, E_i and 1/s
__device__ __forceinline__ float half_err(float N16, float E, float inv_s, int k) {
  return (kHalfU * sqrtf(N16) + sqrtf((float)k) * kHalfAbs + E * inv_s) *
             (1.0f + (float)(k + 16) * kU32) + 1e-30f;
}

__device__ __forceinline__ float dist_ub16(float S, float eps, float yn, int k) {
  return (sqrtf(S) + eps + kShadowU * yn) * (1.0f + (float)(k + 16) * kU32) + 1e-30f;
}
__device__ __forceinline__ float dist_lb16(float S, float eps, float yn, int k) {
  const float v = sqrtf(S) * (1.0f - (float)(k + 16) * kU32) -
                  (eps + kShadowU * yn) * (1.0f + (float)(k + 16) * kU32) - 1e-30f;
  return v > 0.0f ? v : 0.0f;
}

}  // namespace meb
