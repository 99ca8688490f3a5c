// Allocation-free variant of the feasibility check (meb_feas_check_noalloc).
//
// Who this is for: callers that cannot call cudaMalloc -- engines that hand
// every byte of device memory to their own pool or to another framework's
// caching allocator (a cudaMalloc behind their back fragments that pool or
// fails against its reservation), and real-time loops that forbid allocation
// once they run.  meb_feas_check needs a context, whose scratch buffers are
// allocated with cudaMalloc; this entry point needs no context and allocates
// nothing.  Its scratch lives in a file-scope device array of fixed size
// (kScratchBytes below, about 37 KB), which every GPU that loads the library
// holds until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture on the device.
//
// It computes exactly what meb_feas_check computes, in FP64 straight from the
// rows (no FP32 shadow, which would need m-sized scratch):
//   delta_max = max_i (r_i + ||c - c_i|| - r), argmax = lowest maximising index,
//   the ascending list { i : r_i + ||c - c_i|| - r > eps } (first viol_cap),
//   n_viol = its true size.
// Three kernels: per-block maxima and counts over fixed contiguous ranges,
// one block for the global maximum and the block offsets, then a second sweep
// that writes the indices in ascending order (256-ball tiles, ordered by a
// block-wide prefix of the warps' ballots).  A negative or non-finite radius,
// a non-finite row or query centre (any value that is not finite) makes the
// call return MEB_EINVAL, as meb_feas_check does.  Every scratch slot is written
// before it is read in each call, so nothing needs clearing; calls that
// overlap on the GPU (two streams, or two host threads) share the array and
// race.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <climits>
#include <cstddef>
#include <mutex>
#include <stdint.h>

#include "../../include/meb.h"

namespace {

constexpr int kNT = 256;                 // threads per block
constexpr int kBlocks = 1024;            // fixed grid: contiguous ball ranges
constexpr int kMaxD = 4096;              // c is staged in shared memory
constexpr int kMaxDevices = 64;

struct Scratch {
  double bmax[kBlocks];
  long long barg[kBlocks];
  long long bcnt[kBlocks];
  long long boff[kBlocks];
  int bbad[kBlocks];
  double gmax;
  long long garg;
  long long gcnt;
  int gbad;
};
constexpr size_t kScratchBytes = sizeof(Scratch);   // about 37 KB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device ordinal (host code cannot use the
// symbol itself: on the host its name is only a stand-in, not a device
// address).
static void* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// value of ball i (FP64, the definition); warp-cooperative
__device__ __forceinline__ double ball_val(const double* __restrict__ C,
                                           const double* __restrict__ R, const double* s_c,
                                           int64_t i, int d, double r, int lane) {
  const double* row = C + i * (int64_t)d;
  double acc = 0.0;
  for (int j = lane; j < d; j += 32) {
    const double t = s_c[j] - row[j];
    acc = fma(t, t, acc);
  }
  acc = warp_sum(acc);
  return (R[i] + sqrt(acc)) - r;
}

__global__ void __launch_bounds__(kNT) k_nf_count(const double* __restrict__ C,
                                                   const double* __restrict__ R, int64_t m, int d,
                                                   const double* __restrict__ c, double r,
                                                   double eps, Scratch* S) {
  extern __shared__ double s_c[];
  __shared__ double s_v[kNT / 32];
  __shared__ long long s_i[kNT / 32], s_n[kNT / 32];
  __shared__ int s_b[kNT / 32];
  for (int j = threadIdx.x; j < d; j += kNT) s_c[j] = c[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t chunk = (m + kBlocks - 1) / kBlocks;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = (i0 + chunk < m) ? i0 + chunk : m;
  double best = -INFINITY;
  long long bi = LLONG_MAX, cnt = 0;
  int bad = 0;
  for (int64_t i = i0 + w; i < i1; i += kNT / 32) {   // balls in order per warp
    const double v = ball_val(C, R, s_c, i, d, r, lane);
    const double ri = R[i];
    bad |= !isfinite(v) || !(ri >= 0.0) || !isfinite(ri);
    if (v > best) { best = v; bi = i; }
    cnt += (v > eps);
  }
  if (lane == 0) { s_v[w] = best; s_i[w] = bi; s_n[w] = cnt; s_b[w] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -INFINITY;
    long long ix = LLONG_MAX, n = 0;
    int bb = 0;
    for (int k = 0; k < kNT / 32; k++) {
      if (s_v[k] > b || (s_v[k] == b && s_i[k] < ix)) { b = s_v[k]; ix = s_i[k]; }
      n += s_n[k];
      bb |= s_b[k];
    }
    S->bmax[blockIdx.x] = b;
    S->barg[blockIdx.x] = ix;
    S->bcnt[blockIdx.x] = n;
    S->bbad[blockIdx.x] = bb;
  }
}

__global__ void k_nf_reduce(Scratch* S) {
  if (threadIdx.x != 0) return;
  double b = -INFINITY;
  long long ix = LLONG_MAX, off = 0;
  int bad = 0;
  for (int k = 0; k < kBlocks; k++) {
    if (S->bmax[k] > b || (S->bmax[k] == b && S->barg[k] < ix)) { b = S->bmax[k]; ix = S->barg[k]; }
    S->boff[k] = off;
    off += S->bcnt[k];
    bad |= S->bbad[k];
  }
  S->gmax = b;
  S->garg = ix;
  S->gcnt = off;
  S->gbad = bad;
}

__global__ void __launch_bounds__(kNT) k_nf_list(const double* __restrict__ C,
                                                  const double* __restrict__ R, int64_t m, int d,
                                                  const double* __restrict__ c, double r,
                                                  double eps, const Scratch* S,
                                                  int64_t* __restrict__ out, int64_t cap) {
  extern __shared__ double s_c[];
  __shared__ int s_wc[kNT / 32];
  for (int j = threadIdx.x; j < d; j += kNT) s_c[j] = c[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t chunk = (m + kBlocks - 1) / kBlocks;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = (i0 + chunk < m) ? i0 + chunk : m;
  long long pos = S->boff[blockIdx.x];
  if (S->bcnt[blockIdx.x] == 0 || pos >= cap) return;   // the same for the whole block
  // tiles of 256 balls in order: warp w evaluates balls 32w .. 32w+31 of the
  // tile (lane q keeps ball q's flag), then the block writes the members at
  // their ascending positions (the same values as k_nf_count: same code)
  for (int64_t t0 = i0; t0 < i1 && pos < cap; t0 += kNT) {
    const int nt = (int)((i1 - t0) < kNT ? (i1 - t0) : kNT);
    bool mine = false;
    for (int q = 0; q < 32; q++) {
      const int loc = 32 * w + q;
      if (loc >= nt) break;   // uniform within the warp
      const double v = ball_val(C, R, s_c, t0 + loc, d, r, lane);
      if (lane == q) mine = v > eps;
    }
    const bool f = (32 * w + lane < nt) && mine;
    const unsigned msk = __ballot_sync(0xffffffffu, f);
    if (lane == 0) s_wc[w] = __popc(msk);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < kNT / 32; k++) {
      off += (k < w) ? s_wc[k] : 0;
      tot += s_wc[k];
    }
    if (f) {
      const long long p = pos + off + __popc(msk & ((1u << lane) - 1u));
      if (p < cap) out[p] = t0 + 32 * w + lane;
    }
    pos += tot;
    __syncthreads();
  }
}

// Once per device, with that device current: the device address of g_scratch.
static int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MEB_ECUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MEB_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MEB_OK;
}

// The kernels' dynamic shared-memory limits are process-wide: raise them
// (never lower them) under a lock, per device, without allocating.
static size_t g_smem_limit[kMaxDevices] = {};
static std::mutex g_smem_mu;

static int raise_smem_limits(size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MEB_ECUDA;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  if (bytes <= g_smem_limit[dev]) return MEB_OK;
  if (cudaFuncSetAttribute(k_nf_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_nf_list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
          cudaSuccess)
    return MEB_ECUDA;
  g_smem_limit[dev] = bytes;
  return MEB_OK;
}

}  // namespace

extern "C" int meb_feas_check_noalloc(const double* centers, const double* radii, int64_t m,
                                      int32_t d, const double* c, double r, double eps,
                                      void* cuda_stream, double* delta_max, int64_t* argmax,
                                      int64_t* viol_idx, int64_t viol_cap, int64_t* n_viol) {
  if (!centers || !radii || !c || (viol_cap > 0 && !viol_idx) || viol_cap < 0)
    return MEB_EINVAL;
  if (m < 1 || m > (int64_t)2147483647 || d < 1 || d > kMaxD) return MEB_EINVAL;
  if (!isfinite(r) || isnan(eps)) return MEB_EINVAL;
  void* sp = nullptr;
  int rc = scratch_for_current_device(&sp);
  if (rc) return rc;
  Scratch* S = static_cast<Scratch*>(sp);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t sh = sizeof(double) * (size_t)d;
  if (raise_smem_limits(sh) != MEB_OK) return MEB_ECUDA;
  k_nf_count<<<kBlocks, kNT, sh, s>>>(centers, radii, m, d, c, r, eps, S);
  k_nf_reduce<<<1, 32, 0, s>>>(S);
  if (viol_cap > 0) k_nf_list<<<kBlocks, kNT, sh, s>>>(centers, radii, m, d, c, r, eps, S, viol_idx, viol_cap);
  if (cudaGetLastError() != cudaSuccess) return MEB_ECUDA;
  double gmax = 0.0;
  long long garg = 0, gcnt = 0;
  int gbad = 0;
  const char* base = static_cast<const char*>(sp);
  if (cudaMemcpyAsync(&gmax, base + offsetof(Scratch, gmax), sizeof(double),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&garg, base + offsetof(Scratch, garg), sizeof(long long),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&gcnt, base + offsetof(Scratch, gcnt), sizeof(long long),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&gbad, base + offsetof(Scratch, gbad), sizeof(int),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MEB_ECUDA;
  if (gbad) return MEB_EINVAL;
  if (delta_max) *delta_max = gmax;
  if (argmax) *argmax = (int64_t)garg;
  if (n_viol) *n_viol = (int64_t)gcnt;
  return MEB_OK;
}
