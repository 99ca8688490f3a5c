// libmeb streaming kernels: the FP32 shadow of the centres, the full pass of
// Algorithm 2 (step 1 and the per-ball parts of step 2), the support-row
// reduction, and the certified feasibility pass of Sec. 4.2.
//
// Notation (Sec. 2, Sec. 4): for ball i with centre c_i and radius r_i, at
// x = (r, c) with multipliers (u_i, v_i),
//   z_i = (a_i, b_i) = (r_i - r, c_i - c)/s + (u_i, v_i)/sigma,
//   (u_i^+, v_i^+) = sigma * Pi_Q(z_i),
// with the cases of the closed-form projection I: ||b|| <= a (Pi = z),
// Z: ||b|| <= -a (Pi = 0), M: otherwise.  s is the power-of-two scale of the
// problem; multiplying differences by 1/s is exact.
//
// GB300 design: FP64 runs at about 2 lanes/clk/SM on this part, so full
// passes stream the FP32 shadow (ball-interleaved float4, 16*ceil(d/4) bytes
// per ball) and certify, with the rigorous bound of meb_common.cuh, that a
// ball with zero multipliers lies strictly inside the current ball (case Z:
// it contributes exactly nothing).  Every other ball is evaluated in FP64
// from its original row.  All reductions use fixed block-to-ball maps and
// fixed-order trees, so results are deterministic.
#include "meb_pass_dev.cuh"

namespace meb {

__global__ void __launch_bounds__(kShadowNT, 4) k_shadow(const double* __restrict__ C,
                                                      const double* __restrict__ R, int64_t m,
                                                      int d, int64_t m_pad,
                                                      float4* __restrict__ X32,
                                                      float* __restrict__ R32,
                                                      float* __restrict__ E32,
                                                      double* __restrict__ colpart,
                                                      int* __restrict__ bad, int64_t b0) {
  shadow_block((int)(b0 + blockIdx.x), C, R, m, d, m_pad, X32, R32, E32, colpart, bad);
}

__global__ void k_shadow_mean(const double* __restrict__ C, const double* __restrict__ colpart,
                              int nb, int d, int64_t m, double* __restrict__ o,
                              double* __restrict__ c0) {
  shadow_mean_block(blockIdx.x, C, colpart, nb, d, m, o, c0);
}

static_assert(kShadowBallsPerBlock == kShadowBalls, "shadow block size");

cudaError_t launch_shadow_blocks(const double* C, const double* R, int64_t m, int d, Buffers& B,
                                 int64_t b0, int64_t b1, int* bad, cudaStream_t s) {
  const int64_t m_pad = ((m + 255) / 256) * 256;
  const int64_t nb = (m + kShadowBalls - 1) / kShadowBalls;
  if (b0 < 0 || b1 > nb || b0 >= b1) return cudaErrorInvalidValue;
  k_shadow<<<(unsigned)(b1 - b0), kShadowNT, 0, s>>>(C, R, m, d, m_pad, B.X32, B.R32, B.E32,
                                                     B.colsum_part, bad, b0);
  B.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_shadow_mean(const double* C, int64_t m, int d, Buffers& B, double* o,
                               double* c0, cudaStream_t s) {
  const int nb = (int)((m + kShadowBalls - 1) / kShadowBalls);
  k_shadow_mean<<<d, 256, 0, s>>>(C, B.colsum_part, nb, d, m, o, c0);
  B.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_shadow(const double* C, const double* R, int64_t m, int d, Buffers& B,
                          double* o, double* c0, int* bad, cudaStream_t s) {
  const int64_t nb = (m + kShadowBalls - 1) / kShadowBalls;
  cudaError_t e = launch_shadow_blocks(C, R, m, d, B, 0, nb, bad, s);
  if (e != cudaSuccess) return e;
  return launch_shadow_mean(C, m, d, B, o, c0, s);
}

__global__ void k_shadow16(const float4* __restrict__ X32, const float* __restrict__ E32,
                           int64_t m_pad, int d4, float inv_s, uint4* __restrict__ X16,
                           float* __restrict__ EPS) {
  shadow16_block(blockIdx.x, X32, E32, m_pad, d4, inv_s, X16, EPS);
}

cudaError_t launch_shadow16(Buffers& B, int64_t m, int d, double inv_s, cudaStream_t s) {
  const int64_t m_pad = ((m + 255) / 256) * 256;
  k_shadow16<<<(unsigned)(m_pad / 256), 256, 0, s>>>(B.X32, B.E32, m_pad, (d + 3) / 4,
                                                     (float)inv_s, B.X16, B.EPS16);
  B.launches += 1;
  return cudaGetLastError();
}

template <bool HALF>
__global__ void __launch_bounds__(kPassThreads, 4) k_screen(PassArgs A, Buffers B) {
  pdl_wait_and_release();
  DevState* st = A.st;
  if (!screen_gate(st)) return;
  if (A.log_slot >= 0 && blockIdx.x == 0 && threadIdx.x == 0) st->screen_log[A.log_slot] = 1;
  screen_block<HALF>(A, blockIdx.x);
  if (last_block_ticket(&st->ctr_screen)) early_body(B, A.d, gridDim.x);
}

template <bool LOWP>
__global__ void __launch_bounds__(kPassThreads) k_rows64(PassArgs A, Buffers B) {
  pdl_wait_and_release();
  DevState* st = A.st;
  if (!rows_gate(st)) return;
  rows_block<LOWP>(A, blockIdx.x);
  if (last_block_ticket(&st->ctr_rows)) control_a_body(B, A.d, gridDim.x);
}

static int bulk_stages(int d) {
  const int nrows = ((d + 3) / 4 + 1) / 2;
  int st = (kBulkSmemBudget - 32 * nrows - 64) / bulk_stage_bytes(nrows);
  return st > kBulkMaxStages ? kBulkMaxStages : st;
}

static size_t bulk_smem(int d, int nst) {
  const int nrows = ((d + 3) / 4 + 1) / 2;
  return (size_t)nst * bulk_stage_bytes(nrows) + 32 * (size_t)nrows + 8 * kBulkMaxStages;
}

__global__ void __launch_bounds__(kPassThreads, 1) k_screen_bulk(PassArgs A, Buffers B, int nst) {
  pdl_wait_and_release();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  DevState* st = A.st;
  if (st->status != 0 || st->action == ACT_DONE || st->reuse_lists) return;
  if (A.log_slot >= 0 && blockIdx.x == 0 && threadIdx.x == 0) st->screen_log[A.log_slot] = 1;
  const int d4 = A.d4;
  const int nrows = (d4 + 1) / 2;
  const int sb = bulk_stage_bytes(nrows);
  unsigned char* stages = smem_raw;
  float4* s_y = reinterpret_cast<float4*>(smem_raw + (size_t)nst * sb);   // 2 nrows groups
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)nst * sb + 32 * nrows);
  __shared__ int s_wc[kPassWarps];
  __shared__ float s_v2[kPassWarps];
  const float sc = (float)st->sh_inv_s;
  const float4* y4 = reinterpret_cast<const float4*>(A.y32);
  for (int g = threadIdx.x; g < 2 * nrows; g += kPassThreads) {
    const float4 y = g < d4 ? y4[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    s_y[g] = make_float4(-y.x * sc, -y.y * sc, -y.z * sc, -y.w * sc);   // -y, scaled
  }
  const int cur = st->sup_cur;
  const int nsup = st->nsup;
  const int* sidx = cur ? A.sup_idx1 : A.sup_idx0;
  const float rq = st->rq32 * sc, yn = st->yn32 * sc;
  const float unsc = (float)st->sh_s;
  float v2sum = 0.0f;
  const int k8 = 8 * nrows;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t ntiles = (A.m + kPassThreads - 1) / kPassThreads;
  const int64_t t0 = (int64_t)blockIdx.x * A.tiles_per_block;
  const int64_t t1 = imin64(ntiles, t0 + A.tiles_per_block);
  const int ntl = t1 > t0 ? (int)(t1 - t0) : 0;
  const int64_t base = t0 * kPassThreads;
  if (tid == 0) {
    for (int q = 0; q < nst; q++) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // warp 0: copies of local tile k into stage k % nst; lane 0 announces the
  // bytes, then lanes 0 .. nrows+2 issue one copy each (in parallel)
  auto issue = [&](int k) {
    const int q = k % nst;
    const int64_t b0 = (t0 + k) * kPassThreads;
    const int nbt = (int)imin64(kPassThreads, A.m - b0);
    const uint32_t rowb = 16u * (uint32_t)nbt;
    const uint32_t smallb = (4u * (uint32_t)nbt + 15u) & ~15u;
    unsigned char* dst = stages + (size_t)q * sb;
    if (lane == 0) mbar_arrive_expect_tx(&bars[q], (uint32_t)nrows * rowb + 3u * smallb);
    __syncwarp();
    for (int r = lane; r < nrows + 3; r += 32) {
      if (r < nrows)
        bulk_g2s(dst + (size_t)r * 4096, A.X16 + (int64_t)r * A.m_pad + b0, rowb, &bars[q]);
      else if (r == nrows)
        bulk_g2s(dst + (size_t)nrows * 4096, A.EPS16 + b0, smallb, &bars[q]);
      else if (r == nrows + 1)
        bulk_g2s(dst + (size_t)nrows * 4096 + 1024, A.R32 + b0, smallb, &bars[q]);
      else
        bulk_g2s(dst + (size_t)nrows * 4096 + 2048, A.slot + b0, smallb, &bars[q]);
    }
  };
  if (w == 0)
    for (int k = 0; k < nst && k < ntl; k++) issue(k);
  int count = 0;
  for (int k = 0; k < ntl; k++) {
    const int q = k % nst;
    const bool ok = mbar_wait_bounded(&bars[q], (uint32_t)((k / nst) & 1), A.wait_cycles);
    if (__syncthreads_or(!ok)) {
      // give up: record it, let the copies in flight land (bounded by the
      // default limit, whatever the wait limit was), return
      if (tid == 0) {
        st->status = kStatusWaitTimeout;
        for (int j = k; j < ntl && j < k + nst; j++)
          mbar_wait_bounded(&bars[j % nst], (uint32_t)((j / nst) & 1));
      }
      return;
    }
    const unsigned char* sbase = stages + (size_t)q * sb;
    const int64_t i = (t0 + k) * kPassThreads + tid;
    bool need = false;
    if (i < A.m) {
      const uint4* sx = reinterpret_cast<const uint4*>(sbase);
      const float ex = reinterpret_cast<const float*>(sbase + (size_t)nrows * 4096)[tid];
      const float r32 = reinterpret_cast<const float*>(sbase + (size_t)nrows * 4096 + 1024)[tid] * sc;
      const int sl = reinterpret_cast<const int*>(sbase + (size_t)nrows * 4096 + 2048)[tid];
      float2 Sa = make_float2(0.f, 0.f), Sb = Sa;
#pragma unroll 4
      for (int r = 0; r < nrows; r++) {
        const uint4 hv = sx[r * kPassThreads + tid];
        const float4 y0 = s_y[2 * r], y1 = s_y[2 * r + 1];
        acc_pair(h2f(hv.x), make_float2(y0.x, y0.y), Sa);
        acc_pair(h2f(hv.y), make_float2(y0.z, y0.w), Sb);
        acc_pair(h2f(hv.z), make_float2(y1.x, y1.y), Sa);
        acc_pair(h2f(hv.w), make_float2(y1.z, y1.w), Sb);
      }
      const float S = (Sa.x + Sa.y) + (Sb.x + Sb.y);
      if ((unsigned)sl < (unsigned)nsup && sidx[sl] == (int)i) {
        need = true;   // the ball holds a multiplier
      } else {
        const float ub = dist_ub16(S, ex, yn, k8);
        const float lb = (rq - r32) - 6.0f * kU32 * (fabsf(rq) + fabsf(r32)) - 1e-30f;
        need = !(ub <= lb);
        if (need) {
          const float dl = dist_lb16(S, ex, yn, k8);
          const float v = ((dl + r32 - rq) - 3.0f * kU32 * (dl + fabsf(r32) + fabsf(rq))) * unsc;
          if (v > 0.0f) v2sum = fmaf(v, v, v2sum);
        }
      }
    }
    const unsigned msk = __ballot_sync(MEB_FULLMASK, need);
    if (lane == 0) s_wc[w] = __popc(msk);
    __syncthreads();
    // every thread is past its reads of stage q: refill it
    if (w == 0 && k + nst < ntl) {
      fence_proxy_async_smem();   // each issuing lane orders the reads before its copy
      __syncwarp();
      issue(k + nst);
    }
    int off = 0, tot = 0;
#pragma unroll
    for (int kk = 0; kk < kPassWarps; kk++) {
      off += (kk < w) ? s_wc[kk] : 0;
      tot += s_wc[kk];
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
    for (int kk = 0; kk < kPassWarps; kk++) t += s_v2[kk];
    A.unc_cnt[blockIdx.x] = count;
    A.vlb_part[blockIdx.x] = t;
  }
  if (last_block_ticket(&st->ctr_screen)) early_body(B, A.d, gridDim.x);
}

__global__ void __launch_bounds__(kPassThreads) k_screen_all(PassArgs A, Buffers B) {
  pdl_wait_and_release();
  DevState* st = A.st;
  if (!screen_gate(st)) return;
  if (A.log_slot >= 0 && blockIdx.x == 0 && threadIdx.x == 0) st->screen_log[A.log_slot] = 1;
  screen_all_block(A, blockIdx.x);
  if (last_block_ticket(&st->ctr_screen)) early_body(B, A.d, gridDim.x);
}

int screen_variant(const Buffers& B, int d) {
  if (B.fp64_all) return 3;
  if (!B.use_x16) return 0;
  return (B.bulk && bulk_stages(d) >= 2) ? 2 : 1;
}

// Resident k_screen blocks on this GPU for a given dynamic shared memory size
// (one wave of blocks), cached per size.
static int screen_resident_blocks(int d, int variant) {
  // one cached entry per variant (and device)
  static int cached_dev[4] = {-1, -1, -1, -1}, cached_d[4] = {-1, -1, -1, -1},
             cached[4] = {0, 0, 0, 0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (cached_d[variant] != d || cached_dev[variant] != dev) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int d4 = (d + 3) / 4;
    const size_t sh1 = 16 * (size_t)(2 * ((d4 + 1) / 2));
    if (variant == 2) per = 1;
    else if (variant == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_screen_all, kPassThreads, 0);
    else if (variant == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_screen<true>, kPassThreads, sh1);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_screen<false>, kPassThreads, sh1);
    if (per < 1) per = 1;
    if (sms < 1) sms = 1;
    cached[variant] = sms * per;
    cached_d[variant] = d;
    cached_dev[variant] = dev;
  }
  return cached[variant];
}

// Host set-up outside any stream capture: the grid of the current variant
// and the shared-memory size of the bulk-copy screen.
cudaError_t prepare_pass(const Buffers& B, int d) {
  int tpb;
  const int variant = screen_variant(B, d);
  pass_blocks(1, d, variant, &tpb);
  if (variant == 2) {
    const size_t shb = bulk_smem(d, bulk_stages(d));
    return raise_smem_limit((const void*)k_screen_bulk, shb);
  }
  return cudaSuccess;
}

int pass_blocks(int64_t m, int d, int variant, int* tiles_per_block) {
  const int64_t ntiles = (m + kPassThreads - 1) / kPassThreads;
  const int64_t target = screen_resident_blocks(d, variant);
  const int64_t cap = target < kMaxPassBlocks ? target : kMaxPassBlocks;
  int64_t tpb = (ntiles + cap - 1) / cap;
  if (tpb < 1) tpb = 1;
  *tiles_per_block = (int)tpb;
  return (int)((ntiles + tpb - 1) / tpb);
}

cudaError_t launch_pass(const double* C, const double* R, Buffers& B, int64_t m, int d,
                        cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int log_slot) {
  PassArgs A;
  A.log_slot = log_slot;
  A.wait_cycles = B.wait_cycles;
  A.C = C; A.R = R; A.m = m;
  const int d4 = (d + 3) / 4;
  A.m_pad = ((m + 255) / 256) * 256;
  A.d = d; A.d4 = d4;
  const int variant = screen_variant(B, d);
  const int nb = pass_blocks(m, d, variant, &A.tiles_per_block);
  A.X32 = B.X32; A.X16 = B.use_x16 ? B.X16 : nullptr; A.EPS16 = B.EPS16; A.E32 = B.E32; A.R32 = B.R32; A.slot = B.slot;
  A.sup_idx0 = B.sup_idx[0]; A.sup_idx1 = B.sup_idx[1];
  A.sup_u0 = B.sup_u[0]; A.sup_u1 = B.sup_u[1];
  A.sup_v0 = B.sup_v[0]; A.sup_v1 = B.sup_v[1];
  A.sup_vv0 = B.sup_vv[0]; A.sup_vv1 = B.sup_vv[1];
  A.st = B.st; A.ct = B.vec.ct; A.y32 = B.vec.y32;
  A.unc_cnt = B.unc_cnt; A.unc_idx = B.unc_idx; A.unc_slot = B.unc_slot;
  A.vlb_part = B.vlb_part;
  A.part_flag = B.part_flag; A.part = B.part; A.part_cnt = B.part_cnt;
  A.cand_cnt = B.cand_cnt; A.cand_idx = B.cand_idx; A.cand_case = B.cand_case;
  A.cand_a = B.cand_a; A.cand_n = B.cand_n; A.cand_u = B.cand_u;
  const size_t sh1 = 16 * (size_t)(2 * ((d4 + 1) / 2));   // -y padded to whole FP16 rows
  cudaError_t e;
  {
    e = raise_smem_limit((const void*)k_screen<false>, sh1);
    if (e != cudaSuccess) return e;
    e = raise_smem_limit((const void*)k_screen<true>, sh1);
    if (e != cudaSuccess) return e;
  }
  // cudaEventRecordExternal: inside a stream capture the records become event
  // nodes of the graph, so the events carry device times of every launch
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (ev0 || ev1) cudaStreamIsCapturing(s, &cap);
  const unsigned evf = (cap == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : 0u;
  if (ev0) cudaEventRecordWithFlags(ev0, s, evf);
  if (variant == 2) {   // its shared-memory attribute is set by prepare_pass
    const int nst = bulk_stages(d);
    e = launch_pdl(k_screen_bulk, dim3(nb), dim3(kPassThreads), bulk_smem(d, nst), s, A, B, nst);
  } else if (variant == 3) {
    e = launch_pdl(k_screen_all, dim3(nb), dim3(kPassThreads), 0, s, A, B);
  } else if (variant == 1) {
    e = launch_pdl(k_screen<true>, dim3(nb), dim3(kPassThreads), sh1, s, A, B);
  } else {
    e = launch_pdl(k_screen<false>, dim3(nb), dim3(kPassThreads), sh1, s, A, B);
  }
  if (e != cudaSuccess) {
    note_launch_failure("screen", (unsigned)nb, sh1, e);
    return e;
  }
  if (ev1) cudaEventRecordWithFlags(ev1, s, evf);
  const size_t sh2 = 8 * (size_t)d;
  {
    e = raise_smem_limit((const void*)k_rows64<false>, sh2);
    if (e != cudaSuccess) return e;
    e = raise_smem_limit((const void*)k_rows64<true>, sh2);
    if (e != cudaSuccess) return e;
  }
  e = B.lowp ? launch_pdl(k_rows64<true>, dim3(nb), dim3(kPassThreads), sh2, s, A, B)
             : launch_pdl(k_rows64<false>, dim3(nb), dim3(kPassThreads), sh2, s, A, B);
  if (e != cudaSuccess) {
    note_launch_failure(B.lowp ? "rows (FP32)" : "rows", (unsigned)nb, sh2, e);
    return e;
  }
  B.launches += 2;
  return cudaGetLastError();
}

// ctl: controller B in the last block (else k_svec_reduce follows)
template <bool LOWP>
__global__ void __launch_bounds__(256) k_svec(const double* __restrict__ C, Buffers B, int d,
                                              int npb, int64_t seg, int nsvb, int ctl) {
  pdl_wait_and_release();
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_GRAD) return;
  svec_block<LOWP>(C, B, d, npb, seg, blockIdx.x, nsvb);
  if (ctl && last_block_ticket(&st->ctr_svec)) control_b_body(B, d);
}

// Rows of d >= 512: the 3d + 1 sums over the support blocks' partials, one
// entry per thread over the grid (the same order as in controller B), then
// controller B in the last block.
__global__ void __launch_bounds__(256) k_svec_reduce(Buffers B, int d) {
  pdl_wait_and_release();
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_GRAD) return;
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e < 3 * d + 1) svec_sum_entry(B, d, e, st->svec_nb);
  if (last_block_ticket(&st->ctr_svecr)) control_b_body(B, d, true);
}

bool support_rows_wide(const Buffers& B, int d) { return !B.lowp && d >= 512; }

cudaError_t launch_support_rows(const double* C, Buffers& B, int64_t m, int d, cudaStream_t s) {
  int tpb;
  const int nb = pass_blocks(m, d, screen_variant(B, d), &tpb);
  // wide rows: three blocks per SM for the FP64 work, the partial sums spread
  // over a grid of their own
  const bool wide = support_rows_wide(B, d);
  const int nsvb = wide ? kSvecBlocksWide : kSvecBlocks;
  cudaError_t e = B.lowp ? launch_pdl(k_svec<true>, dim3(nsvb), dim3(256), 0, s, C, B, d,
                                      nb, (int64_t)tpb * kPassThreads, nsvb, 1)
                        : launch_pdl(k_svec<false>, dim3(nsvb), dim3(256), 0, s, C, B, d,
                                      nb, (int64_t)tpb * kPassThreads, nsvb, wide ? 0 : 1);
  if (e != cudaSuccess) return e;
  B.launches += 1;
  if (wide) {
    e = launch_pdl(k_svec_reduce, dim3((3 * d + 1 + 255) / 256), dim3(256), 0, s, B, d);
    if (e != cudaSuccess) return e;
    B.launches += 1;
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kFeasNT) k_feas_a(FeasArgs A) { feas_a_block(A, blockIdx.x); }

__global__ void k_feas_L(const float* __restrict__ blb, int nb, float* __restrict__ L) {
  feas_L_body(blb, nb, L);
}

__global__ void __launch_bounds__(kFeasNT) k_feas_b(FeasArgs A) { feas_b_block(A, blockIdx.x); }

__global__ void k_feas_final(const double* __restrict__ bmax, const int64_t* __restrict__ barg,
                             const int* __restrict__ bcnt, int nb, double* out_max,
                             int64_t* out_arg, int64_t* out_cnt) {
  feas_final_body(bmax, barg, bcnt, nb, out_max, out_arg, out_cnt);
}

__global__ void k_gather_lists(const int* __restrict__ cnt, const int64_t* __restrict__ lists,
                               int nb, int T, int64_t* __restrict__ out, int64_t cap) {
  gather_lists_block(blockIdx.x, cnt, lists, nb, T, out, cap);
}

// Sum of per-tile counts into *out (one block).
__global__ void k_count_sum(const int* __restrict__ cnt, int nb, int64_t* __restrict__ out) {
  __shared__ long long sh[256];
  long long v = 0;
  for (int b = threadIdx.x; b < nb; b += 256) v += cnt[b];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_query_shadow(const double* __restrict__ c, const double* __restrict__ o, int d,
                               float* __restrict__ y32, float* __restrict__ yn, int* bad) {
  query_shadow_body(c, o, d, y32, yn, bad);
}

cudaError_t launch_feas_cert(const double* C, const double* R, int64_t m, int d, const double* c,
                             double r, double eps, int mode, int want_max, Buffers& B,
                             double* dmax_out, int64_t* argmax_out, int64_t* nviol_out,
                             cudaStream_t s, bool reuse_bounds, int* bad) {
  FeasArgs A;
  A.C = C; A.R = R; A.m = m;
  A.m_pad = ((m + 255) / 256) * 256;
  A.d = d; A.d4 = (d + 3) / 4;
  A.X32 = B.X32; A.R32 = B.R32; A.E32 = B.E32;
  A.c = c;
  A.y32 = B.fq_y32;
  A.r = r; A.eps = eps; A.mode = mode; A.want_max = want_max;
  A.all64 = B.fp64_all ? 1 : 0;
  A.eub = B.fe_ub; A.elb = B.fe_lb; A.blb = B.fe_blb;
  A.bmax = B.feas_part; A.barg = B.feas_ipart; A.bcnt = B.feas_cnt; A.blist = B.list_tmp;
  A.L = B.fe_L;
  A.ynp = B.fe_L + 1;
  const int nb = (int)((m + kFeasNT - 1) / kFeasNT);
  cudaError_t e;
  int launched = 3;
  // the bounds on e_i depend only on c: a second check at the same centre
  // (reuse_bounds) skips the shadow sweep; the plain FP64 pass has no bounds
  if (!reuse_bounds) {
    k_query_shadow<<<1, 256, 0, s>>>(c, B.vec.o, d, B.fq_y32, B.fe_L + 1, bad);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launched += 1;
  }
  if (!reuse_bounds && !A.all64) {
    const size_t sha = 16 * (size_t)A.d4;
    {
      e = raise_smem_limit((const void*)k_feas_a, sha);
      if (e != cudaSuccess) return e;
    }
    k_feas_a<<<nb, kFeasNT, sha, s>>>(A);
    launched += 1;
  }
  if (want_max && !A.all64) {
    k_feas_L<<<1, 256, 0, s>>>(B.fe_blb, nb, B.fe_L);
    launched += 1;
  }
  const size_t shb = 8 * (size_t)d;
  {
    e = raise_smem_limit((const void*)k_feas_b, shb);
    if (e != cudaSuccess) return e;
  }
  k_feas_b<<<nb, kFeasNT, shb, s>>>(A);
  k_feas_final<<<1, 256, 0, s>>>(B.feas_part, B.feas_ipart, B.feas_cnt, nb, dmax_out, argmax_out,
                                 nviol_out);
  k_gather_lists<<<(nb + 255) / 256, 256, 0, s>>>(B.feas_cnt, B.list_tmp, nb, kFeasNT, B.viol, m);
  B.launches += launched;
  return cudaGetLastError();
}

// ===========================================================================
// Evaluation entry: support from dense (U, V) rows.
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
  const unsigned msk = __ballot_sync(MEB_FULLMASK, nz);
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
    double vv = 0.0;
    for (int j = lane; j < d; j += 32) {
      const double v = V[i * (int64_t)d + j];
      B.sup_v[0][k * d + j] = v;
      vv = fma(v, v, vv);
    }
    vv = warp_sum_t(vv);
    if (lane == 0) {
      B.sup_vv[0][k] = vv;
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
  B.launches += 4;
  return cudaGetLastError();
}

}  // namespace meb
