// libmeb C ABI (include/meb.h): contexts, device memory, and the host loop
// that launches the device-resident ripALM / SSN steps.  The host never does
// arithmetic of the method: it validates sizes, moves buffers, launches the
// kernels of meb_pass.cu and meb_solve.cu and reads back the controller's
// action/status.
#include <cuda_runtime.h>
#include <math.h>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <iterator>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/meb.h"
#include "meb_internal.cuh"

using namespace meb;


struct meb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Buffers B{};
  void* arena = nullptr;        // one allocation holding every array of B
  size_t arena_bytes = 0;
  int64_t buf_m = 0;
  int buf_d = 0;
  bool batch_per_item = false;  // meb_solve_batch: one scratch slot per instance
  bool release = false;         // free all device scratch at the end of each call
  cudaMemPool_t mempool = nullptr;   // with release: the pool to allocate from (else the device's)
  bool blocking = false;        // waits sleep on sync_ev instead of spinning (MEB_OPT_BLOCKING_SYNC)
  cudaEvent_t sync_ev = nullptr;
  int depth = 0;                // nesting of public calls (a batch falls back to meb_solve)
  void* pool_ptr[32] = {};
  size_t pool_cap[32] = {};
  DevState* h_st = nullptr;     // pinned mirror of the device state
  double* h_scal = nullptr;     // pinned scalars
  int* d_flags = nullptr;       // device int flags
  double* d_scal = nullptr;     // device scalars
  int64_t* d_i64 = nullptr;     // device int64 scalars
  int profiling = 0;            // time every pass launch with CUDA events
  // device-resident solve loops: CUDA graphs of controller ticks, one per
  // buffer set in use (the full instance and, in the mixed-precision
  // pipeline, the reduced one); rebuilt when the problem or buffers change
  struct TickGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t m = 0;
    int d = 0, mode = -1, var = -1, prof = -1, lowp = -1, dense = -1;
    long long wait = -1;
  } tg[2];
  cudaStream_t stream2 = nullptr;   // captures the CG loop bodies of tick graphs; chunked copy-in
  cudaEvent_t stage_ev[2] = {};     // chunked copy-in: buffers free, chunk landed
  int tg_next = 0;
  cudaEvent_t gev[2 * 8] = {};
  // the reduced instance of the mixed-precision pipeline
  Buffers Bred{};
  void* red_arena = nullptr;
  size_t red_bytes = 0;
  // options (meb_set_option)
  // tick loop: 0 = graph of kUnrollTicks ticks relaunched until the controller
  // stops (default), 1 = host-driven ticks, 2 = graph with a while-node
  int loop_mode = 0;
  int screen_mode = MEB_SCREEN_FP16;      // solves
  int eval_screen = MEB_SCREEN_FP32;      // meb_eval_alm
  int eval_shadow_exp = 0;                // FP16 shadow scale 2^exp of meb_eval_alm
  long long wait_cycles = 2000000000LL;   // bound of the bulk-copy screen's waits
  // multipliers of the last solve (meb_get_multipliers): 0 none, 1 the
  // support arrays of the final point, 2 one ball, 3 all balls the same point,
  // 4 the reduced instance's support arrays (indices mapped back to the balls)
  int mult_kind = 0;
  const int64_t* mult_map = nullptr;
  int64_t mult_n = 0, mult_m = 0;
  int mult_d = 0;
  // batched solver: configuration per class of d (meb_tune_batch)
  BatchConfig batch_cfg[MEB_BATCH_CLASSES] = {
      {0, 8, 8, 0}, {1, 8, 8, 0}, {1, 8, 8, 0}, {1, 8, 8, 0}, {1, 8, 8, 0}};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  meb_stats stats{};
  int prof_screens = 0;
  char err[512] = {0};
};

// kernels launched per controller tick of the device-resident loop
// kernels of one controller tick: pass (2), support rows (1), the dense
// Newton step, the multiplier update (1)
static int64_t tick_launches(int d) { return 2 + 1 + newton_dense_launches(d) + 1; }
static const int kUnrollTicks = 8;

enum { POOL_C, POOL_R, POOL_U, POOL_V, POOL_X, POOL_XB, POOL_Q, POOL_UP, POOL_VP, POOL_HQ,
       POOL_H, POOL_G, POOL_COUT, POOL_ACT, POOL_BIN, POOL_BOUT, POOL_BITEMS, POOL_BRES,
       POOL_BSLOTS, POOL_BSLOTB, POOL_BCFG, POOL_RED_IDX, POOL_RED_C, POOL_RED_R, POOL_WIDX,
       POOL_WU, POOL_WV, POOL_WX, POOL_N };
static_assert(POOL_N <= 32, "pool table");

static int fail(meb_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MEB_ENOMEM : MEB_ECUDA,      \
                  "%s: %s (%s:%d) [%s]", #call, cudaGetErrorString(e_), __FILE__, __LINE__, \
                  launch_failure_note());                                             \
  } while (0)

// Device allocations of the context's scratch.  With MEB_OPT_RELEASE_SCRATCH
// they are stream-ordered on the context's stream (cudaMallocAsync /
// cudaFreeAsync), so that allocating and freeing on one context never waits
// for work of another; otherwise plain cudaMalloc / cudaFree.
static cudaError_t dev_alloc(meb_ctx* ctx, void** p, size_t bytes) {
  if (!ctx->release) return cudaMalloc(p, bytes);
  return ctx->mempool ? cudaMallocFromPoolAsync(p, bytes, ctx->mempool, ctx->stream)
                      : cudaMallocAsync(p, bytes, ctx->stream);
}
static void dev_free(meb_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->release) cudaFreeAsync(p, ctx->stream);
  else cudaFree(p);
}

static void drop_graphs(meb_ctx* ctx) {
  for (auto& g : ctx->tg) {
    if (g.gexec) cudaGraphExecDestroy(g.gexec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = meb_ctx::TickGraph{};
  }
}

static void free_buffers(meb_ctx* ctx) {
  Buffers& B = ctx->B;
  dev_free(ctx, ctx->red_arena);
  ctx->red_arena = nullptr;
  ctx->red_bytes = 0;
  ctx->Bred = Buffers{};
  dev_free(ctx, ctx->arena);
  ctx->arena = nullptr;
  ctx->arena_bytes = 0;
  const int64_t launches = B.launches;
  memset(&B, 0, sizeof(B));
  B.launches = launches;
  ctx->buf_m = 0;
  ctx->buf_d = 0;
  // captured tick graphs hold freed pointers: rebuild them on next use
  drop_graphs(ctx);
}

// The scratch of a multi-block solve of (m, d), laid out in one arena
// (base == nullptr: only the size).  Every array starts on a 256-byte boundary.
static size_t solve_layout(Buffers* Bp, char* base, int64_t m, int d) {
  Buffers B{};
  size_t off = 0;
  auto take = [&](auto** p, size_t n) {
    using T = std::remove_reference_t<decltype(**p)>;
    off = (off + 255) & ~(size_t)255;
    if (base) *p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * (n ? n : 1);
  };
  const int64_t m_pad = ((m + 255) / 256) * 256;
  const int64_t nblk = m_pad / 256;
  const int d4 = (d + 3) / 4;
  const int n1 = d + 1;
  const int64_t md = m * (int64_t)d;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int64_t ntri = (int64_t)nt * (nt + 1) / 2;
  int64_t hp = (int64_t)152 * n1;
  if (d + 1 <= kMaxDenseN) hp = hp > 24 * ntri * 1024 ? hp : 24 * ntri * 1024;
  const size_t dn = (size_t)(d + 1 <= kMaxDenseN ? n1 * n1 : 1);
  take(&B.X32, (size_t)d4 * m_pad);
  take(&B.X16, (size_t)((d4 + 1) / 2) * m_pad);
  take(&B.EPS16, m_pad);
  take(&B.E32, m_pad);
  take(&B.Hhi, dn);
  take(&B.Hlo, dn);
  take(&B.Ainv, n1 <= kAinvMaxN ? (size_t)kAinvLen : 0);
  if (n1 > kAinvMaxN) B.Ainv = nullptr;
  take(&B.R32, m_pad);
  take(&B.slot, m_pad);   // whole tiles are bulk-copied
  for (int k = 0; k < 2; k++) {
    take(&B.sup_idx[k], m);
    take(&B.sup_u[k], m);
    take(&B.sup_v[k], md);
    take(&B.sup_vv[k], m);
  }
  // segments of 256 per tile and block: at most (tiles + blocks) * 256 for any grid
  const int64_t ncand = (nblk + kMaxPassBlocks) * 256;
  take(&B.part_flag, nblk);
  take(&B.part, nblk * P_NREC);
  take(&B.part_cnt, nblk * P_NCNT);
  take(&B.cand_off, nblk + 1);
  take(&B.cand_cnt, nblk);
  take(&B.unc_cnt, nblk);
  take(&B.vlb_part, nblk);
  take(&B.unc_idx, ncand);
  take(&B.unc_slot, ncand);
  take(&B.cand_idx, ncand);
  take(&B.cand_case, ncand);
  take(&B.cand_a, ncand);
  take(&B.cand_n, ncand);
  take(&B.cand_u, ncand);
  take(&B.S_idx, m);
  take(&B.S_case, m);
  take(&B.S_a, m);
  take(&B.S_n, m);
  take(&B.S_u, m);
  take(&B.S_t, m);
  take(&B.W, md);
  if (d + 1 > kMaxDenseN) take(&B.W32, md);   // the matrix-free path for sure: FP32 rows
  take(&B.svec_part, (size_t)(d >= 512 ? kSvecBlocksWide : kSvecBlocks) * (3 * d + 1));
  take(&B.hpart, hp);
  take(&B.H, dn);
  take(&B.hq, n1);
  take(&B.colsum_part, (size_t)((m + 63) / 64) * d);
  take(&B.fe_ub, m);
  take(&B.fe_lb, m);
  take(&B.fe_blb, nblk);
  take(&B.fe_L, 4);
  take(&B.fq_y32, (size_t)4 * d4 + 4);
  take(&B.feas_part, nblk + 8);
  take(&B.feas_ipart, nblk + 8);
  take(&B.feas_cnt, nblk + 8);
  take(&B.viol, m);
  take(&B.list_tmp, m_pad);
  take(&B.count64, 8);
  take(&B.scal, 8);
  take(&B.wq, m);
  take(&B.cf32, m);
  take(&B.st, 1);
  // vectors of length n1 (x, xt, xk, ab, g, gt, dx, ct, o, sv, sw, st1, cg_*) and y32;
  // each starts on a 16-byte boundary (y32 is read as float4)
  const size_t stride = (size_t)((n1 + 8 + 1) / 2) * 2;
  const size_t nv = 20 * stride + (size_t)(d4 * 4 + 8);
  take(&B.vec_store, nv);
  if (base) {
    double* p = B.vec_store;
    auto vtake = [&](double** q) { *q = p; p += stride; };
    vtake(&B.vec.x); vtake(&B.vec.xt); vtake(&B.vec.xk); vtake(&B.vec.ab); vtake(&B.vec.g);
    vtake(&B.vec.gt); vtake(&B.vec.dx); vtake(&B.vec.ct); vtake(&B.vec.o); vtake(&B.vec.c0);
    vtake(&B.vec.sv);
    vtake(&B.vec.sw); vtake(&B.vec.st1); vtake(&B.vec.cg_r); vtake(&B.vec.cg_z); vtake(&B.vec.cg_p);
    vtake(&B.vec.cg_ap); vtake(&B.vec.cg_diag);
    B.vec.y32 = reinterpret_cast<float*>(p);
    B.m_cap = m;
    B.d_cap = d;
    B.nblk_cap = nblk;
    B.hpart_cap = hp;
    const int64_t launches = Bp->launches;
    *Bp = B;
    Bp->launches = launches;
  }
  return (off + 255) & ~(size_t)255;
}

// Device buffers sized for (m, d) in one arena; grown on demand.
static int ensure_buffers(meb_ctx* ctx, int64_t m, int d) {
  if (ctx->buf_m >= m && ctx->buf_d >= d && ctx->buf_m * (int64_t)ctx->buf_d >= m * (int64_t)d &&
      ctx->buf_d == d)
    return MEB_OK;
  free_buffers(ctx);
  const size_t bytes = solve_layout(nullptr, nullptr, m, d);
  CK(dev_alloc(ctx, &ctx->arena, bytes));
  ctx->arena_bytes = bytes;
  solve_layout(&ctx->B, (char*)ctx->arena, m, d);
  const int n1 = d + 1, d4 = (d + 3) / 4;
  const size_t nv = 20 * (size_t)((n1 + 8 + 1) / 2) * 2 + (size_t)(d4 * 4 + 8);
  CK(cudaMemsetAsync(ctx->B.vec_store, 0, sizeof(double) * nv, ctx->stream));
  ctx->buf_m = m;
  ctx->buf_d = d;
  return MEB_OK;
}

// Release every device scratch of the context (buffers, pools, tick graph).
// Wait for the context's stream: a spin (cudaStreamSynchronize), or with
// MEB_OPT_BLOCKING_SYNC a sleep on a blocking-sync event, so that many
// threads waiting on their own contexts do not occupy the host cores.
static cudaError_t ctx_sync(meb_ctx* ctx) {
  if (!ctx->blocking || !ctx->sync_ev) return cudaStreamSynchronize(ctx->stream);
  cudaError_t e = cudaEventRecord(ctx->sync_ev, ctx->stream);
  return e == cudaSuccess ? cudaEventSynchronize(ctx->sync_ev) : e;
}

static void release_scratch(meb_ctx* ctx) {
  free_buffers(ctx);
  for (int k = 0; k < 32; k++) {
    dev_free(ctx, ctx->pool_ptr[k]);
    ctx->pool_ptr[k] = nullptr;
    ctx->pool_cap[k] = 0;
  }
}

// Scope of a public compute call: with MEB_OPT_RELEASE_SCRATCH set, the
// outermost call frees the context's device scratch when it returns.
struct CallScope {
  meb_ctx* c;
  explicit CallScope(meb_ctx* ctx) : c(ctx) {
    // an earlier failed launch of this thread must not surface here
    if (c->depth++ == 0) (void)cudaGetLastError();
  }
  ~CallScope() {
    if (--c->depth == 0 && c->release) {
      ctx_sync(c);
      release_scratch(c);
    }
  }
};

static int pool(meb_ctx* ctx, int id, size_t bytes, void** out) {
  if (ctx->pool_cap[id] < bytes) {
    dev_free(ctx, ctx->pool_ptr[id]);
    ctx->pool_ptr[id] = nullptr;
    ctx->pool_cap[id] = 0;
    CK(dev_alloc(ctx, &ctx->pool_ptr[id], bytes ? bytes : 8));
    ctx->pool_cap[id] = bytes;
  }
  *out = ctx->pool_ptr[id];
  return MEB_OK;
}

// Device view of an input array (copy-in when it is a host array).
static int stage_in(meb_ctx* ctx, int id, const void* src, size_t bytes, unsigned flags,
                    const void** out) {
  if (flags & MEB_PTR_DEVICE) {
    *out = src;
    return MEB_OK;
  }
  void* d = nullptr;
  int rc = pool(ctx, id, bytes, &d);
  if (rc) return rc;
  CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *out = d;
  return MEB_OK;
}

// Host centres of a large instance: copied in chunks of about 64 MB on the
// second stream; the shadow sweep of each chunk (whole 64-ball shadow blocks)
// runs on the solve's stream as soon as that chunk has landed, under the copy
// of the next one.  The radii and the first centre (the shadow origin) land
// with the first chunk.  Leaves the shadow blocks done and the input flag set;
// the mean centre is left to the caller.
constexpr size_t kStageChunkBytes = size_t(64) << 20;

static bool stage_chunked(unsigned flags, int64_t m, int d) {
  return !(flags & MEB_PTR_DEVICE) && sizeof(double) * (size_t)m * d > 2 * kStageChunkBytes;
}

static int stage_in_shadowed(meb_ctx* ctx, Buffers& B, const double* centers, const double* radii,
                             int64_t m, int d, const double** Cp, const double** Rp) {
  cudaStream_t s = ctx->stream;
  double* dC = nullptr;
  double* dR = nullptr;
  int rc = pool(ctx, POOL_C, sizeof(double) * (size_t)m * d, (void**)&dC);
  if (rc) return rc;
  if ((rc = pool(ctx, POOL_R, sizeof(double) * (size_t)m, (void**)&dR))) return rc;
  if (!ctx->stream2) CK(cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
  for (int k = 0; k < 2; k++)
    if (!ctx->stage_ev[k]) CK(cudaEventCreateWithFlags(&ctx->stage_ev[k], cudaEventDisableTiming));
  cudaStream_t s2 = ctx->stream2;
  // the copies wait for earlier work of this context on the same buffers
  CK(cudaEventRecord(ctx->stage_ev[0], s));
  CK(cudaStreamWaitEvent(s2, ctx->stage_ev[0], 0));
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
  CK(cudaMemcpyAsync(dR, radii, sizeof(double) * (size_t)m, cudaMemcpyHostToDevice, s2));
  const int64_t nb = (m + kShadowBallsPerBlock - 1) / kShadowBallsPerBlock;
  const int64_t per = std::max<int64_t>(
      1, (int64_t)(kStageChunkBytes / (sizeof(double) * (size_t)kShadowBallsPerBlock * d)));
  cudaError_t e = cudaSuccess;
  for (int64_t b0 = 0; b0 < nb && e == cudaSuccess; b0 += per) {
    const int64_t b1 = std::min(nb, b0 + per);
    const int64_t i0 = b0 * kShadowBallsPerBlock;
    const int64_t i1 = std::min(m, b1 * kShadowBallsPerBlock);
    e = cudaMemcpyAsync(dC + i0 * d, centers + i0 * d, sizeof(double) * (size_t)(i1 - i0) * d,
                        cudaMemcpyHostToDevice, s2);
    // a wait takes the event's latest record at the time of the call
    if (e == cudaSuccess) e = cudaEventRecord(ctx->stage_ev[1], s2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->stage_ev[1], 0);
    if (e == cudaSuccess) e = launch_shadow_blocks(dC, dR, m, d, B, b0, b1, ctx->d_flags, s);
  }
  if (e != cudaSuccess) {
    // whatever was issued on the second stream finishes before the solve's
    // stream goes on (and before the buffers can be freed on it)
    const cudaError_t e2 = cudaEventRecord(ctx->stage_ev[1], s2);
    if (e2 == cudaSuccess) cudaStreamWaitEvent(s, ctx->stage_ev[1], 0);
    else cudaStreamSynchronize(s2);
    return fail(ctx, MEB_ECUDA, "chunked copy-in: %s", cudaGetErrorString(e));
  }
  *Cp = dC;
  *Rp = dR;
  return MEB_OK;
}

static int copy_out(meb_ctx* ctx, void* dst, const void* dsrc, size_t bytes, unsigned flags) {
  if (!bytes) return MEB_OK;
  CK(cudaMemcpyAsync(dst, dsrc, bytes,
                     (flags & MEB_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->stream));
  return MEB_OK;
}

namespace meb {

// The dynamic shared-memory limit of a kernel is process-wide (per device):
// several host threads launching the same kernel with different sizes must
// never lower it under one another, so it is only ever raised, under a lock.
// (A kernel with static shared memory needs the opt-in for any dynamic size
// that takes the total past 48 KB, so it is set for every size asked.)
cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cur;
  if (bytes == 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& c = cur[std::make_pair(dev, fn)];
  if (bytes <= c) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) c = bytes;
  return e;
}

// The kernel launch that failed last on this host thread (for the message).
static thread_local char g_launch_note[160] = {0};
void note_launch_failure(const char* what, unsigned grid, size_t smem, cudaError_t e) {
  snprintf(g_launch_note, sizeof(g_launch_note), "%s grid %u smem %zu: %s", what, grid, smem,
           cudaGetErrorString(e));
}
const char* launch_failure_note() { return g_launch_note; }

}  // namespace meb

extern "C" {

void meb_params_default(meb_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tol = 1e-10;
  p->rho = 0.5;
  p->sigma0 = 10.0;
  p->sigma_max = 1e7;
  p->sigma_growth = 10.0;
  p->sigma_ratio = 0.1;
  p->tau = 10.0;
  p->armijo_mu = 1e-4;
  p->active_theta = 2e-6;
  p->max_outer = 500;
  p->max_ssn = 50;
  p->max_backtrack = 40;
  p->dense_max_d = kMaxDenseN - 1;
  p->max_cg = 500;
  p->mixed = 0;
  p->max_readd = 8;
  p->tol_lp = 1e-2;
  p->tol_red = 0.0;
}

int meb_create(meb_ctx** out, int device, void* cuda_stream) {
  if (!out) return MEB_EINVAL;
  *out = nullptr;
  meb_ctx* ctx = new (std::nothrow) meb_ctx();
  if (!ctx) return MEB_ENOMEM;
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess && cuda_stream) ctx->stream = (cudaStream_t)cuda_stream;
  if (e == cudaSuccess && !cuda_stream) {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    ctx->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_scal, 64 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_flags, 16 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_scal, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_i64, 16 * sizeof(int64_t));
  if (e != cudaSuccess) {
    meb_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? MEB_ENOMEM : MEB_ECUDA;
  }
  *out = ctx;
  return MEB_OK;
}

void meb_destroy(meb_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) ctx_sync(ctx);
  release_scratch(ctx);
  if (ctx->stream) ctx_sync(ctx);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->d_flags) cudaFree(ctx->d_flags);
  if (ctx->d_scal) cudaFree(ctx->d_scal);
  if (ctx->d_i64) cudaFree(ctx->d_i64);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
  for (int k = 0; k < 2; k++)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  drop_graphs(ctx);
  for (int k = 0; k < 16; k++)
    if (ctx->gev[k]) cudaEventDestroy(ctx->gev[k]);
  if (ctx->sync_ev) cudaEventDestroy(ctx->sync_ev);
  for (int k = 0; k < 2; k++)
    if (ctx->stage_ev[k]) cudaEventDestroy(ctx->stage_ev[k]);
  delete ctx;
}

const char* meb_last_error(const meb_ctx* ctx) { return ctx ? ctx->err : "no context"; }

int meb_set_option(meb_ctx* ctx, int32_t option, int64_t value) {
  if (!ctx) return MEB_EINVAL;
  switch (option) {
    case MEB_OPT_SCREEN:
    case MEB_OPT_EVAL_SCREEN:
      if (value < MEB_SCREEN_FP16 || value > MEB_SCREEN_FP64)
        return fail(ctx, MEB_EINVAL, "unknown screen mode %lld", (long long)value);
      (option == MEB_OPT_SCREEN ? ctx->screen_mode : ctx->eval_screen) = (int)value;
      return MEB_OK;
    case MEB_OPT_EVAL_SHADOW_EXP:
      if (value < -60 || value > 60) return fail(ctx, MEB_EINVAL, "shadow exponent out of range");
      ctx->eval_shadow_exp = (int)value;
      return MEB_OK;
    case MEB_OPT_TICK_LOOP:
      if (value < 0 || value > 2) return fail(ctx, MEB_EINVAL, "unknown tick loop %lld", (long long)value);
      ctx->loop_mode = (int)value;
      return MEB_OK;
    case MEB_OPT_WAIT_CYCLES:
      if (value < 0) return fail(ctx, MEB_EINVAL, "negative wait limit");
      ctx->wait_cycles = (long long)value;
      return MEB_OK;
    case MEB_OPT_BATCH_SLOTS:
      if (value < 0 || value > 1) return fail(ctx, MEB_EINVAL, "batch slots: 0 or 1");
      ctx->batch_per_item = value == 1;
      return MEB_OK;
    case MEB_OPT_RELEASE_SCRATCH:
      if (value < 0 || value > 1) return fail(ctx, MEB_EINVAL, "release scratch: 0 or 1");
      ctx->release = value == 1;
      return MEB_OK;
    case MEB_OPT_BLOCKING_SYNC:
      if (value < 0 || value > 1) return fail(ctx, MEB_EINVAL, "blocking sync: 0 or 1");
      if (value == 1 && !ctx->sync_ev) {
        CK(cudaSetDevice(ctx->device));
        CK(cudaEventCreateWithFlags(&ctx->sync_ev, cudaEventBlockingSync | cudaEventDisableTiming));
      }
      ctx->blocking = value == 1;
      return MEB_OK;
    default:
      return fail(ctx, MEB_EINVAL, "unknown option %d", (int)option);
  }
}

// Library-internal (the serving loop, meb_serve.cpp): with
// MEB_OPT_RELEASE_SCRATCH, allocate the context's scratch from `pool`.
__attribute__((visibility("hidden"))) void meb_ctx_use_pool(meb_ctx* ctx, cudaMemPool_t pool) {
  if (ctx) ctx->mempool = pool;
}

int meb_set_profiling(meb_ctx* ctx, int on) {
  if (!ctx) return MEB_EINVAL;
  if (on && !ctx->ev[0]) {
    CK(cudaSetDevice(ctx->device));
    CK(cudaEventCreate(&ctx->ev[0]));
    CK(cudaEventCreate(&ctx->ev[1]));
  }
  ctx->profiling = on ? 1 : 0;
  return MEB_OK;
}

int meb_get_stats(meb_ctx* ctx, meb_stats* out) {
  if (!ctx || !out) return MEB_EINVAL;
  *out = ctx->stats;
  out->kernel_launches = ctx->B.launches - ctx->stats.kernel_launches;
  return MEB_OK;
}

int meb_reset_stats(meb_ctx* ctx) {
  if (!ctx) return MEB_EINVAL;
  memset(&ctx->stats, 0, sizeof(ctx->stats));
  ctx->stats.kernel_launches = ctx->B.launches;   // baseline
  return MEB_OK;
}

}  // extern "C"

static int resolve_params(meb_ctx* ctx, const meb_params* params, double tol, meb_params* out) {
  meb_params P;
  if (params) P = *params; else meb_params_default(&P);
  if (tol > 0) P.tol = tol;
  if (!(P.tol > 0) || !(P.rho >= 0 && P.rho < 1) || !(P.sigma0 > 0) || !(P.tau > 0) ||
      !(P.sigma_max >= P.sigma0) || !(P.sigma_growth >= 1) || P.max_outer < 1 || P.max_ssn < 1 ||
      P.max_backtrack < 0 || P.max_cg < 1 || P.max_cg > 20000 || !(P.active_theta >= 0) ||
      (P.mixed && (!(P.tol_lp > 0) || !(P.tol_red >= 0) || P.max_readd < 0)))
    return fail(ctx, MEB_EINVAL, "invalid parameters");
  *out = P;
  return MEB_OK;
}

static int64_t tick_cap(const meb_params& P) {
  return (int64_t)P.max_outer * (P.max_ssn + 2) * (P.max_backtrack + 2) + 16;
}

static int check_sizes(meb_ctx* ctx, int64_t m, int32_t d) {
  if (m < 1 || m > (int64_t)2147483647 - 256) return fail(ctx, MEB_EINVAL, "m out of range");
  if (d < 1 || d > 16384) return fail(ctx, MEB_EINVAL, "d out of range");
  return MEB_OK;
}


static int read_state(meb_ctx* ctx, const Buffers& B) {
  CK(cudaMemcpyAsync(ctx->h_st, B.st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx_sync(ctx));
  return MEB_OK;
}

// During the capture of a tick graph on s: append a conditional while node
// (its handle defaults to 1 at every launch, so the body runs at least once)
// whose body, captured on the context's second stream, is one CG iteration
// and k_cg_cond; then continue the capture after the node.
static cudaError_t cg_loop_node(meb_ctx* ctx, Buffers& B, int64_t m, int d, cudaStream_t s) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !graph) return cudaErrorStreamCaptureInvalidated;
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
  memset(npbuf, 0, sizeof(npbuf));
  cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(npbuf);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, dv.empty() ? nullptr : dv.data(), nullptr, dv.size(), np);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = np->conditional.phGraph_out[0];
  cudaStream_t s2 = ctx->stream2;
  e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  e = launch_cg_iter(B, m, d, s2);
  if (e == cudaSuccess) e = launch_cg_cond(B, h, s2);
  cudaGraph_t got = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s2, &got);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Build (or reuse) the tick graph of buffer set B: kUnrollTicks ticks of
// { pass; controller; Newton; multiplier update } (mode 0; the matrix-free
// Newton system as CG setup, a while node of CG iterations and the finish),
// or a while-node running ticks until the controller stops (mode 2, dense).
// Every kernel of the tick is gated on the controller's action, so the tick
// is a fixed sequence.  *out: the cached entry.
static int solve_graph(meb_ctx* ctx, Buffers& B, const double* C, const double* R, int64_t m,
                       int d, bool dense, meb_ctx::TickGraph** out) {
  const int mode = ctx->loop_mode;
  const int prof = ctx->profiling;
  const void* xs = B.use_x16 ? (const void*)B.X16 : (const void*)B.X32;
  for (auto& g : ctx->tg) {
    if (g.gexec && g.key[0] == C && g.key[1] == R && g.key[2] == B.st && g.key[3] == xs &&
        g.key[4] == B.W && g.var == screen_variant(B, d) && g.wait == B.wait_cycles &&
        g.m == m && g.d == d && g.mode == mode && g.prof == prof && g.lowp == (int)B.lowp &&
        g.dense == (int)dense) {
      *out = &g;
      return MEB_OK;
    }
  }
  if (prof && !ctx->gev[0])
    for (int k = 0; k < 16; k++) CK(cudaEventCreate(&ctx->gev[k]));
  meb_ctx::TickGraph& g = ctx->tg[ctx->tg_next];
  ctx->tg_next ^= 1;
  if (g.gexec) { cudaGraphExecDestroy(g.gexec); g.gexec = nullptr; }
  if (g.graph) { cudaGraphDestroy(g.graph); g.graph = nullptr; }
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (mode == 2) {
    CK(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g.graph, 1, cudaGraphCondAssignDefault));
    // cudaGraphNodeParams holds a union without a default constructor: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = h;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, np));
    cudaGraph_t body = np->conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    e = launch_pass(C, R, B, m, d, s);
    if (e == cudaSuccess) e = launch_tick_control(B, m, d, s);
    if (e == cudaSuccess) e = launch_newton_dense(B, d, s);
    if (e == cudaSuccess) e = launch_mult_update(C, B, m, d, s);
    if (e == cudaSuccess) e = launch_loop_cond(B, h, s);
    cudaGraph_t got = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &got);
    if (e != cudaSuccess) return fail(ctx, MEB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    CK(e2);
  } else {
    if (!dense && !ctx->stream2)
      CK(cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    for (int t = 0; t < kUnrollTicks && e == cudaSuccess; t++) {
      // profiling: CUDA events around every k_screen of the batch (event nodes)
      e = prof ? launch_pass(C, R, B, m, d, s, ctx->gev[2 * t], ctx->gev[2 * t + 1], t)
               : launch_pass(C, R, B, m, d, s);
      if (e == cudaSuccess) e = launch_tick_control(B, m, d, s);
      if (dense) {
        if (e == cudaSuccess) e = launch_newton_dense(B, d, s);
      } else {
        // matrix-free Newton system: CG setup, then a conditional while node
        // whose body is one CG iteration and the loop condition, then the
        // finish (each kernel gated on the controller's action)
        if (e == cudaSuccess) e = launch_cg_setup(B, d, s);
        if (e == cudaSuccess) e = cg_loop_node(ctx, B, m, d, s);
        if (e == cudaSuccess) e = launch_cg_finish(B, d, s);
      }
      if (e == cudaSuccess) e = launch_mult_update(C, B, m, d, s);
    }
    cudaError_t e2 = cudaStreamEndCapture(s, &g.graph);
    if (e != cudaSuccess) return fail(ctx, MEB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    CK(e2);
  }
  CK(cudaGraphInstantiate(&g.gexec, g.graph, 0));
  g.key[0] = C; g.key[1] = R; g.key[2] = B.st; g.key[3] = xs; g.key[4] = B.W;
  g.var = screen_variant(B, d);
  g.wait = B.wait_cycles;
  g.m = m; g.d = d; g.mode = mode; g.prof = prof; g.lowp = (int)B.lowp; g.dense = (int)dense;
  *out = &g;
  return MEB_OK;
}

// The input check, the FP32 shadow (origin c_0), the mean centre c0 and
// r0 = max_i ||c0 - c_i|| + r_i (certified feasibility pass at c0).
// With swept = true the shadow blocks have run already (stage_in_shadowed).
static int setup_instance(meb_ctx* ctx, Buffers& B, const double* C, const double* R, int64_t m,
                          int d, double* r0, bool swept = false) {
  cudaStream_t s = ctx->stream;
  if (swept) {
    CK(launch_shadow_mean(C, m, d, B, B.vec.o, B.vec.c0, s));
  } else {
    CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    CK(launch_shadow(C, R, m, d, B, B.vec.o, B.vec.c0, ctx->d_flags, s));
  }
  CK(launch_feas_cert(C, R, m, d, B.vec.c0, 0.0, INFINITY, 2, 1, B, ctx->d_scal, ctx->d_i64,
                      ctx->d_i64 + 1, s));
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  int bad;
  memcpy(&bad, ctx->h_scal + 1, sizeof(int));
  if (bad) return fail(ctx, MEB_EINVAL, "non-finite centre or radius, or negative radius");
  *r0 = ctx->h_scal[0];
  return MEB_OK;
}

// The controller's initial state on buffer set B: multipliers cleared, the
// FP16 shadow at scale sc, x = (r0, c0)/sc.
static int init_state(meb_ctx* ctx, Buffers& B, int64_t m, int d, const meb_params& P, double sc,
                      double r0) {
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(B.slot, 0xff, sizeof(int) * (size_t)m, s));
  CK(prepare_pass(B, d));
  CK(prepare_newton(d));
  if (B.use_x16) CK(launch_shadow16(B, m, d, 1.0 / sc, s));
  state_defaults(*ctx->h_st, m, d, P, sc, (d <= P.dense_max_d && d + 1 <= kMaxDenseN) ? 1 : 0);
  ctx->h_st->sh_s = sc;
  ctx->h_st->sh_inv_s = 1.0 / sc;
  ctx->h_st->rt_abs = r0;   // initial radius; k_state_init scales it
  // FP32 rows (the low-precision run): per-ball terms carry about
  // (d + 16) 2^-24 relative error, of which sums keep about sqrt(d)
  if (B.lowp) ctx->h_st->rnd = FLT_EPSILON * (2.0 + std::sqrt((double)d));
  CK(cudaMemcpyAsync(B.st, ctx->h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(launch_state_init(B, d, s));
  return MEB_OK;
}

// The controller ticks on buffer set B until the controller stops (status in
// ctx->h_st afterwards): graph batches, a while-node graph (dense Newton path),
// or host launches (MEB_OPT_TICK_LOOP = 1, and the while mode on the
// matrix-free path or with profiling).
static int run_ticks(meb_ctx* ctx, Buffers& B, const double* C, const double* R, int64_t m,
                     int d, const meb_params& P) {
  cudaStream_t s = ctx->stream;
  const bool dense = (d <= P.dense_max_d && d + 1 <= kMaxDenseN);
  ctx->prof_screens = 0;
  // per ball: the shadow row (FP16: 16 bytes per 8 coordinates; FP32: 16
  // bytes per 4 coordinates), its error bound, the FP32 radius and the slot
  const int64_t d4 = (d + 3) / 4;
  const int64_t pass_bytes = B.fp64_all ? m * 8   // the slot read and the list written
                                         : m * (B.use_x16 ? 16 * ((d4 + 1) / 2) + 12 : 16 * d4 + 12);
  const int64_t max_ticks = tick_cap(P);
  int rc;
  // graph ticks: batches of kUnrollTicks (both Newton paths), or the while
  // node (dense path, without profiling); otherwise host launches
  const bool graph_ticks =
      ctx->loop_mode == 0 || (ctx->loop_mode == 2 && dense && !ctx->profiling);
  if (graph_ticks) {
    // device-resident ticks: graph launches, one status read per kUnrollTicks ticks
    meb_ctx::TickGraph* g = nullptr;
    rc = solve_graph(ctx, B, C, R, m, d, dense, &g);
    if (rc) return rc;
    const int64_t before = B.launches;
    if (ctx->loop_mode == 2) {
      ctx->h_st->max_ticks = max_ticks < 20000 ? max_ticks : 20000;
      CK(cudaMemcpyAsync(&B.st->max_ticks, &ctx->h_st->max_ticks, sizeof(int64_t),
                         cudaMemcpyHostToDevice, s));
      CK(cudaGraphLaunch(g->gexec, s));
      rc = read_state(ctx, B);
      if (rc) return rc;
      B.launches = before + ctx->h_st->ticks * (tick_launches(d) + 1);
      if (ctx->h_st->status == kStatusTickCap)
        return fail(ctx, MEB_ECUDA, "controller did not terminate");
    } else {
      int64_t ticks = 0;
      for (;;) {
        if (ctx->profiling)
          CK(cudaMemsetAsync(B.st->screen_log, 0, sizeof(B.st->screen_log), s));
        CK(cudaGraphLaunch(g->gexec, s));
        ticks += kUnrollTicks;
        rc = read_state(ctx, B);
        if (rc) return rc;
        if (ctx->profiling) {
          for (int t = 0; t < kUnrollTicks; t++) {
            if (!ctx->h_st->screen_log[t]) continue;
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->gev[2 * t], ctx->gev[2 * t + 1]));
            ctx->stats.pass_ms += ms;
            ctx->stats.pass_launches += 1;
            ctx->stats.pass_balls += m;
            ctx->stats.pass_bytes += pass_bytes;
          }
        }
        if (ctx->h_st->status != 0) break;
        if (ticks > max_ticks) return fail(ctx, MEB_ECUDA, "controller did not terminate");
      }
      // dense: a fixed count per tick; matrix-free: pass, controller, CG
      // setup and finish, multipliers, plus 4 per run of the CG loop body
      B.launches = before + (dense ? ticks * tick_launches(d)
                                   : ticks * (support_rows_wide(B, d) ? 7 : 6) +
                                         4 * ctx->h_st->cg_bodies);
    }
  } else {
    int64_t ticks = 0;
    const bool prof = ctx->profiling != 0;
    cudaEvent_t* pe = ctx->gev;   // phase marks (the graph loop's events are unused here)
    if (prof && !pe[0])
      for (int k = 0; k < 16; k++) CK(cudaEventCreate(&ctx->gev[k]));
    auto phase = [&](int k, int a, int b) -> int {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, pe[a], pe[b]));
      ctx->stats.phase_ms[k] += ms;
      return MEB_OK;
    };
    for (;;) {
      if (prof) CK(cudaEventRecord(pe[10], s));
      CK(launch_pass(C, R, B, m, d, s, ctx->profiling ? ctx->ev[0] : nullptr,
                     ctx->profiling ? ctx->ev[1] : nullptr));
      if (prof) CK(cudaEventRecord(pe[11], s));
      CK(launch_tick_control(B, m, d, s));
      if (prof) CK(cudaEventRecord(pe[12], s));
      rc = read_state(ctx, B);
      if (rc) return rc;
      if (prof && ((rc = phase(0, 10, 11)) || (rc = phase(1, 11, 12)))) return rc;
      if (ctx->profiling && ctx->h_st->screens > ctx->prof_screens) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
        ctx->stats.pass_ms += ms;
        ctx->stats.pass_launches += 1;
        ctx->stats.pass_balls += m;
        ctx->stats.pass_bytes += pass_bytes;
        ctx->stats.pass_fp64_rows += (int64_t)ctx->h_st->last[P_N64];
      }
      ctx->prof_screens = ctx->h_st->screens;
      if (ctx->h_st->status != 0) break;
      if (prof) CK(cudaEventRecord(pe[13], s));
      if (ctx->h_st->action == ACT_NEWTON) {
        if (dense) {
          CK(launch_newton_dense(B, d, s));
        } else {
          CK(launch_cg_setup(B, d, s));
          for (int round = 0; round <= P.max_cg / 4 + 1; round++) {
            for (int k = 0; k < 4; k++) CK(launch_cg_iter(B, m, d, s));
            rc = read_state(ctx, B);
            if (rc) return rc;
            if (ctx->h_st->cg_done || ctx->h_st->status != 0 || ctx->h_st->action != ACT_NEWTON) break;
          }
          CK(launch_cg_finish(B, d, s));
        }
      }
      if (prof) CK(cudaEventRecord(pe[14], s));
      CK(launch_mult_update(C, B, m, d, s));
      if (prof) {
        CK(cudaEventRecord(pe[15], s));
        CK(ctx_sync(ctx));
        if ((rc = phase(2, 13, 14)) || (rc = phase(3, 14, 15))) return rc;
      }
      if (++ticks > max_ticks) return fail(ctx, MEB_ECUDA, "controller did not terminate");
    }
  }
  if (ctx->h_st->status == kStatusWaitTimeout)
    return fail(ctx, MEB_ETIMEOUT, "a device wait timed out (a bulk copy did not complete)");
  return MEB_OK;
}

// The final point, the radius lift (max-type value at c over all m balls,
// Sec. 4.2) and the active set, on the full instance's buffers B.  Fills
// info's radius and active fields; the active list stays in B.viol.
static int finish_solve(meb_ctx* ctx, Buffers& Bx, Buffers& B, const double* C, const double* R,
                        int64_t m, int d, const meb_params& P, double* dcout, double* r_alm_out,
                        double* r_out_out, int64_t* n_active_out) {
  cudaStream_t s = ctx->stream;
  double* d_ralm = ctx->d_scal + 1;
  CK(launch_final_point(Bx, d, dcout, d_ralm, s));
  CK(launch_feas_cert(C, R, m, d, dcout, 0.0, INFINITY, 2, 1, B, ctx->d_scal + 2, ctx->d_i64 + 2,
                      ctx->d_i64 + 3, s));
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  const double r_alm = ctx->h_scal[1];
  const double r_out = ctx->h_scal[2];
  CK(launch_feas_cert(C, R, m, d, dcout, r_out, P.active_theta * r_out, 1, 0, B, nullptr, nullptr,
                      ctx->d_i64 + 5, s, /*reuse_bounds=*/true));
  CK(cudaMemcpyAsync(ctx->h_scal + 8, ctx->d_i64 + 5, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  memcpy(n_active_out, ctx->h_scal + 8, sizeof(int64_t));
  *r_alm_out = r_alm;
  *r_out_out = r_out;
  return MEB_OK;
}

static void fill_info(meb_info* info, const DevState& S, double sc, double r_alm, double r_out,
                      int64_t n_active) {
  if (!info) return;
  info->r = r_out;
  info->r_alm = r_alm;
  info->kkt[0] = S.kkt[0];
  info->kkt[1] = S.kkt[1];
  info->kkt[2] = S.kkt[2] * sc;
  info->kkt[3] = S.kkt[3];
  info->kkt[4] = S.kkt[4] * sc;
  info->kkt_max = S.kkt_max;
  info->delta_max = r_out - r_alm;
  info->scale = sc;
  info->n_active = n_active;
  info->fp64_rows = S.n64_total;
  info->outer_iters = S.outer;
  info->ssn_iters = S.tot_ssn;
  info->cg_iters = S.tot_cg;
  info->passes = S.tot_passes;
  info->backtracks = S.tot_bt;
  info->status = S.status == 1 ? 0 : 1;
  info->newton_inverses = S.gj_inverses;
  info->newton_fp64 = S.fp64_solves;
}

static int solve_mixed(meb_ctx* ctx, const double* C, const double* R, int64_t m, int d,
                       const meb_params& P, double sc, double r0, double* dcout, meb_info* info,
                       int64_t* n_active, DevState* Sout);

extern "C" int meb_solve(meb_ctx* ctx, const double* centers, const double* radii, int64_t m,
                         int32_t d, double tol, const meb_params* params, unsigned flags,
                         double* c_out, int64_t* active_idx, int64_t active_cap,
                         meb_info* info) {
  if (!ctx) return MEB_EINVAL;
  CallScope scope(ctx);
  ctx->err[0] = 0;
  int rc = check_sizes(ctx, m, d);
  if (rc) return rc;
  if (!centers || !radii || !c_out || (active_cap > 0 && !active_idx) || active_cap < 0)
    return fail(ctx, MEB_EINVAL, "NULL argument");
  meb_params P;
  rc = resolve_params(ctx, params, tol, &P);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  rc = ensure_buffers(ctx, m, d);
  if (rc) return rc;
  Buffers& B = ctx->B;
  const double* C;
  const double* R;
  const bool swept = stage_chunked(flags, m, d);
  if (swept) {
    rc = stage_in_shadowed(ctx, B, centers, radii, m, d, &C, &R);
    if (rc) return rc;
  } else {
    rc = stage_in(ctx, POOL_C, centers, sizeof(double) * (size_t)m * d, flags, (const void**)&C);
    if (rc) return rc;
    rc = stage_in(ctx, POOL_R, radii, sizeof(double) * (size_t)m, flags, (const void**)&R);
    if (rc) return rc;
  }
  B.C_in = C;
  ctx->mult_kind = 0;
  B.use_x16 = ctx->screen_mode == MEB_SCREEN_FP16 || ctx->screen_mode == MEB_SCREEN_FP16_BULK;
  B.bulk = ctx->screen_mode == MEB_SCREEN_FP16_BULK;
  B.fp64_all = ctx->screen_mode == MEB_SCREEN_FP64;
  B.lowp = false;
  B.wait_cycles = ctx->wait_cycles;
  if (info) memset(info, 0, sizeof(*info));

  // the input check, the FP32 shadow and r0 at the mean centre
  double r0 = 0.0;
  rc = setup_instance(ctx, B, C, R, m, d, &r0, swept);
  if (rc) return rc;
  void* dcout = nullptr;
  if (flags & MEB_PTR_DEVICE) dcout = c_out;
  else { rc = pool(ctx, POOL_COUT, sizeof(double) * (size_t)d, &dcout); if (rc) return rc; }

  if (m == 1 || r0 == 0.0) {
    // one ball, or every ball the same point: the answer is that ball
    CK(cudaMemcpyAsync(dcout, m == 1 ? C : B.vec.c0, sizeof(double) * d,
                       cudaMemcpyDeviceToDevice, s));
    if (!(flags & MEB_PTR_DEVICE))
      CK(cudaMemcpyAsync(c_out, dcout, sizeof(double) * d, cudaMemcpyDeviceToHost, s));
    CK(ctx_sync(ctx));
    const double r = (m == 1) ? r0 : 0.0;
    const int64_t na = m;
    const int64_t nw = std::min(active_cap, na);
    if (flags & MEB_PTR_DEVICE) {
      if (nw > 0) {
        std::vector<int64_t> seq(nw);
        for (int64_t k = 0; k < nw; k++) seq[k] = k;
        CK(cudaMemcpyAsync(active_idx, seq.data(), sizeof(int64_t) * (size_t)nw,
                           cudaMemcpyHostToDevice, s));
        CK(ctx_sync(ctx));
      }
    } else {
      for (int64_t k = 0; k < nw; k++) active_idx[k] = k;
    }
    if (info) {
      info->r = r; info->r_alm = r; info->scale = 1.0; info->n_active = na; info->status = 0;
      info->n_reduced = m;
    }
    ctx->mult_kind = (m == 1) ? 2 : 3;
    ctx->mult_n = m;
    ctx->mult_m = m;
    ctx->mult_d = d;
    return MEB_OK;
  }

  int ex;
  frexp(r0, &ex);
  double sc = ldexp(1.0, ex);
  if (sc / 2.0 >= r0) sc /= 2.0;
  int64_t n_active = 0;
  DevState S;
  if (P.mixed) {
    // Sec. 4.2: low-precision run, screening, FP64 on the reduced set, re-adds
    rc = solve_mixed(ctx, C, R, m, d, P, sc, r0, (double*)dcout, info, &n_active, &S);
    if (rc) return rc;
  } else {
    rc = init_state(ctx, B, m, d, P, sc, r0);
    if (rc) return rc;
    rc = run_ticks(ctx, B, C, R, m, d, P);
    if (rc) return rc;
    S = *ctx->h_st;
    ctx->mult_kind = 1;
    ctx->mult_n = S.nS;
    ctx->mult_m = m;
    ctx->mult_d = d;
    double r_alm, r_out;
    rc = finish_solve(ctx, B, B, C, R, m, d, P, (double*)dcout, &r_alm, &r_out, &n_active);
    if (rc) return rc;
    fill_info(info, S, sc, r_alm, r_out, n_active);
    if (info) info->n_reduced = m;
  }
  if (!(flags & MEB_PTR_DEVICE))
    CK(cudaMemcpyAsync(c_out, dcout, sizeof(double) * d, cudaMemcpyDeviceToHost, s));
  const int64_t ncp = n_active < active_cap ? n_active : active_cap;
  if (ncp > 0) {
    rc = copy_out(ctx, active_idx, B.viol, sizeof(int64_t) * (size_t)ncp, flags);
    if (rc) return rc;
  }
  CK(ctx_sync(ctx));
  return S.status == 1 ? MEB_OK : fail(ctx, MEB_ENOTCONV, "iteration cap reached");
}

extern "C" int meb_eval_alm(meb_ctx* ctx, const double* centers, const double* radii, int64_t m,
                            int32_t d, const double* x, const double* xbar, const double* U,
                            const double* V, double sigma, double tau, const double* q,
                            unsigned flags, double* psi, double* grad, double* Uplus,
                            double* Vplus, double* Hq, double* H, int64_t* case_counts) {
  if (!ctx) return MEB_EINVAL;
  CallScope scope(ctx);
  ctx->err[0] = 0;
  int rc = check_sizes(ctx, m, d);
  if (rc) return rc;
  if (!centers || !radii || !x || !xbar || !U || !V)
    return fail(ctx, MEB_EINVAL, "NULL argument");
  if ((Uplus == nullptr) != (Vplus == nullptr))
    return fail(ctx, MEB_EINVAL, "Uplus and Vplus must both be given or both be NULL");
  if ((Hq != nullptr) && q == nullptr) return fail(ctx, MEB_EINVAL, "Hq needs q");
  if (H && d + 1 > kMaxDenseN) return fail(ctx, MEB_EINVAL, "dense H output needs d <= 224");
  if (!(sigma > 0) || !(tau > 0) || !isfinite(sigma) || !isfinite(tau))
    return fail(ctx, MEB_EINVAL, "sigma and tau must be positive");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  rc = ensure_buffers(ctx, m, d);
  if (rc) return rc;
  Buffers& B = ctx->B;
  const size_t n1b = sizeof(double) * (size_t)(d + 1);
  const double *C, *R, *dx, *dxb, *dU, *dV, *dq = nullptr;
  if ((rc = stage_in(ctx, POOL_C, centers, sizeof(double) * (size_t)m * d, flags, (const void**)&C))) return rc;
  if ((rc = stage_in(ctx, POOL_R, radii, sizeof(double) * (size_t)m, flags, (const void**)&R))) return rc;
  if ((rc = stage_in(ctx, POOL_X, x, n1b, flags, (const void**)&dx))) return rc;
  if ((rc = stage_in(ctx, POOL_XB, xbar, n1b, flags, (const void**)&dxb))) return rc;
  if ((rc = stage_in(ctx, POOL_U, U, sizeof(double) * (size_t)m, flags, (const void**)&dU))) return rc;
  if ((rc = stage_in(ctx, POOL_V, V, sizeof(double) * (size_t)m * d, flags, (const void**)&dV))) return rc;
  if (q && (rc = stage_in(ctx, POOL_Q, q, n1b, flags, (const void**)&dq))) return rc;
  B.C_in = C;
  ctx->mult_kind = 0;
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
  CK(launch_shadow(C, R, m, d, B, B.vec.o, B.vec.c0, ctx->d_flags, s));
  CK(cudaMemsetAsync(B.slot, 0xff, sizeof(int) * (size_t)m, s));
  // the evaluation is of the unscaled problem (s = 1); an FP16 screen reads
  // the shadow of the data divided by sh = 2^eval_shadow_exp
  B.use_x16 = ctx->eval_screen == MEB_SCREEN_FP16 || ctx->eval_screen == MEB_SCREEN_FP16_BULK;
  B.bulk = ctx->eval_screen == MEB_SCREEN_FP16_BULK;
  B.fp64_all = ctx->eval_screen == MEB_SCREEN_FP64;
  B.wait_cycles = ctx->wait_cycles;
  const double sh = ldexp(1.0, ctx->eval_shadow_exp);
  if (B.use_x16) CK(launch_shadow16(B, m, d, 1.0 / sh, s));
  CK(prepare_pass(B, d));
  meb_params P;
  meb_params_default(&P);
  P.sigma0 = sigma;
  P.sigma_max = sigma;
  P.tau = tau;
  state_defaults(*ctx->h_st, m, d, P, 1.0, (d <= P.dense_max_d && d + 1 <= kMaxDenseN) ? 1 : 0);
  ctx->h_st->sh_s = sh;
  ctx->h_st->sh_inv_s = 1.0 / sh;
  ctx->h_st->eval_only = 1;
  CK(cudaMemcpyAsync(B.st, ctx->h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(launch_support_from_dense(dU, dV, B, m, d, s));
  CK(launch_eval_prepare(B, dx, dxb, d, s));
  CK(launch_pass(C, R, B, m, d, s));
  CK(launch_tick_control(B, m, d, s));
  double *dUp = nullptr, *dVp = nullptr, *dHq = nullptr, *dH = nullptr;
  if (Uplus) {
    if (flags & MEB_PTR_DEVICE) { dUp = Uplus; dVp = Vplus; }
    else {
      if ((rc = pool(ctx, POOL_UP, sizeof(double) * (size_t)m, (void**)&dUp))) return rc;
      if ((rc = pool(ctx, POOL_VP, sizeof(double) * (size_t)m * d, (void**)&dVp))) return rc;
    }
  }
  if (Hq) {
    if (flags & MEB_PTR_DEVICE) dHq = Hq;
    else if ((rc = pool(ctx, POOL_HQ, n1b, (void**)&dHq))) return rc;
  }
  if (H) {
    if (flags & MEB_PTR_DEVICE) dH = H;
    else if ((rc = pool(ctx, POOL_H, n1b * (d + 1), (void**)&dH))) return rc;
  }
  CK(launch_eval_outputs(C, B, m, d, dq, dUp, dVp, dHq, dH, s));
  if (grad && (rc = copy_out(ctx, grad, B.vec.gt, n1b, flags))) return rc;
  if (Uplus && !(flags & MEB_PTR_DEVICE)) {
    if ((rc = copy_out(ctx, Uplus, dUp, sizeof(double) * (size_t)m, flags))) return rc;
    if ((rc = copy_out(ctx, Vplus, dVp, sizeof(double) * (size_t)m * d, flags))) return rc;
  }
  if (Hq && !(flags & MEB_PTR_DEVICE) && (rc = copy_out(ctx, Hq, dHq, n1b, flags))) return rc;
  if (H && !(flags & MEB_PTR_DEVICE) && (rc = copy_out(ctx, H, dH, n1b * (d + 1), flags))) return rc;
  CK(cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  rc = read_state(ctx, ctx->B);
  if (rc) return rc;
  int bad;
  memcpy(&bad, ctx->h_scal + 1, sizeof(int));
  if (bad) return fail(ctx, MEB_EINVAL, "non-finite centre or radius, or negative radius");
  if (psi) *psi = ctx->h_st->psi;
  if (case_counts) {
    const int64_t nI = (int64_t)ctx->h_st->last[P_NI], nM = (int64_t)ctx->h_st->last[P_NM];
    case_counts[0] = m - nI - nM;
    case_counts[1] = nI;
    case_counts[2] = nM;
  }
  return MEB_OK;
}

extern "C" int meb_feas_check(meb_ctx* ctx, const double* centers, const double* radii,
                              int64_t m, int32_t d, const double* c, double r, double eps,
                              unsigned flags, double* delta_max, int64_t* argmax,
                              int64_t* viol_idx, int64_t viol_cap, int64_t* n_viol) {
  if (!ctx) return MEB_EINVAL;
  CallScope scope(ctx);
  ctx->err[0] = 0;
  int rc = check_sizes(ctx, m, d);
  if (rc) return rc;
  if (!centers || !radii || !c || (viol_cap > 0 && !viol_idx) || viol_cap < 0)
    return fail(ctx, MEB_EINVAL, "NULL argument");
  if (!isfinite(r) || isnan(eps)) return fail(ctx, MEB_EINVAL, "r must be finite");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  rc = ensure_buffers(ctx, m, d);
  if (rc) return rc;
  Buffers& B = ctx->B;
  ctx->mult_kind = 0;
  B.fp64_all = ctx->eval_screen == MEB_SCREEN_FP64;
  const double *C, *R, *dc;
  if ((rc = stage_in(ctx, POOL_C, centers, sizeof(double) * (size_t)m * d, flags, (const void**)&C))) return rc;
  if ((rc = stage_in(ctx, POOL_R, radii, sizeof(double) * (size_t)m, flags, (const void**)&R))) return rc;
  if ((rc = stage_in(ctx, POOL_X, c, sizeof(double) * (size_t)d, flags, (const void**)&dc))) return rc;
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
  CK(launch_shadow(C, R, m, d, B, B.vec.o, B.vec.c0, ctx->d_flags, s));
  CK(launch_feas_cert(C, R, m, d, dc, r, eps, 0, 1, B, ctx->d_scal, ctx->d_i64, ctx->d_i64 + 1, s,
                      false, ctx->d_flags));
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_i64, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_scal + 3, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  int bad;
  memcpy(&bad, ctx->h_scal + 3, sizeof(int));
  if (bad) return fail(ctx, MEB_EINVAL, "non-finite centre, radius or query, or negative radius");
  int64_t am, nv;
  memcpy(&am, ctx->h_scal + 1, sizeof(int64_t));
  memcpy(&nv, ctx->h_scal + 2, sizeof(int64_t));
  if (delta_max) *delta_max = ctx->h_scal[0];
  if (argmax) *argmax = am;
  if (n_viol) *n_viol = nv;
  const int64_t ncp = nv < viol_cap ? nv : viol_cap;
  if (ncp > 0) {
    rc = copy_out(ctx, viol_idx, B.viol, sizeof(int64_t) * (size_t)ncp, flags);
    if (rc) return rc;
    CK(ctx_sync(ctx));
  }
  return MEB_OK;
}


extern "C" int meb_get_multipliers(meb_ctx* ctx, unsigned flags, int64_t* idx, double* u,
                                   double* v, int64_t cap, int64_t* n_sup) {
  if (!ctx) return MEB_EINVAL;
  CallScope scope(ctx);
  if (!n_sup || cap < 0 || (cap > 0 && (!idx || !u || !v)))
    return fail(ctx, MEB_EINVAL, "NULL argument");
  if (ctx->mult_kind == 0) return fail(ctx, MEB_EINVAL, "no solve to report multipliers of");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->mult_n;
  const int d = ctx->mult_d;
  *n_sup = n;
  const int64_t k = n < cap ? n : cap;
  if (k == 0) return MEB_OK;
  const bool dev = (flags & MEB_PTR_DEVICE) != 0;
  if (ctx->mult_kind == 1 || ctx->mult_kind == 4) {
    Buffers& Bs = ctx->mult_kind == 4 ? ctx->Bred : ctx->B;
    int64_t* didx;
    double *du, *dv;
    int rc;
    if (dev) { didx = idx; du = u; dv = v; }
    else {
      if ((rc = pool(ctx, POOL_ACT, sizeof(int64_t) * (size_t)k, (void**)&didx))) return rc;
      if ((rc = pool(ctx, POOL_UP, sizeof(double) * (size_t)k, (void**)&du))) return rc;
      if ((rc = pool(ctx, POOL_VP, sizeof(double) * (size_t)k * d, (void**)&dv))) return rc;
    }
    CK(launch_mult_out(Bs, d, didx, du, dv, k, s));
    if (ctx->mult_kind == 4) CK(launch_map_idx(didx, k, ctx->mult_map, s));
    if (!dev) {
      CK(cudaMemcpyAsync(idx, didx, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(u, du, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(v, dv, sizeof(double) * (size_t)k * d, cudaMemcpyDeviceToHost, s));
    }
    CK(ctx_sync(ctx));
    return MEB_OK;
  }
  // one ball (u = 1) or every ball the same point (u = 1/m); v = 0
  const double uval = ctx->mult_kind == 2 ? 1.0 : 1.0 / (double)ctx->mult_m;
  if (dev) {
    int64_t* hi = nullptr;
    double* hu = nullptr;
    CK(cudaMallocHost((void**)&hi, sizeof(int64_t) * (size_t)k));
    CK(cudaMallocHost((void**)&hu, sizeof(double) * (size_t)k));
    for (int64_t t = 0; t < k; t++) { hi[t] = t; hu[t] = uval; }
    cudaError_t e = cudaMemcpyAsync(idx, hi, sizeof(int64_t) * (size_t)k, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, hu, sizeof(double) * (size_t)k, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(double) * (size_t)k * d, s);
    if (e == cudaSuccess) e = ctx_sync(ctx);
    cudaFreeHost(hi);
    cudaFreeHost(hu);
    CK(e);
  } else {
    for (int64_t t = 0; t < k; t++) { idx[t] = t; u[t] = uval; }
    memset(v, 0, sizeof(double) * (size_t)k * d);
  }
  return MEB_OK;
}

// ===========================================================================
// Batched solver (meb_solve_batch, meb_tune_batch).

static int batch_class(int d) { return d <= 4 ? 0 : d <= 16 ? 1 : d <= 64 ? 2 : d <= 128 ? 3 : 4; }
static const int kBatchMaxD = 4096;

static bool batch_item_ok(const meb_batch_item& it) {
  return it.m >= 1 && it.m <= (int64_t)2147483647 - 256 && it.d >= 1 && it.d <= kBatchMaxD &&
         it.centers && it.radii && it.c_out && it.active_cap >= 0 &&
         (it.active_cap == 0 || it.active_idx);
}

// Device views of the valid items (host arrays are copied into the context's
// input arena, and their outputs get room in the output arena).
static int batch_stage(meb_ctx* ctx, int32_t n, const meb_batch_item* items, unsigned flags,
                       std::vector<BatchItemDev>* dev, std::vector<int>* idx) {
  cudaStream_t s = ctx->stream;
  dev->clear();
  idx->clear();
  size_t in_bytes = 0, out_bytes = 0;
  for (int k = 0; k < n; k++) {
    if (!batch_item_ok(items[k])) continue;
    idx->push_back(k);
    in_bytes += sizeof(double) * (size_t)items[k].m * (items[k].d + 1);
    out_bytes += sizeof(double) * (size_t)items[k].d + sizeof(int64_t) * (size_t)items[k].active_cap;
  }
  char *inb = nullptr, *outb = nullptr;
  const bool host = !(flags & MEB_PTR_DEVICE);
  if (host && !idx->empty()) {
    int rc;
    if ((rc = pool(ctx, POOL_BIN, in_bytes, (void**)&inb))) return rc;
    if ((rc = pool(ctx, POOL_BOUT, out_bytes + 16, (void**)&outb))) return rc;
  }
  size_t io = 0, oo = 0;
  for (int k : *idx) {
    const meb_batch_item& it = items[k];
    BatchItemDev b{};
    b.m = it.m;
    b.d = it.d;
    b.cfg = batch_class(it.d);
    b.act_cap = it.active_cap;
    b.sup_cap = batch_support_cap(it.m, it.d);
    if (host) {
      const size_t cb = sizeof(double) * (size_t)it.m * it.d, rb = sizeof(double) * (size_t)it.m;
      CK(cudaMemcpyAsync(inb + io, it.centers, cb, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(inb + io + cb, it.radii, rb, cudaMemcpyHostToDevice, s));
      b.C = reinterpret_cast<const double*>(inb + io);
      b.R = reinterpret_cast<const double*>(inb + io + cb);
      io += cb + rb;
      b.c_out = reinterpret_cast<double*>(outb + oo);
      oo += sizeof(double) * (size_t)it.d;
      b.act = it.active_cap ? reinterpret_cast<int64_t*>(outb + oo) : nullptr;
      oo += sizeof(int64_t) * (size_t)it.active_cap;
    } else {
      b.C = it.centers;
      b.R = it.radii;
      b.c_out = it.c_out;
      b.act = it.active_idx;
    }
    dev->push_back(b);
  }
  return MEB_OK;
}

// One launch of the batch kernel over `items` (device views) with the
// configuration table `cfg`; results in items' order.  *ms: the launch's
// device time.
static int batch_run(meb_ctx* ctx, const std::vector<BatchItemDev>& items, const BatchConfig* cfg,
                     const meb_params& P, std::vector<BatchOut>* outs, float* ms) {
  cudaStream_t s = ctx->stream;
  const int n = (int)items.size();
  outs->assign(n, BatchOut{});
  if (n == 0) return MEB_OK;
  // largest first (the queue order), ties by position
  std::vector<int> order(n);
  for (int k = 0; k < n; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return items[a].m * (double)(items[a].d + 12) > items[b].m * (double)(items[b].d + 12);
  });
  int64_t m_max = 1, sup_max = 1;
  int d_max = 1;
  for (const auto& it : items) {
    m_max = std::max(m_max, it.m);
    d_max = std::max(d_max, it.d);
    sup_max = std::max(sup_max, it.sup_cap);
  }
  const size_t smem = batch_smem(d_max);
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int per_sm = std::max(1, batch_blocks_per_sm(smem));
  const bool per_item = ctx->batch_per_item;
  // shared slots: one per resident block, each sized for the largest
  // instance; per-item slots: one per instance, each sized for it
  const int nslots = per_item ? n : std::min(n, std::max(1, sms * per_sm));
  std::vector<size_t> soff(nslots + 1, 0);
  for (int k = 0; k < nslots; k++) {
    const BatchItemDev& it = items[order[k]];
    soff[k + 1] = soff[k] + (per_item ? batch_slot_layout(nullptr, nullptr, it.m, it.d, it.sup_cap)
                                      : batch_slot_layout(nullptr, nullptr, m_max, d_max, sup_max));
  }
  char* arena = nullptr;
  int rc;
  if ((rc = pool(ctx, POOL_BSLOTS, soff[nslots], (void**)&arena))) return rc;
  std::vector<Buffers> hb(nslots);
  for (int k = 0; k < nslots; k++) {
    const BatchItemDev& it = items[order[k]];
    if (per_item) batch_slot_layout(&hb[k], arena + soff[k], it.m, it.d, it.sup_cap);
    else batch_slot_layout(&hb[k], arena + soff[k], m_max, d_max, sup_max);
  }
  Buffers* dslots = nullptr;
  BatchItemDev* ditems = nullptr;
  BatchOut* dout = nullptr;
  BatchConfig* dcfg = nullptr;
  if ((rc = pool(ctx, POOL_BSLOTB, sizeof(Buffers) * nslots, (void**)&dslots))) return rc;
  if ((rc = pool(ctx, POOL_BITEMS, sizeof(BatchItemDev) * n, (void**)&ditems))) return rc;
  if ((rc = pool(ctx, POOL_BRES, sizeof(BatchOut) * n, (void**)&dout))) return rc;
  if ((rc = pool(ctx, POOL_BCFG, sizeof(BatchConfig) * MEB_BATCH_CLASSES, (void**)&dcfg))) return rc;
  std::vector<BatchItemDev> qi(n);
  for (int k = 0; k < n; k++) qi[k] = items[order[k]];
  CK(cudaMemcpyAsync(dslots, hb.data(), sizeof(Buffers) * nslots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ditems, qi.data(), sizeof(BatchItemDev) * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dcfg, cfg, sizeof(BatchConfig) * MEB_BATCH_CLASSES, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ctx->d_flags + 1, 0, sizeof(int), s));
  BatchArgs G;
  G.items = ditems;
  G.out = dout;
  G.n = n;
  G.next = ctx->d_flags + 1;
  G.slots = dslots;
  G.cfg = dcfg;
  G.P = P;
  G.max_ticks = tick_cap(P);
  G.per_item = per_item ? 1 : 0;
  if (ms && !ctx->ev[0]) {
    CK(cudaEventCreate(&ctx->ev[0]));
    CK(cudaEventCreate(&ctx->ev[1]));
  }
  if (ms) CK(cudaEventRecord(ctx->ev[0], s));
  CK(launch_batch(G, nslots, smem, s));
  ctx->B.launches += 1;
  if (ms) CK(cudaEventRecord(ctx->ev[1], s));
  std::vector<BatchOut> qo(n);
  CK(cudaMemcpyAsync(qo.data(), dout, sizeof(BatchOut) * n, cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  if (ms) CK(cudaEventElapsedTime(ms, ctx->ev[0], ctx->ev[1]));
  for (int k = 0; k < n; k++) (*outs)[order[k]] = qo[k];
  return MEB_OK;
}

static void batch_info(const BatchOut& o, meb_info* info) {
  memset(info, 0, sizeof(*info));
  info->r = o.r;
  info->r_alm = o.r_alm;
  for (int k = 0; k < 5; k++) info->kkt[k] = o.kkt[k];
  info->kkt_max = o.kkt_max;
  info->delta_max = o.r - o.r_alm;
  info->scale = o.scale;
  info->n_active = o.n_active;
  info->fp64_rows = o.fp64_rows;
  info->outer_iters = o.outer;
  info->ssn_iters = o.ssn;
  info->cg_iters = o.cg;
  info->passes = o.passes;
  info->backtracks = o.backtracks;
  info->status = o.status;
  info->newton_inverses = o.inverses;
  info->newton_fp64 = o.fp64_solves;
}

extern "C" int meb_solve_batch(meb_ctx* ctx, int32_t n, const meb_batch_item* items, double tol,
                               const meb_params* params, unsigned flags, meb_info* infos) {
  if (!ctx) return MEB_EINVAL;
  CallScope scope(ctx);
  ctx->err[0] = 0;
  if (n < 0 || (n > 0 && !items)) return fail(ctx, MEB_EINVAL, "NULL argument");
  meb_params P;
  int rc = resolve_params(ctx, params, tol, &P);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  ctx->mult_kind = 0;
  if (infos)
    for (int k = 0; k < n; k++) {
      memset(&infos[k], 0, sizeof(meb_info));
      infos[k].status = -1;
    }
  std::vector<BatchItemDev> dev;
  std::vector<int> idx;
  if ((rc = batch_stage(ctx, n, items, flags, &dev, &idx))) return rc;
  std::vector<BatchOut> outs;
  if ((rc = batch_run(ctx, dev, ctx->batch_cfg, P, &outs, nullptr))) return rc;
  bool bad = (int)idx.size() < n, notconv = false;
  for (size_t q = 0; q < idx.size(); q++) {
    const int k = idx[q];
    const BatchItemDev& b = dev[q];
    BatchOut& o = outs[q];
    meb_info info;
    memset(&info, 0, sizeof(info));
    if (o.status == -1) {
      bad = true;
      info.status = -1;
    } else if (o.status == kStatusSupportCap || o.status == kStatusTickCap) {
      // the support outgrew the block's rows: the multi-block path, in place
      const int r2 = meb_solve(ctx, b.C, b.R, b.m, b.d, P.tol, &P, MEB_PTR_DEVICE, b.c_out, b.act,
                               b.act_cap, &info);
      ctx->stats.batch_fallbacks += 1;
      if (r2 == MEB_ENOTCONV) notconv = true;
      else if (r2 != MEB_OK) return r2;
    } else {
      batch_info(o, &info);
      if (o.status != 0) notconv = true;
    }
    if (infos) infos[k] = info;
    if (!(flags & MEB_PTR_DEVICE) && info.status >= 0) {
      const meb_batch_item& it = items[k];
      CK(cudaMemcpyAsync(it.c_out, b.c_out, sizeof(double) * (size_t)b.d, cudaMemcpyDeviceToHost, s));
      const int64_t na = std::min<int64_t>(info.n_active, it.active_cap);
      if (na > 0)
        CK(cudaMemcpyAsync(it.active_idx, b.act, sizeof(int64_t) * (size_t)na, cudaMemcpyDeviceToHost, s));
    }
  }
  CK(ctx_sync(ctx));
  ctx->stats.batch_instances += (int64_t)idx.size();
  if (bad) return fail(ctx, MEB_EINVAL, "invalid instance in the batch (its info has status -1)");
  if (notconv) return fail(ctx, MEB_ENOTCONV, "iteration cap reached by an instance");
  return MEB_OK;
}

extern "C" int meb_tune_batch(meb_ctx* ctx, int32_t n, const meb_batch_item* items,
                              int32_t per_class, unsigned flags, int32_t* configs) {
  if (!ctx) return MEB_EINVAL;
  CallScope scope(ctx);
  ctx->err[0] = 0;
  if (n < 0 || (n > 0 && !items) || per_class < 1) return fail(ctx, MEB_EINVAL, "bad argument");
  CK(cudaSetDevice(ctx->device));
  meb_params P;
  meb_params_default(&P);
  std::vector<BatchItemDev> dev;
  std::vector<int> idx;
  int rc = batch_stage(ctx, n, items, flags, &dev, &idx);
  if (rc) return rc;
  // candidates: shadow precision (vector width), balls per pass block, and
  // the blocks of the support-row reduction
  const BatchConfig cands[] = {{1, 2, 1, 0}, {1, 16, 8, 0}, {1, 2, 8, 0}, {1, 16, 1, 0},
                               {0, 2, 1, 0}, {0, 16, 8, 0}, {0, 2, 8, 0}, {0, 16, 1, 0}};
  for (int c = 0; c < MEB_BATCH_CLASSES; c++) {
    std::vector<BatchItemDev> sample;
    for (const auto& b : dev)
      if (b.cfg == c && (int)sample.size() < per_class) sample.push_back(b);
    if (sample.empty()) continue;
    float best = INFINITY;
    BatchConfig pick = ctx->batch_cfg[c];
    for (const BatchConfig& cand : cands) {
      BatchConfig table[MEB_BATCH_CLASSES];
      memcpy(table, ctx->batch_cfg, sizeof(table));
      table[c] = cand;
      std::vector<BatchOut> outs;
      float ms = 0.f;
      if ((rc = batch_run(ctx, sample, table, P, &outs, nullptr))) return rc;   // warm-up
      if ((rc = batch_run(ctx, sample, table, P, &outs, &ms))) return rc;
      bool ok = true;
      for (const auto& o : outs) ok = ok && (o.status == 0);
      if (ok && ms < best) { best = ms; pick = cand; }
    }
    ctx->batch_cfg[c] = pick;
  }
  if (configs) {
    for (int c = 0; c < MEB_BATCH_CLASSES; c++) {
      configs[3 * c] = ctx->batch_cfg[c].half;
      configs[3 * c + 1] = ctx->batch_cfg[c].tiles_per_vb;
      configs[3 * c + 2] = ctx->batch_cfg[c].nsvb;
    }
    configs[3 * MEB_BATCH_CLASSES] = 1;
  }
  return MEB_OK;
}

extern "C" int meb_footprint(int64_t m, int32_t d, int32_t path, int64_t* bytes) {
  if (!bytes || m < 1 || m > (int64_t)2147483647 - 256 || d < 1 || d > 16384 || path < 0 ||
      path > 1)
    return MEB_EINVAL;
  if (path == 1 && d > kBatchMaxD) return MEB_EINVAL;
  *bytes = path == 0 ? (int64_t)solve_layout(nullptr, nullptr, m, d)
                     : (int64_t)batch_slot_layout(nullptr, nullptr, m, d, batch_support_cap(m, d));
  return MEB_OK;
}

// ===========================================================================
// The mixed-precision reduction pipeline of Sec. 4.2.

// Buffers of the reduced instance (n balls): re-laid out in place when the
// arena is large enough, else reallocated.
static int ensure_red(meb_ctx* ctx, int64_t n, int d) {
  const size_t bytes = solve_layout(nullptr, nullptr, n, d);
  if (!ctx->red_arena || ctx->red_bytes < bytes) {
    dev_free(ctx, ctx->red_arena);
    ctx->red_arena = nullptr;
    ctx->red_bytes = 0;
    drop_graphs(ctx);
    CK(dev_alloc(ctx, &ctx->red_arena, bytes));
    ctx->red_bytes = bytes;
  }
  solve_layout(&ctx->Bred, (char*)ctx->red_arena, n, d);
  const int n1 = d + 1, d4 = (d + 3) / 4;
  const size_t nv = 20 * (size_t)((n1 + 8 + 1) / 2) * 2 + (size_t)(d4 * 4 + 8);
  CK(cudaMemsetAsync(ctx->Bred.vec_store, 0, sizeof(double) * nv, ctx->stream));
  return MEB_OK;
}

// Sorted union of two ascending index lists.
static std::vector<int64_t> merge_sorted(const std::vector<int64_t>& a, const std::vector<int64_t>& b) {
  std::vector<int64_t> out;
  out.reserve(a.size() + b.size());
  std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
  return out;
}

// The warm start's source: the point x (scaled), the penalty, and the
// multipliers of the last accepted point of buffer set Bs (map: its ball
// indices in the full instance, or null when they already are), into the
// warm pools.  Returns their count in *nw.
static int save_warm(meb_ctx* ctx, Buffers& Bs, int d, const DevState& S, const int64_t* map,
                     int64_t* nw, std::vector<int64_t>* host_idx) {
  cudaStream_t s = ctx->stream;
  const int64_t n = S.nS;
  int64_t* widx;
  double *wu, *wv, *wx;
  int rc;
  if ((rc = pool(ctx, POOL_WIDX, sizeof(int64_t) * (size_t)(n + 1), (void**)&widx))) return rc;
  if ((rc = pool(ctx, POOL_WU, sizeof(double) * (size_t)(n + 1), (void**)&wu))) return rc;
  if ((rc = pool(ctx, POOL_WV, sizeof(double) * (size_t)(n + 1) * d, (void**)&wv))) return rc;
  if ((rc = pool(ctx, POOL_WX, sizeof(double) * (size_t)(d + 1), (void**)&wx))) return rc;
  if (n > 0) {
    CK(launch_mult_out(Bs, d, widx, wu, wv, n, s));
    if (map) CK(launch_map_idx(widx, n, map, s));
  }
  CK(cudaMemcpyAsync(wx, Bs.vec.x, sizeof(double) * (size_t)(d + 1), cudaMemcpyDeviceToDevice, s));
  host_idx->resize(n);
  if (n > 0)
    CK(cudaMemcpyAsync(host_idx->data(), widx, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  *nw = n;
  return MEB_OK;
}

static int solve_mixed(meb_ctx* ctx, const double* C, const double* R, int64_t m, int d,
                       const meb_params& P, double sc, double r0, double* dcout, meb_info* info,
                       int64_t* n_active, DevState* Sout) {
  cudaStream_t s = ctx->stream;
  Buffers& B = ctx->B;
  int rc;
  // 1. the low-precision ripALM on all balls, to tol_lp
  // (its FP32 rows resolve u = sigma Pi(z) to about sigma 2^-24: the penalty
  // stays at most 1e4, so that floor stays below tol_lp; it is a warm start,
  // so at most 50 outer steps)
  meb_params P1 = P;
  P1.tol = P.tol_lp;
  P1.sigma_max = std::min(P.sigma_max, std::max(P.sigma0, 1e4));
  P1.max_outer = std::min(P.max_outer, 50);
  B.lowp = true;
  rc = init_state(ctx, B, m, d, P1, sc, r0);
  if (rc == MEB_OK) rc = run_ticks(ctx, B, C, R, m, d, P1);
  B.lowp = false;
  if (rc) return rc;
  const DevState S1 = *ctx->h_st;
  // 2. screening at the low-precision point: I_red = {slack <= tol_red r_hat}
  //    (certified bounds, FP64 where they do not decide) plus every ball with
  //    a multiplier
  CK(launch_final_point(B, d, dcout, ctx->d_scal + 1, s));
  CK(cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  const double r_hat = ctx->h_scal[1];
  const double fac = P.tol_red > 0 ? P.tol_red : std::max(10.0 * S1.kkt_max, 1e-3);
  CK(launch_feas_cert(C, R, m, d, dcout, r_hat, fac * r_hat, 1, 0, B, nullptr, nullptr,
                      ctx->d_i64 + 6, s));
  int64_t n_scr = 0;
  CK(cudaMemcpyAsync(&n_scr, ctx->d_i64 + 6, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(ctx_sync(ctx));
  std::vector<int64_t> scr(n_scr);
  if (n_scr > 0)
    CK(cudaMemcpyAsync(scr.data(), B.viol, sizeof(int64_t) * (size_t)n_scr, cudaMemcpyDeviceToHost, s));
  int64_t nw = 0;
  std::vector<int64_t> wsup;
  rc = save_warm(ctx, B, d, S1, nullptr, &nw, &wsup);
  if (rc) return rc;
  double sigma = S1.sigma;
  std::vector<int64_t> ired = merge_sorted(scr, wsup);
  // 3.-5. the FP64 ripALM on I_red, warm-started; the full feasibility pass;
  //        violated balls join I_red and the reduced solve runs again
  const double eps_feas = 2.0 * P.tol * sc;
  DevState S2{};
  int rounds = 0;
  int passes = S1.tot_passes, outer = S1.outer, ssn = S1.tot_ssn, cg = S1.tot_cg, bt = S1.tot_bt;
  int64_t fp64_rows = S1.n64_total;
  int64_t* dired = nullptr;
  for (;;) {
    const int64_t nred = (int64_t)ired.size();
    if ((rc = pool(ctx, POOL_RED_IDX, sizeof(int64_t) * (size_t)nred, (void**)&dired))) return rc;
    double *Cr, *Rr;
    if ((rc = pool(ctx, POOL_RED_C, sizeof(double) * (size_t)nred * d, (void**)&Cr))) return rc;
    if ((rc = pool(ctx, POOL_RED_R, sizeof(double) * (size_t)nred, (void**)&Rr))) return rc;
    CK(cudaMemcpyAsync(dired, ired.data(), sizeof(int64_t) * (size_t)nred, cudaMemcpyHostToDevice, s));
    CK(launch_gather_rows(C, R, dired, nred, d, Cr, Rr, s));
    rc = ensure_red(ctx, nred, d);
    if (rc) return rc;
    Buffers& Br = ctx->Bred;
    Br.C_in = Cr;
    Br.use_x16 = B.use_x16;
    Br.bulk = B.bulk;
    Br.fp64_all = B.fp64_all;
    Br.lowp = false;
    Br.wait_cycles = B.wait_cycles;
    CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
    CK(launch_shadow(Cr, Rr, nred, d, Br, Br.vec.o, Br.vec.c0, ctx->d_flags, s));
    rc = init_state(ctx, Br, nred, d, P, sc, r0);
    if (rc) return rc;
    int64_t* widx;
    double *wu, *wv, *wx;
    pool(ctx, POOL_WIDX, 0, (void**)&widx);
    pool(ctx, POOL_WU, 0, (void**)&wu);
    pool(ctx, POOL_WV, 0, (void**)&wv);
    pool(ctx, POOL_WX, 0, (void**)&wx);
    CK(launch_warm_start(Br, d, wx, sigma, widx, wu, wv, nw, dired, nred, s));
    rc = run_ticks(ctx, Br, Cr, Rr, nred, d, P);
    if (rc) return rc;
    S2 = *ctx->h_st;
    passes += S2.tot_passes;
    outer += S2.outer;
    ssn += S2.tot_ssn;
    cg += S2.tot_cg;
    bt += S2.tot_bt;
    fp64_rows += S2.n64_total;
    // the reduced solution against every ball
    CK(launch_final_point(Br, d, dcout, ctx->d_scal + 1, s));
    CK(cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(ctx_sync(ctx));
    const double r_bar = ctx->h_scal[1];
    CK(launch_feas_cert(C, R, m, d, dcout, r_bar, eps_feas, 0, 1, B, ctx->d_scal + 2, ctx->d_i64,
                        ctx->d_i64 + 1, s));
    int64_t nv = 0;
    CK(cudaMemcpyAsync(&nv, ctx->d_i64 + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(ctx_sync(ctx));
    std::vector<int64_t> viol(nv), add;
    if (nv > 0) {
      CK(cudaMemcpyAsync(viol.data(), B.viol, sizeof(int64_t) * (size_t)nv, cudaMemcpyDeviceToHost, s));
      CK(ctx_sync(ctx));
      std::set_difference(viol.begin(), viol.end(), ired.begin(), ired.end(), std::back_inserter(add));
    }
    if (add.empty() || rounds >= P.max_readd || S2.status != 1) break;
    rc = save_warm(ctx, Br, d, S2, dired, &nw, &wsup);
    if (rc) return rc;
    sigma = S2.sigma;
    ired = merge_sorted(ired, add);
    rounds++;
  }
  // the radius lift and the active set over all balls, at the reduced solution
  double r_alm, r_out;
  rc = finish_solve(ctx, ctx->Bred, B, C, R, m, d, P, dcout, &r_alm, &r_out, n_active);
  if (rc) return rc;
  ctx->mult_kind = 4;
  ctx->mult_map = dired;
  ctx->mult_n = S2.nS;
  ctx->mult_m = m;
  ctx->mult_d = d;
  fill_info(info, S2, sc, r_alm, r_out, *n_active);
  if (info) {
    info->passes = passes;
    info->outer_iters = outer;
    info->ssn_iters = ssn;
    info->cg_iters = cg;
    info->backtracks = bt;
    info->fp64_rows = fp64_rows;
    info->n_reduced = (int64_t)ired.size();
    info->readd_rounds = rounds;
    info->lowp_passes = S1.tot_passes;
  }
  *Sout = S2;
  return MEB_OK;
}
