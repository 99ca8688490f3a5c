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

#include "../../include/meb.h"
#include "meb_internal.cuh"

using namespace meb;


struct meb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Buffers B{};
  int64_t buf_m = 0;
  int buf_d = 0;
  void* pool_ptr[16] = {};
  size_t pool_cap[16] = {};
  DevState* h_st = nullptr;     // pinned mirror of the device state
  double* h_scal = nullptr;     // pinned scalars
  int* d_flags = nullptr;       // device int flags
  double* d_scal = nullptr;     // device scalars
  int64_t* d_i64 = nullptr;     // device int64 scalars
  int profiling = 0;            // time every pass launch with CUDA events
  // device-resident solve loop: a CUDA graph whose while-node runs controller
  // ticks until the controller stops; rebuilt when the problem or buffers change
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t gm = 0;
  int gd = 0;
  int gmode = -1;
  int gvar = -1;
  int gprof = -1;
  cudaEvent_t gev[2 * 8] = {};
  long long gwait = -1;
  // options (meb_set_option)
  // tick loop: 0 = graph of kUnrollTicks ticks relaunched until the controller
  // stops (default), 1 = host-driven ticks, 2 = graph with a while-node
  int loop_mode = 0;
  int screen_mode = MEB_SCREEN_FP16;      // solves
  int eval_screen = MEB_SCREEN_FP32;      // meb_eval_alm
  int eval_shadow_exp = 0;                // FP16 shadow scale 2^exp of meb_eval_alm
  long long wait_cycles = 2000000000LL;   // bound of the bulk-copy screen's waits
  // multipliers of the last solve (meb_get_multipliers): 0 none, 1 the
  // support arrays of the final point, 2 one ball, 3 all balls the same point
  int mult_kind = 0;
  int64_t mult_n = 0, mult_m = 0;
  int mult_d = 0;
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
       POOL_H, POOL_G, POOL_COUT, POOL_ACT, POOL_N };

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
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

static void free_buffers(meb_ctx* ctx) {
  Buffers& B = ctx->B;
  void* ptrs[] = {B.X32, B.X16, B.EPS16, B.E32, B.Hhi, B.Hlo, B.R32, B.slot, B.sup_idx[0], B.sup_idx[1], B.sup_u[0], B.sup_u[1],
                  B.sup_v[0], B.sup_v[1], B.part_flag, B.part, B.part_cnt, B.cand_off, B.cand_cnt, B.cand_idx,
                  B.unc_cnt, B.unc_idx, B.unc_slot, B.vlb_part,
                  B.cand_case, B.cand_a, B.cand_n, B.cand_u, B.S_idx, B.S_case, B.S_a, B.S_n,
                  B.S_u, B.S_t, B.W, B.svec_part, B.hpart, B.H, B.hq, B.colsum_part, B.fe_ub, B.fe_lb,
                  B.fe_blb, B.fe_L, B.fq_y32,
                  B.feas_part, B.feas_ipart, B.feas_cnt, B.viol, B.list_tmp, B.count64, B.wq,
                  B.st, B.vec_store};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  const int64_t launches = B.launches;
  memset(&B, 0, sizeof(B));
  B.launches = launches;
  ctx->buf_m = 0;
  ctx->buf_d = 0;
  // the captured tick graph holds the freed pointers: rebuild it on next use
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

// Device buffers sized for (m, d); grown on demand.
static int ensure_buffers(meb_ctx* ctx, int64_t m, int d) {
  if (ctx->buf_m >= m && ctx->buf_d >= d && ctx->buf_m * (int64_t)ctx->buf_d >= m * (int64_t)d &&
      ctx->buf_d == d)
    return MEB_OK;
  free_buffers(ctx);
  Buffers& B = ctx->B;
  const int64_t m_pad = ((m + 255) / 256) * 256;
  const int64_t nblk = m_pad / 256;
  const int d4 = (d + 3) / 4;
  const int n1 = d + 1;
  const int64_t md = m * (int64_t)d;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int64_t ntri = (int64_t)nt * (nt + 1) / 2;
  int64_t hp = (int64_t)152 * n1;
  if (d + 1 <= kMaxDenseN) hp = hp > 24 * ntri * 1024 ? hp : 24 * ntri * 1024;
  B.m_cap = m;
  B.d_cap = d;
  B.nblk_cap = nblk;
  B.hpart_cap = hp;
  CK(dalloc(&B.X32, (size_t)d4 * m_pad));
  CK(dalloc(&B.X16, (size_t)((d4 + 1) / 2) * m_pad));
  CK(dalloc(&B.EPS16, (size_t)m_pad));
  CK(dalloc(&B.E32, (size_t)m_pad));
  CK(dalloc(&B.Hhi, (size_t)(d + 1 <= kMaxDenseN ? n1 * n1 : 1)));
  CK(dalloc(&B.Hlo, (size_t)(d + 1 <= kMaxDenseN ? n1 * n1 : 1)));
  CK(dalloc(&B.R32, (size_t)m_pad));
  CK(dalloc(&B.slot, (size_t)m_pad));   // whole tiles are bulk-copied
  for (int k = 0; k < 2; k++) {
    CK(dalloc(&B.sup_idx[k], (size_t)m));
    CK(dalloc(&B.sup_u[k], (size_t)m));
    CK(dalloc(&B.sup_v[k], (size_t)md));
  }
  // segments of 256 per tile and block: at most (tiles + blocks) * 256 for any grid
  const int64_t ncand = (nblk + kMaxPassBlocks) * 256;
  CK(dalloc(&B.part_flag, (size_t)nblk));
  CK(dalloc(&B.part, (size_t)nblk * P_NREC));
  CK(dalloc(&B.part_cnt, (size_t)nblk * P_NCNT));
  CK(dalloc(&B.cand_off, (size_t)nblk + 1));
  CK(dalloc(&B.cand_cnt, (size_t)nblk));
  CK(dalloc(&B.unc_cnt, (size_t)nblk));
  CK(dalloc(&B.vlb_part, (size_t)nblk));
  CK(dalloc(&B.unc_idx, (size_t)ncand));
  CK(dalloc(&B.unc_slot, (size_t)ncand));
  CK(dalloc(&B.cand_idx, (size_t)ncand));
  CK(dalloc(&B.cand_case, (size_t)ncand));
  CK(dalloc(&B.cand_a, (size_t)ncand));
  CK(dalloc(&B.cand_n, (size_t)ncand));
  CK(dalloc(&B.cand_u, (size_t)ncand));
  CK(dalloc(&B.S_idx, (size_t)m));
  CK(dalloc(&B.S_case, (size_t)m));
  CK(dalloc(&B.S_a, (size_t)m));
  CK(dalloc(&B.S_n, (size_t)m));
  CK(dalloc(&B.S_u, (size_t)m));
  CK(dalloc(&B.S_t, (size_t)m));
  CK(dalloc(&B.W, (size_t)md));
  CK(dalloc(&B.svec_part, (size_t)kSvecBlocks * (3 * d + 1)));
  CK(dalloc(&B.hpart, (size_t)hp));
  CK(dalloc(&B.H, (size_t)(d + 1 <= kMaxDenseN ? n1 * n1 : 1)));
  CK(dalloc(&B.hq, (size_t)n1));
  CK(dalloc(&B.colsum_part, (size_t)((m + 63) / 64) * d));
  CK(dalloc(&B.fe_ub, (size_t)m));
  CK(dalloc(&B.fe_lb, (size_t)m));
  CK(dalloc(&B.fe_blb, (size_t)nblk));
  CK(dalloc(&B.fe_L, 4));
  CK(dalloc(&B.fq_y32, (size_t)4 * d4 + 4));
  CK(dalloc(&B.feas_part, (size_t)nblk + 8));
  CK(dalloc(&B.feas_ipart, (size_t)nblk + 8));
  CK(dalloc(&B.feas_cnt, (size_t)nblk + 8));
  CK(dalloc(&B.viol, (size_t)m));
  CK(dalloc(&B.list_tmp, (size_t)m_pad));
  CK(dalloc(&B.count64, 8));
  CK(dalloc(&B.wq, (size_t)m));
  CK(dalloc(&B.st, 1));
  // vectors of length n1 (x, xt, xk, ab, g, gt, dx, ct, o, sv, sw, st1, cg_*) and y32;
  // each starts on a 16-byte boundary (y32 is read as float4)
  const size_t stride = (size_t)((n1 + 8 + 1) / 2) * 2;
  const size_t nv = 20 * stride + (size_t)(d4 * 4 + 8);
  CK(dalloc(&B.vec_store, nv));
  double* p = B.vec_store;
  auto take = [&](double** q) { *q = p; p += stride; };
  take(&B.vec.x); take(&B.vec.xt); take(&B.vec.xk); take(&B.vec.ab); take(&B.vec.g);
  take(&B.vec.gt); take(&B.vec.dx); take(&B.vec.ct); take(&B.vec.o); take(&B.vec.c0);
  take(&B.vec.sv);
  take(&B.vec.sw); take(&B.vec.st1); take(&B.vec.cg_r); take(&B.vec.cg_z); take(&B.vec.cg_p);
  take(&B.vec.cg_ap); take(&B.vec.cg_diag);
  B.vec.y32 = reinterpret_cast<float*>(p);
  CK(cudaMemsetAsync(B.vec_store, 0, sizeof(double) * nv, ctx->stream));
  ctx->buf_m = m;
  ctx->buf_d = d;
  return MEB_OK;
}

static int pool(meb_ctx* ctx, int id, size_t bytes, void** out) {
  if (ctx->pool_cap[id] < bytes) {
    if (ctx->pool_ptr[id]) cudaFree(ctx->pool_ptr[id]);
    ctx->pool_ptr[id] = nullptr;
    ctx->pool_cap[id] = 0;
    CK(cudaMalloc(&ctx->pool_ptr[id], bytes ? bytes : 8));
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

static int copy_out(meb_ctx* ctx, void* dst, const void* dsrc, size_t bytes, unsigned flags) {
  if (!bytes) return MEB_OK;
  CK(cudaMemcpyAsync(dst, dsrc, bytes,
                     (flags & MEB_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->stream));
  return MEB_OK;
}

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
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_buffers(ctx);
  for (int k = 0; k < 16; k++)
    if (ctx->pool_ptr[k]) cudaFree(ctx->pool_ptr[k]);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->d_flags) cudaFree(ctx->d_flags);
  if (ctx->d_scal) cudaFree(ctx->d_scal);
  if (ctx->d_i64) cudaFree(ctx->d_i64);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  for (int k = 0; k < 2; k++)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  for (int k = 0; k < 16; k++)
    if (ctx->gev[k]) cudaEventDestroy(ctx->gev[k]);
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
    default:
      return fail(ctx, MEB_EINVAL, "unknown option %d", (int)option);
  }
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

static int check_sizes(meb_ctx* ctx, int64_t m, int32_t d) {
  if (m < 1 || m > (int64_t)2147483647 - 256) return fail(ctx, MEB_EINVAL, "m out of range");
  if (d < 1 || d > 16384) return fail(ctx, MEB_EINVAL, "d out of range");
  return MEB_OK;
}

static void host_state_defaults(DevState& S, int64_t m, int d, const meb_params& P, double s) {
  memset(&S, 0, sizeof(S));
  S.m = m;
  S.m_pad = ((m + 255) / 256) * 256;
  S.d = d;
  S.d4 = (d + 3) / 4;
  S.n1 = d + 1;
  S.dense = (d <= P.dense_max_d && d + 1 <= kMaxDenseN) ? 1 : 0;
  S.force_fp64_solve = P.newton_fp64 != 0;
  S.s = s;
  S.inv_s = 1.0 / s;
  S.tol = P.tol;
  S.rho = P.rho;
  S.sigma_max = P.sigma_max;
  S.sigma_growth = P.sigma_growth;
  S.sigma_ratio = P.sigma_ratio;
  S.tau = P.tau;
  S.mu = P.armijo_mu;
  S.max_outer = P.max_outer;
  S.max_ssn = P.max_ssn;
  S.max_backtrack = P.max_backtrack;
  S.max_cg = P.max_cg;
  S.sigma = P.sigma0;
  S.inv_sigma = 1.0 / P.sigma0;
  S.tos = P.tau / P.sigma0;
  S.pinf_prev = INFINITY;
  S.phase = 0;
  S.action = ACT_NONE;
  S.status = 0;
}

static int read_state(meb_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_st, ctx->B.st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MEB_OK;
}

// Build (or reuse) the graph: while (status == 0) { pass; controller; Newton
// (dense); multiplier update; loop condition }.  Every kernel of the tick is
// gated on the controller's action, so the tick is a fixed sequence.
static int solve_graph(meb_ctx* ctx, const double* C, const double* R, int64_t m, int d) {
  Buffers& B = ctx->B;
  const int mode = ctx->loop_mode;
  const int prof = ctx->profiling;
  if (ctx->gexec && ctx->gkey[0] == C && ctx->gkey[1] == R && ctx->gkey[2] == B.st &&
      ctx->gkey[3] == (const void*)(B.use_x16 ? (const void*)B.X16 : (const void*)B.X32) &&
      ctx->gvar == screen_variant(B, d) && ctx->gwait == B.wait_cycles &&
      ctx->gm == m && ctx->gd == d && ctx->gmode == mode && ctx->gprof == prof)
    return MEB_OK;
  if (prof && !ctx->gev[0])
    for (int k = 0; k < 16; k++) CK(cudaEventCreate(&ctx->gev[k]));
  if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (mode == 2) {
    CK(cudaGraphCreate(&ctx->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, ctx->graph, 1, cudaGraphCondAssignDefault));
    // cudaGraphNodeParams holds a union without a default constructor: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = h;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, ctx->graph, nullptr, nullptr, 0, np));
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
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    for (int t = 0; t < kUnrollTicks && e == cudaSuccess; t++) {
      // profiling: CUDA events around every k_screen of the batch (event nodes)
      e = prof ? launch_pass(C, R, B, m, d, s, ctx->gev[2 * t], ctx->gev[2 * t + 1], t)
               : launch_pass(C, R, B, m, d, s);
      if (e == cudaSuccess) e = launch_tick_control(B, m, d, s);
      if (e == cudaSuccess) e = launch_newton_dense(B, d, s);
      if (e == cudaSuccess) e = launch_mult_update(C, B, m, d, s);
    }
    cudaError_t e2 = cudaStreamEndCapture(s, &ctx->graph);
    if (e != cudaSuccess) return fail(ctx, MEB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    CK(e2);
  }
  CK(cudaGraphInstantiate(&ctx->gexec, ctx->graph, 0));
  ctx->gkey[0] = C; ctx->gkey[1] = R; ctx->gkey[2] = B.st;
  ctx->gkey[3] = B.use_x16 ? (const void*)B.X16 : (const void*)B.X32;
  ctx->gvar = screen_variant(B, d);
  ctx->gwait = B.wait_cycles;
  ctx->gm = m; ctx->gd = d; ctx->gmode = mode; ctx->gprof = prof;
  return MEB_OK;
}

extern "C" int meb_solve(meb_ctx* ctx, const double* centers, const double* radii, int64_t m,
                         int32_t d, double tol, const meb_params* params, unsigned flags,
                         double* c_out, int64_t* active_idx, int64_t active_cap,
                         meb_info* info) {
  if (!ctx) return MEB_EINVAL;
  ctx->err[0] = 0;
  int rc = check_sizes(ctx, m, d);
  if (rc) return rc;
  if (!centers || !radii || !c_out || (active_cap > 0 && !active_idx) || active_cap < 0)
    return fail(ctx, MEB_EINVAL, "NULL argument");
  meb_params P;
  if (params) P = *params; else meb_params_default(&P);
  if (tol > 0) P.tol = tol;
  if (!(P.tol > 0) || !(P.rho >= 0 && P.rho < 1) || !(P.sigma0 > 0) || !(P.tau > 0) ||
      !(P.sigma_max >= P.sigma0) || !(P.sigma_growth >= 1) || P.max_outer < 1 || P.max_ssn < 1 ||
      P.max_backtrack < 0 || P.max_cg < 1 || !(P.active_theta >= 0))
    return fail(ctx, MEB_EINVAL, "invalid parameters");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  rc = ensure_buffers(ctx, m, d);
  if (rc) return rc;
  Buffers& B = ctx->B;
  const double* C;
  const double* R;
  rc = stage_in(ctx, POOL_C, centers, sizeof(double) * (size_t)m * d, flags, (const void**)&C);
  if (rc) return rc;
  rc = stage_in(ctx, POOL_R, radii, sizeof(double) * (size_t)m, flags, (const void**)&R);
  if (rc) return rc;
  B.C_in = C;
  ctx->mult_kind = 0;
  B.use_x16 = ctx->screen_mode == MEB_SCREEN_FP16 || ctx->screen_mode == MEB_SCREEN_FP16_BULK;
  B.bulk = ctx->screen_mode == MEB_SCREEN_FP16_BULK;
  B.fp64_all = ctx->screen_mode == MEB_SCREEN_FP64;
  B.wait_cycles = ctx->wait_cycles;
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s));
  if (info) memset(info, 0, sizeof(*info));

  // FP32 shadow (origin c_0) and the mean centre c0; r0 = max_i ||c0 - c_i|| + r_i
  // (the shadow also checks the input; the plain FP64 mode reads it no further)
  CK(launch_shadow(C, R, m, d, B, B.vec.o, B.vec.c0, ctx->d_flags, s));
  CK(launch_feas_cert(C, R, m, d, B.vec.c0, 0.0, INFINITY, 2, 1, B, ctx->d_scal, ctx->d_i64,
                      ctx->d_i64 + 1, s));
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int bad;
  memcpy(&bad, ctx->h_scal + 1, sizeof(int));
  if (bad) return fail(ctx, MEB_EINVAL, "non-finite centre or radius, or negative radius");
  const double r0 = ctx->h_scal[0];
  void* dcout = nullptr;
  if (flags & MEB_PTR_DEVICE) dcout = c_out;
  else { rc = pool(ctx, POOL_COUT, sizeof(double) * (size_t)d, &dcout); if (rc) return rc; }

  if (m == 1 || r0 == 0.0) {
    // one ball, or every ball the same point: the answer is that ball
    CK(cudaMemcpyAsync(dcout, m == 1 ? C : B.vec.c0, sizeof(double) * d,
                       cudaMemcpyDeviceToDevice, s));
    if (!(flags & MEB_PTR_DEVICE))
      CK(cudaMemcpyAsync(c_out, dcout, sizeof(double) * d, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double r = (m == 1) ? r0 : 0.0;
    const int64_t na = m;
    for (int64_t k = 0; k < active_cap && k < na; k++) {
      if (flags & MEB_PTR_DEVICE) CK(cudaMemcpy(active_idx + k, &k, sizeof(int64_t), cudaMemcpyHostToDevice));
      else active_idx[k] = k;
    }
    if (info) {
      info->r = r; info->r_alm = r; info->scale = 1.0; info->n_active = na; info->status = 0;
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
  CK(cudaMemsetAsync(B.slot, 0xff, sizeof(int) * (size_t)m, s));
  CK(prepare_pass(B, d));
  CK(prepare_newton(d));
  if (B.use_x16) CK(launch_shadow16(B, m, d, 1.0 / sc, s));
  host_state_defaults(*ctx->h_st, m, d, P, sc);
  ctx->h_st->sh_s = sc;
  ctx->h_st->sh_inv_s = 1.0 / sc;
  ctx->h_st->rt_abs = r0;   // initial radius; k_state_init scales it
  CK(cudaMemcpyAsync(B.st, ctx->h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(launch_state_init(B, d, s));
  const bool dense = ctx->h_st->dense;
  ctx->prof_screens = 0;
  // per ball: the shadow row (FP16: 16 bytes per 8 coordinates; FP32: 16
  // bytes per 4 coordinates), its error bound, the FP32 radius and the slot
  const int64_t d4 = (d + 3) / 4;
  const int64_t pass_bytes = B.fp64_all ? m * 8   // the slot read and the list written
                                         : m * (B.use_x16 ? 16 * ((d4 + 1) / 2) + 12 : 16 * d4 + 12);

  const int64_t max_ticks =
      (int64_t)P.max_outer * (P.max_ssn + 2) * (P.max_backtrack + 2) + 16;
  if (dense && ctx->loop_mode != 1 && !(ctx->profiling && ctx->loop_mode == 2)) {
    // device-resident ticks: graph launches, one status read per kUnrollTicks ticks
    rc = solve_graph(ctx, C, R, m, d);
    if (rc) return rc;
    const int64_t before = B.launches;
    if (ctx->loop_mode == 2) {
      ctx->h_st->max_ticks = max_ticks < 20000 ? max_ticks : 20000;
      CK(cudaMemcpyAsync(&B.st->max_ticks, &ctx->h_st->max_ticks, sizeof(int64_t),
                         cudaMemcpyHostToDevice, s));
      CK(cudaGraphLaunch(ctx->gexec, s));
      rc = read_state(ctx);
      if (rc) return rc;
      B.launches = before + ctx->h_st->ticks * (tick_launches(d) + 1);
      if (ctx->h_st->status == kStatusTickCap)
        return fail(ctx, MEB_ECUDA, "controller did not terminate");
    } else {
      int64_t ticks = 0;
      for (;;) {
        if (ctx->profiling)
          CK(cudaMemsetAsync(B.st->screen_log, 0, sizeof(B.st->screen_log), s));
        CK(cudaGraphLaunch(ctx->gexec, s));
        ticks += kUnrollTicks;
        rc = read_state(ctx);
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
      B.launches = before + ticks * tick_launches(d);
    }
  } else {
    int64_t ticks = 0;
    for (;;) {
      CK(launch_pass(C, R, B, m, d, s, ctx->profiling ? ctx->ev[0] : nullptr,
                     ctx->profiling ? ctx->ev[1] : nullptr));
      CK(launch_tick_control(B, m, d, s));
      rc = read_state(ctx);
      if (rc) return rc;
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
      if (ctx->h_st->action == ACT_NEWTON) {
        if (dense) {
          CK(launch_newton_dense(B, d, s));
        } else {
          CK(launch_cg_setup(B, d, s));
          for (int round = 0; round <= P.max_cg / 4 + 1; round++) {
            for (int k = 0; k < 4; k++) CK(launch_cg_iter(B, d, s));
            rc = read_state(ctx);
            if (rc) return rc;
            if (ctx->h_st->cg_done || ctx->h_st->status != 0 || ctx->h_st->action != ACT_NEWTON) break;
          }
          CK(launch_cg_finish(B, d, s));
        }
      }
      CK(launch_mult_update(C, B, m, d, s));
      if (++ticks > max_ticks) return fail(ctx, MEB_ECUDA, "controller did not terminate");
    }
  }
  const DevState S = *ctx->h_st;
  if (S.status == kStatusWaitTimeout)
    return fail(ctx, MEB_ETIMEOUT, "a device wait timed out (a bulk copy did not complete)");
  ctx->mult_kind = 1;
  ctx->mult_n = S.nS;
  ctx->mult_m = m;
  ctx->mult_d = d;

  // final point, radius lift (max-type value at c) and active set
  double* d_ralm = ctx->d_scal + 1;
  CK(launch_final_point(B, d, (double*)dcout, d_ralm, s));
  CK(launch_feas_cert(C, R, m, d, (const double*)dcout, 0.0, INFINITY, 2, 1, B, ctx->d_scal + 2,
                      ctx->d_i64 + 2, ctx->d_i64 + 3, s));
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double r_alm = ctx->h_scal[1];
  const double r_out = ctx->h_scal[2];
  CK(launch_feas_cert(C, R, m, d, (const double*)dcout, r_out, P.active_theta * r_out, 1, 0, B,
                      nullptr, nullptr, ctx->d_i64 + 5, s, /*reuse_bounds=*/true));
  CK(cudaMemcpyAsync(ctx->h_scal + 8, ctx->d_i64 + 5, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (!(flags & MEB_PTR_DEVICE))
    CK(cudaMemcpyAsync(c_out, dcout, sizeof(double) * d, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int64_t n_active;
  memcpy(&n_active, ctx->h_scal + 8, sizeof(int64_t));
  const int64_t ncp = n_active < active_cap ? n_active : active_cap;
  if (ncp > 0) {
    rc = copy_out(ctx, active_idx, B.viol, sizeof(int64_t) * (size_t)ncp, flags);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
  }
  if (info) {
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
  return S.status == 1 ? MEB_OK : fail(ctx, MEB_ENOTCONV, "iteration cap reached");
}

extern "C" int meb_eval_alm(meb_ctx* ctx, const double* centers, const double* radii, int64_t m,
                            int32_t d, const double* x, const double* xbar, const double* U,
                            const double* V, double sigma, double tau, const double* q,
                            unsigned flags, double* psi, double* grad, double* Uplus,
                            double* Vplus, double* Hq, double* H, int64_t* case_counts) {
  if (!ctx) return MEB_EINVAL;
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
  host_state_defaults(*ctx->h_st, m, d, P, 1.0);
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
  rc = read_state(ctx);
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
  CK(cudaStreamSynchronize(s));
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
    CK(cudaStreamSynchronize(s));
  }
  return MEB_OK;
}


extern "C" int meb_get_multipliers(meb_ctx* ctx, unsigned flags, int64_t* idx, double* u,
                                   double* v, int64_t cap, int64_t* n_sup) {
  if (!ctx) return MEB_EINVAL;
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
  if (ctx->mult_kind == 1) {
    int64_t* didx;
    double *du, *dv;
    int rc;
    if (dev) { didx = idx; du = u; dv = v; }
    else {
      if ((rc = pool(ctx, POOL_ACT, sizeof(int64_t) * (size_t)k, (void**)&didx))) return rc;
      if ((rc = pool(ctx, POOL_UP, sizeof(double) * (size_t)k, (void**)&du))) return rc;
      if ((rc = pool(ctx, POOL_VP, sizeof(double) * (size_t)k * d, (void**)&dv))) return rc;
    }
    CK(launch_mult_out(ctx->B, d, didx, du, dv, k, s));
    if (!dev) {
      CK(cudaMemcpyAsync(idx, didx, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(u, du, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(v, dv, sizeof(double) * (size_t)k * d, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeHost(hi);
    cudaFreeHost(hu);
    CK(e);
  } else {
    for (int64_t t = 0; t < k; t++) { idx[t] = t; u[t] = uval; }
    memset(v, 0, sizeof(double) * (size_t)k * d);
  }
  return MEB_OK;
}
