// libmeb solver kernels: the device-resident controller of Algorithms 1 and 2,
// the Newton systems (dense and matrix-free), the multiplier update and the
// evaluation-entry outputs, for sm_103a.
//
// Notation (Sec. 2, Sec. 4): at x = (r, c) with multipliers (u_i, v_i),
// z_i = (r_i - r, c_i - c)/s + (u_i, v_i)/sigma and (u_i^+, v_i^+) = sigma Pi_Q(z_i).
// The iterate lives on the scaled problem (data divided by the power of two
// s); the streaming kernels read the unscaled input.  The controller kernels
// run on one block; their vector work (length d + 1) is spread over it.
#include <algorithm>

#include "meb_solve_dev.cuh"

namespace meb {

cudaError_t launch_tick_control(Buffers& B, int64_t m, int d, cudaStream_t s) {
  // the line-search controller runs in the last block of k_rows64 and the
  // stop-test controller in the last block of k_svec (meb_control.cuh)
  return launch_support_rows(B.C_in, B, m, d, s);
}

__global__ void __launch_bounds__(256) k_syrk(Buffers B, int d, int force) {
  pdl_wait_and_release();
  if (!force && (!newton_gate(B.st) || syrk_in_solve(B.st, d))) return;
  syrk_block(B, d, blockIdx.x, blockIdx.y);
}

__global__ void k_syrk_reduce(Buffers B, int d, int force) {
  pdl_wait_and_release();
  if (!force && (!newton_gate(B.st) || syrk_in_solve(B.st, d))) return;
  syrk_reduce_block(B, d, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_newton_chol(Buffers B, int d) {
  pdl_wait_and_release();
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_NEWTON || !st->need_fp64_solve) return;
  extern __shared__ double Lp[];
  newton_chol_body(B, d, Lp);
}

__global__ void __launch_bounds__(256) k_newton_gj(Buffers B, int d) {
  pdl_wait_and_release();
  if (!newton_gate(B.st)) return;
  newton_gj_body(B, d);
}

__global__ void __launch_bounds__(256, 1) k_newton_gj_reg(Buffers B, int d) {
  pdl_wait_and_release();
  if (!newton_gate(B.st)) return;
  newton_gj_reg_body(B, d);
}

// n <= 32: the single-warp sweep (with the same Cholesky fallback)
__global__ void __launch_bounds__(256, 1) k_newton_gj_warp(Buffers B, int d) {
  pdl_wait_and_release();
  if (!newton_gate(B.st)) return;
  newton_gj_small_body(B, d);
}

// Launches per Newton step of the dense path: SYRK, its reduction and the
// solve (n <= kGjRegN: Gauss-Jordan with the Cholesky fallback inside), or
// SYRK, reduction, shared-memory Gauss-Jordan and a separate Cholesky.
int newton_dense_launches(int d) { return d + 1 <= kGjRegN ? 3 : 4; }

// Host set-up outside any stream capture: dynamic shared memory limits.
static cudaError_t prepare_hvp(int d);

cudaError_t prepare_newton(int d) {
  const int n = d + 1;
  if (n > kMaxDenseN) return prepare_hvp(d);   // matrix-free path
  const size_t shc = sizeof(double) * (size_t)n * (n + 1) / 2;
  cudaError_t e = cudaSuccess;
  if (n <= kGjWarpN) return raise_smem_limit((const void*)k_newton_gj_warp, shc);
  if (n <= kGjRegN) return raise_smem_limit((const void*)k_newton_gj_reg, shc);
  const size_t shg = sizeof(float) * (size_t)n * n;
  e = raise_smem_limit((const void*)k_newton_gj, shg);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)k_newton_chol, shc);
  return e;
}

cudaError_t launch_newton_dense(Buffers& B, int d, cudaStream_t s) {
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  cudaError_t e = launch_pdl(k_syrk, dim3(ntri, kSyrkGroups), dim3(256), 0, s, B, d, 0);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_syrk_reduce, dim3(64), dim3(256), 0, s, B, d, 0);
  if (e != cudaSuccess) return e;
  const int n = d + 1;
  const size_t shc = sizeof(double) * (size_t)n * (n + 1) / 2;
  if (n <= kGjWarpN) {
    e = launch_pdl(k_newton_gj_warp, dim3(1), dim3(256), shc, s, B, d);
  } else if (n <= kGjRegN) {
    e = launch_pdl(k_newton_gj_reg, dim3(1), dim3(256), shc, s, B, d);
  } else {
    e = launch_pdl(k_newton_gj, dim3(1), dim3(256), sizeof(float) * (size_t)n * n, s, B, d);
    // FP64 Cholesky only when the FP32 inverse could not be refined
    if (e == cudaSuccess) e = launch_pdl(k_newton_chol, dim3(1), dim3(256), shc, s, B, d);
  }
  if (e != cudaSuccess) return e;
  B.launches += newton_dense_launches(d);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_hvp_dot(Buffers B, int d, const double* __restrict__ q,
                                                  double* __restrict__ wq, int force) {
  extern __shared__ float dyn_q32[];   // d floats with FP32 rows
  if (!force && !cg_gate(B.st)) return;
  if (B.W32 && !force) hvp_dot_block<true>(B, d, q, wq, blockIdx.x, gridDim.x, dyn_q32);
  else hvp_dot_block<false>(B, d, q, wq, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_hvp_acc(Buffers B, int d, const double* __restrict__ q,
                                                  const double* __restrict__ wq,
                                                  double* __restrict__ part, int force) {
  if (!force && !cg_gate(B.st)) return;
  if (B.W32 && !force) hvp_acc_block<true>(B, d, q, wq, part, blockIdx.x, gridDim.x, blockIdx.y);
  else hvp_acc_block<false>(B, d, q, wq, part, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_cg_setup(Buffers B, int d) {
  if (!newton_gate(B.st)) return;
  cg_setup_body(B, d);
}

__global__ void __launch_bounds__(256) k_cg_update(Buffers B, int d, int nblk) {
  if (!cg_gate(B.st)) return;
  cg_update_body(B, d, nblk);
}

__global__ void __launch_bounds__(256) k_cg_finish(Buffers B, int d) {
  if (!newton_gate(B.st)) return;
  cg_finish_body(B, d);
}

cudaError_t launch_cg_setup(Buffers& B, int d, cudaStream_t s) {
  k_cg_setup<<<1, 256, 0, s>>>(B, d);
  B.launches += 1;
  return cudaGetLastError();
}

// the FP32 query of the products in shared memory (set before any capture)
static cudaError_t prepare_hvp(int d) {
  return raise_smem_limit((const void*)k_hvp_dot, sizeof(float) * (size_t)d);
}

cudaError_t launch_cg_iter(Buffers& B, int64_t m, int d, cudaStream_t s) {
  const size_t qsm = B.W32 ? sizeof(float) * (size_t)d : 0;
  cudaError_t e = raise_smem_limit((const void*)k_hvp_dot, qsm);
  if (e != cudaSuccess) return e;
  k_hvp_dot<<<kHvpBlocks * 4, 256, qsm, s>>>(B, d, B.vec.cg_p, B.wq, 0);
  if (B.W32) {   // FP32 products: row groups x column chunks, four blocks per SM
    const int chunks = (d + 255) / 256;
    // four blocks per SM, and groups of at least 256 of the instance's balls
    // (the support is at most m rows; a fixed count per instance, so the
    // order of the sums does not depend on the iteration)
    const int64_t by_m = (m + 255) / 256;
    const int groups = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)kHvpGroups32, (int64_t)(4 * 152 + chunks - 1) / chunks, by_m}));
    k_hvp_acc<<<dim3(groups, chunks), 256, 0, s>>>(B, d, B.vec.cg_p, B.wq, B.hpart, 0);
    k_cg_update<<<1, 256, 0, s>>>(B, d, groups);
  } else {
    k_hvp_acc<<<kHvpBlocks, 256, 0, s>>>(B, d, B.vec.cg_p, B.wq, B.hpart, 0);
    k_cg_update<<<1, 256, 0, s>>>(B, d, kHvpBlocks);
  }
  B.launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_cg_finish(Buffers& B, int d, cudaStream_t s) {
  k_cg_finish<<<1, 256, 0, s>>>(B, d);
  B.launches += 1;
  return cudaGetLastError();
}

template <bool LOWP>
__global__ void __launch_bounds__(256) k_mult_rows(const double* __restrict__ C, Buffers B,
                                                   int d) {
  pdl_wait_and_release();
  DevState* st = B.st;
  if (st->status != 0 || st->action != ACT_OUTER) return;
  mult_rows_block<LOWP>(C, B, d, blockIdx.x, gridDim.x);
  // the last block switches to the new multiplier buffers
  if (last_block_ticket(&st->ctr_slots) && threadIdx.x == 0) mult_flip(st);
}

cudaError_t launch_mult_update(const double* C, Buffers& B, int64_t m, int d, cudaStream_t s) {
  (void)m;
  cudaError_t e = B.lowp ? launch_pdl(k_mult_rows<true>, dim3(304), dim3(256), 0, s, C, B, d)
                        : launch_pdl(k_mult_rows<false>, dim3(304), dim3(256), 0, s, C, B, d);
  if (e != cudaSuccess) return e;
  B.launches += 1;
  return cudaGetLastError();
}

__global__ void k_state_init(Buffers B, int d) { state_init_body(B, d); }

cudaError_t launch_state_init(Buffers& B, int d, cudaStream_t s) {
  k_state_init<<<1, 256, 0, s>>>(B, d);
  B.launches += 1;
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
    cudaMemcpyAsync(H, B.H, sizeof(double) * (size_t)n2, cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

__global__ void k_final_point(Buffers B, int d, double* __restrict__ c_out,
                              double* __restrict__ r_alm) {
  final_point_body(B, d, c_out, r_alm);
}

// Loop condition of the device-resident solve (CUDA graph while-node): one
// more tick while the controller runs; a tick cap ends a loop that does not
// terminate with status kStatusTickCap.
__global__ void k_loop_cond(Buffers B, cudaGraphConditionalHandle h) {
  DevState* st = B.st;
  st->ticks += 1;
  if (st->status == 0 && st->ticks >= st->max_ticks) st->status = kStatusTickCap;
  cudaGraphSetConditional(h, st->status == 0 ? 1u : 0u);
}

cudaError_t launch_loop_cond(Buffers& B, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_loop_cond<<<1, 1, 0, s>>>(B, h);
  B.launches += 1;
  return cudaGetLastError();
}

// The condition of the CG loop node of a tick graph: another CG iteration
// while the conjugate gradients of this Newton system run (cg_update ends them
// at convergence or at max_cg, so the loop ends).
__global__ void k_cg_cond(Buffers B, cudaGraphConditionalHandle h) {
  DevState* st = B.st;
  st->cg_bodies += 1;
  cudaGraphSetConditional(h, cg_gate(st) ? 1u : 0u);
}

cudaError_t launch_cg_cond(Buffers& B, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_cg_cond<<<1, 1, 0, s>>>(B, h);
  return cudaGetLastError();
}

// Multipliers (u_i, v_i)^{k+1} = sigma Pi(z_i) at the last accepted point
// (Algorithm 1's multiplier update), compacted over the support S in ball
// order: idx[k], u[k], v[k*d ..]; v = sigma b (case I) or u w (case M), with
// W holding b (I) or w = b/||b|| (M).  The first `cap` support entries.
__global__ void k_mult_out(Buffers B, int d, int64_t* __restrict__ idx, double* __restrict__ u,
                           double* __restrict__ v, int64_t cap) {
  const DevState* st = B.st;
  const int64_t nS = st->nS < cap ? st->nS : cap;
  const double sigma = st->sigma;
  const int lane = threadIdx.x & 31;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nS;
       k += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double coef = (B.S_case[k] == CASE_I) ? sigma : B.S_u[k];
    for (int j = lane; j < d; j += 32) v[k * d + j] = coef * B.W[k * d + j];
    if (lane == 0) {
      idx[k] = B.S_idx[k];
      u[k] = B.S_u[k];
    }
  }
}

cudaError_t launch_mult_out(Buffers& B, int d, int64_t* idx, double* u, double* v, int64_t cap,
                            cudaStream_t s) {
  k_mult_out<<<152, 256, 0, s>>>(B, d, idx, u, v, cap);
  B.launches += 1;
  return cudaGetLastError();
}

// ===========================================================================
// The mixed-precision pipeline (Sec. 4.2): the reduced instance and its warm
// start.

// Rows idx[k] of (C, R), k < n, into (Cr, Rr): warp per row.
__global__ void k_gather_rows(const double* __restrict__ C, const double* __restrict__ R,
                              const int64_t* __restrict__ idx, int64_t n, int d,
                              double* __restrict__ Cr, double* __restrict__ Rr) {
  const int lane = threadIdx.x & 31;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n;
       k += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t i = idx[k];
    for (int j = lane; j < d; j += 32) Cr[k * d + j] = C[i * d + j];
    if (lane == 0) Rr[k] = R[i];
  }
}

cudaError_t launch_gather_rows(const double* C, const double* R, const int64_t* idx, int64_t n,
                               int d, double* Cr, double* Rr, cudaStream_t s) {
  k_gather_rows<<<304, 256, 0, s>>>(C, R, idx, n, d, Cr, Rr);
  return cudaGetLastError();
}

// Warm start of the reduced solve (the state was initialised by
// k_state_init): x = xk = (alpha, beta) = the previous point (scaled), the
// previous penalty, and the previous multipliers (full-instance indices widx,
// all present in the sorted list ired of the reduced instance's balls) as the
// current multipliers, then the first trial's query shadow.  One block.
__global__ void k_warm_start(Buffers B, int d, const double* __restrict__ wx, double sigma,
                             const int64_t* __restrict__ widx, const double* __restrict__ wu,
                             const double* __restrict__ wv, int64_t nw,
                             const int64_t* __restrict__ ired, int64_t nred) {
  __shared__ double sh[32];
  DevState* st = B.st;
  const DevVecs& V = B.vec;
  for (int k = threadIdx.x; k <= d; k += blockDim.x) {
    V.x[k] = wx[k]; V.xt[k] = wx[k]; V.xk[k] = wx[k]; V.ab[k] = wx[k];
  }
  for (int64_t k = threadIdx.x; k < nw; k += blockDim.x) {
    const int64_t i = widx[k];
    int64_t lo = 0, hi = nred;   // the position of i in ired
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ired[mid] < i) lo = mid + 1; else hi = mid;
    }
    B.sup_idx[0][k] = (int)lo;
    B.sup_u[0][k] = wu[k];
    B.slot[lo] = (int)k;
  }
  for (int64_t e = threadIdx.x; e < nw * d; e += blockDim.x) B.sup_v[0][e] = wv[e];
  // ||v_k||^2 as the rows sum it (lane-strided FMAs, warp tree)
  const int lane = threadIdx.x & 31;
  for (int64_t k = threadIdx.x >> 5; k < nw; k += blockDim.x >> 5) {
    double vv = 0.0;
    for (int j = lane; j < d; j += 32) {
      const double v = wv[k * d + j];
      vv = fma(v, v, vv);
    }
    vv = warp_sum_t(vv);
    if (lane == 0) B.sup_vv[0][k] = vv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->sigma = sigma;
    st->inv_sigma = 1.0 / sigma;
    st->tos = st->tau / sigma;
    st->sup_cur = 0;
    st->nsup = (int)nw;
  }
  __syncthreads();
  set_trial(st, V, d, sh);
}

cudaError_t launch_warm_start(Buffers& B, int d, const double* wx, double sigma,
                              const int64_t* widx, const double* wu, const double* wv, int64_t nw,
                              const int64_t* ired, int64_t nred, cudaStream_t s) {
  k_warm_start<<<1, 256, 0, s>>>(B, d, wx, sigma, widx, wu, wv, nw, ired, nred);
  B.launches += 1;
  return cudaGetLastError();
}

// idx[k] = map[idx[k]] (reduced-instance indices to full-instance indices).
__global__ void k_map_idx(int64_t* __restrict__ idx, int64_t n, const int64_t* __restrict__ map) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    idx[k] = map[idx[k]];
}

cudaError_t launch_map_idx(int64_t* idx, int64_t n, const int64_t* map, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_map_idx<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(idx, n, map);
  return cudaGetLastError();
}

cudaError_t launch_final_point(Buffers& B, int d, double* c_out, double* r_alm, cudaStream_t s) {
  k_final_point<<<1, 256, 0, s>>>(B, d, c_out, r_alm);
  B.launches += 1;
  return cudaGetLastError();
}

}  // namespace meb
