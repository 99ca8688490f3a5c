// The ragged-batch solver: one persistent launch in which every thread block
// takes instances from a device queue (largest first, by the order of the
// items) and solves each one completely: Algorithm 1 with Algorithm 2 and the
// feasibility pass of Sec. 4.2, the same steps as meb_solve's multi-block
// tick loop.
//
// The block runs the same bodies as the multi-block kernels (meb_pass_dev.cuh,
// meb_solve_dev.cuh), walking each of their grids one block at a time: a pass
// over the instance is its pass blocks in order, the controller runs after
// the last of them, and every phase is gated on the controller's action as
// the kernels of the tick are.  Sums keep their fixed per-block order, so an
// instance's result depends only on the instance and its configuration, not
// on the rest of the batch or the block that took it.
//
// GB300 layout: one or two resident blocks per SM (152 SMs) each stream their
// instance's shadow rows (coalesced 16-byte loads, 32 balls per warp); small
// instances stay in L2 between passes, large ones stream from HBM, and the
// largest-first queue keeps the tail short.  The controller and the Newton
// solve of one instance overlap the passes of the others on the same SM.
#include <type_traits>

#include "meb_pass_dev.cuh"
#include "meb_solve_dev.cuh"

namespace meb {

__device__ __forceinline__ bool batch_grad_gate(const DevState* st) {
  return st->status == 0 && st->action == ACT_GRAD;
}
__device__ __forceinline__ bool batch_outer_gate(const DevState* st) {
  return st->status == 0 && st->action == ACT_OUTER;
}

// The feasibility pass of Sec. 4.2 by one block (the phases of
// launch_feas_cert in order).  mode/want_max/eps/r as there; the maximum goes
// to *dmax, the list (when list_out) to list_out[0 .. cap), its size to *cnt.
__device__ void batch_feas(FeasArgs& F, const Buffers& B, const double* c, double r, double eps,
                           int mode, int want_max, bool reuse_bounds, double* dmax,
                           int64_t* cnt, int64_t* list_out, int64_t cap) {
  if (threadIdx.x == 0) {
    F.c = c;
    F.r = r;
    F.eps = eps;
    F.mode = mode;
    F.want_max = want_max;
  }
  __syncthreads();
  const int nb = (int)((F.m + kFeasNT - 1) / kFeasNT);
  if (!reuse_bounds) {
    query_shadow_body(c, B.vec.o, F.d, B.fq_y32, B.fe_L + 1, nullptr);
    __syncthreads();
    for (int b = 0; b < nb; b++) {
      feas_a_block(F, b);
      __syncthreads();
    }
  }
  if (want_max) {
    feas_L_body(B.fe_blb, nb, B.fe_L);
    __syncthreads();
  }
  for (int b = 0; b < nb; b++) {
    feas_b_block(F, b);
    __syncthreads();
  }
  feas_final_body(B.feas_part, B.feas_ipart, B.feas_cnt, nb, dmax, nullptr, cnt);
  __syncthreads();
  if (list_out && cap > 0) {
    for (int b = 0; b < (nb + 255) / 256; b++) {
      gather_lists_block(b, B.feas_cnt, B.list_tmp, nb, kFeasNT, list_out, cap);
      __syncthreads();
    }
  }
}

template <bool HALF>
__device__ void batch_solve_one(const BatchArgs& G, int j, const Buffers& B,
                                const BatchConfig& cf) {
  __shared__ PassArgs sA;
  __shared__ FeasArgs sF;
  const BatchItemDev& I = G.items[j];
  BatchOut* O = G.out + j;
  const double* C = I.C;
  const double* R = I.R;
  const int64_t m = I.m;
  const int d = I.d;
  const int64_t m_pad = ((m + 255) / 256) * 256;
  const int d4 = (d + 3) / 4;
  const int tid = threadIdx.x;
  DevState* st = B.st;
  double* scal = B.scal;              // [0] r0, [1] r_out, [2] r_alm
  int64_t* cnt = B.count64;           // [0] n_active, [1] scratch count
  int* bad = reinterpret_cast<int*>(B.count64 + 4);
  if (tid == 0) {
    *bad = 0;
    sF.C = C; sF.R = R; sF.m = m; sF.m_pad = m_pad; sF.d = d; sF.d4 = d4;
    sF.X32 = B.X32; sF.R32 = B.R32; sF.E32 = B.E32;
    sF.y32 = B.fq_y32; sF.ynp = B.fe_L + 1; sF.all64 = 0;
    sF.eub = B.fe_ub; sF.elb = B.fe_lb; sF.blb = B.fe_blb;
    sF.bmax = B.feas_part; sF.barg = B.feas_ipart; sF.bcnt = B.feas_cnt; sF.blist = B.list_tmp;
    sF.L = B.fe_L;
  }
  __syncthreads();
  // the FP32 shadow (relative to the first centre), the input check and the
  // column sums; the mean centre c0 (column sums in block order)
  const int nsb = (int)((m + kShadowBalls - 1) / kShadowBalls);
  for (int b = 0; b < nsb; b++) {
    shadow_block(b, C, R, m, d, m_pad, B.X32, B.R32, B.E32, B.colsum_part, bad);
    __syncthreads();
  }
  for (int jj = tid; jj < d; jj += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nsb; b++) t += B.colsum_part[(int64_t)b * d + jj];
    B.vec.o[jj] = (double)f64_to_f32_trunc(C[jj]);
    B.vec.c0[jj] = C[jj] + t / (double)m;
  }
  __syncthreads();
  if (*bad) {
    if (tid == 0) {
      O->status = -1;
      O->n_active = 0;
    }
    return;
  }
  // r0 = max_i ||c0 - c_i|| + r_i (certified bounds + FP64 candidates)
  batch_feas(sF, B, B.vec.c0, 0.0, INFINITY, 2, 1, false, scal, nullptr, nullptr, 0);
  const double r0 = scal[0];
  if (m == 1 || r0 == 0.0) {
    // one ball, or every ball the same point: the answer is that ball
    const double* src = (m == 1) ? C : B.vec.c0;
    for (int jj = tid; jj < d; jj += blockDim.x) I.c_out[jj] = src[jj];
    for (int64_t k = tid; k < I.act_cap && k < m; k += blockDim.x) I.act[k] = k;
    if (tid == 0) {
      O->r = (m == 1) ? r0 : 0.0;
      O->r_alm = O->r;
      O->scale = 1.0;
      O->n_active = m;
      O->status = 0;
      for (int k = 0; k < 5; k++) O->kkt[k] = 0.0;
      O->kkt_max = 0.0;
      O->outer = O->ssn = O->cg = O->passes = O->backtracks = 0;
      O->inverses = O->fp64_solves = 0;
      O->fp64_rows = 0;
    }
    __syncthreads();
    return;
  }
  int ex;
  frexp(r0, &ex);
  double sc = ldexp(1.0, ex);
  if (sc / 2.0 >= r0) sc /= 2.0;
  const int dense = (d + 1 <= kGjRegN && d <= G.P.dense_max_d) ? 1 : 0;
  for (int64_t i = tid; i < m; i += blockDim.x) B.slot[i] = -1;
  if (HALF) {
    for (int64_t b = 0; b < m_pad / 256; b++)
      shadow16_block((int)b, B.X32, B.E32, m_pad, d4, (float)(1.0 / sc), B.X16, B.EPS16);
  }
  const int64_t ntiles = (m + kPassThreads - 1) / kPassThreads;
  int tpvb = cf.tiles_per_vb < 1 ? 1 : cf.tiles_per_vb;
  if ((ntiles + tpvb - 1) / tpvb > kMaxPassBlocks) tpvb = (int)((ntiles + kMaxPassBlocks - 1) / kMaxPassBlocks);
  const int nvb = (int)((ntiles + tpvb - 1) / tpvb);
  if (tid == 0) {
    state_defaults(*st, m, d, G.P, sc, dense);
    st->rt_abs = r0;
    PassArgs& A = sA;
    A.C = C; A.R = R; A.m = m; A.m_pad = m_pad; A.d = d; A.d4 = d4;
    A.tiles_per_block = tpvb;
    A.log_slot = -1;
    A.wait_cycles = 0;
    A.X32 = B.X32; A.X16 = HALF ? B.X16 : nullptr; A.EPS16 = B.EPS16; A.E32 = B.E32;
    A.R32 = B.R32; A.slot = B.slot;
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
  }
  __syncthreads();
  state_init_body(B, d);
  __syncthreads();

  // the controller ticks (screen, FP64 rows + line-search control, support
  // rows + stop test, Newton step, multiplier update), each phase gated on
  // the action exactly as the kernels of the multi-block tick
  const int64_t seg = (int64_t)tpvb * kPassThreads;
  const int nt = (d + kSyrkTile - 1) / kSyrkTile;
  const int ntri = nt * (nt + 1) / 2;
  for (int64_t tick = 0;; tick++) {
    if (screen_gate(st)) {
      for (int vb = 0; vb < nvb; vb++) {
        screen_block<HALF>(sA, vb);
        __syncthreads();
      }
      early_body(B, d, nvb);
      __syncthreads();
    }
    if (rows_gate(st)) {
      for (int vb = 0; vb < nvb; vb++) {
        rows_block(sA, vb);
        __syncthreads();
      }
      control_a_body(B, d, nvb);
      __syncthreads();
    }
    if (batch_grad_gate(st)) {
      const int nS = st->nS;
      if (nS > I.sup_cap) {   // the support rows would not fit the instance's room
        if (tid == 0) st->status = kStatusSupportCap;
        __syncthreads();
        break;
      }
      const int rpb = svec_rows_per_block(nS, cf.nsvb);
      const int nblk = (nS + rpb - 1) / rpb;
      for (int b = 0; b < (nblk > 1 ? nblk : 1); b++) {
        svec_block(C, B, d, nvb, seg, b, cf.nsvb);
        __syncthreads();
      }
      control_b_body(B, d);
      __syncthreads();
    }
    if (newton_gate(st)) {
      if (dense) {
        if (!syrk_in_solve(st, d)) {   // else the solve assembles H itself
          for (int t = 0; t < ntri; t++) {
            syrk_block(B, d, t, 0, 1);
            __syncthreads();
          }
          syrk_reduce_block(B, d, 0, 1, 1);
          __syncthreads();
        }
        newton_gj_small_body(B, d);
        __syncthreads();
      } else {
        cg_setup_body(B, d);
        __syncthreads();
        while (cg_gate(st)) {
          if (B.W32) hvp_dot_block<true>(B, d, B.vec.cg_p, B.wq, 0, 1);
          else hvp_dot_block<false>(B, d, B.vec.cg_p, B.wq, 0, 1);
          __syncthreads();
          if (B.W32) hvp_acc_block<true>(B, d, B.vec.cg_p, B.wq, B.hpart, 0, 1, -1);
          else hvp_acc_block<false>(B, d, B.vec.cg_p, B.wq, B.hpart, 0, 1);
          __syncthreads();
          cg_update_body(B, d, 1);
          __syncthreads();
        }
        if (newton_gate(st)) {
          cg_finish_body(B, d);
          __syncthreads();
        }
      }
    }
    if (batch_outer_gate(st)) {
      mult_rows_block(C, B, d, 0, 1);
      __syncthreads();
      if (tid == 0) mult_flip(st);
      __syncthreads();
    }
    if (st->status != 0) break;
    if (tick >= G.max_ticks) {
      if (tid == 0) st->status = kStatusTickCap;
      __syncthreads();
      break;
    }
  }
  const int status = st->status;
  if (status == kStatusSupportCap || status == kStatusTickCap) {
    if (tid == 0) O->status = status;
    __syncthreads();
    return;
  }
  // final point, the radius lift (max-type value at c) and the active set
  final_point_body(B, d, I.c_out, scal + 2);
  __syncthreads();
  batch_feas(sF, B, I.c_out, 0.0, INFINITY, 2, 1, false, scal + 1, nullptr, nullptr, 0);
  const double r_out = scal[1];
  batch_feas(sF, B, I.c_out, r_out, G.P.active_theta * r_out, 1, 0, true, nullptr, cnt,
             I.act, I.act_cap);
  if (tid == 0) {
    O->r = r_out;
    O->r_alm = scal[2];
    O->kkt[0] = st->kkt[0];
    O->kkt[1] = st->kkt[1];
    O->kkt[2] = st->kkt[2] * sc;
    O->kkt[3] = st->kkt[3];
    O->kkt[4] = st->kkt[4] * sc;
    O->kkt_max = st->kkt_max;
    O->scale = sc;
    O->n_active = cnt[0];
    O->fp64_rows = st->n64_total;
    O->status = status == 1 ? 0 : 1;
    O->outer = st->outer;
    O->ssn = st->tot_ssn;
    O->cg = st->tot_cg;
    O->passes = st->tot_passes;
    O->backtracks = st->tot_bt;
    O->inverses = st->gj_inverses;
    O->fp64_solves = st->fp64_solves;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256, 1) k_batch(BatchArgs G) {
  __shared__ int s_j;
  if (G.per_item) {   // block j, item j, slot j
    const int j = blockIdx.x;
    if (j >= G.n) return;
    const BatchConfig cf = G.cfg[G.items[j].cfg];
    if (cf.half) batch_solve_one<true>(G, j, G.slots[j], cf);
    else batch_solve_one<false>(G, j, G.slots[j], cf);
    return;
  }
  const Buffers& B = G.slots[blockIdx.x];
  for (;;) {
    if (threadIdx.x == 0) s_j = atomicAdd(G.next, 1);
    __syncthreads();
    const int j = s_j;
    __syncthreads();
    if (j >= G.n) return;
    const BatchConfig cf = G.cfg[G.items[j].cfg];
    if (cf.half) batch_solve_one<true>(G, j, B, cf);
    else batch_solve_one<false>(G, j, B, cf);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side: the scratch of one block (the arrays of Buffers a solve of an
// instance with at most m_cap balls in d_cap dimensions touches, with room
// for sup_cap support rows), laid out in one arena.
size_t batch_slot_layout(Buffers* Bp, char* base, int64_t m_cap, int d_cap, int64_t sup_cap) {
  Buffers B{};
  size_t off = 0;
  auto take = [&](auto** p, size_t n) {
    using T = std::remove_reference_t<decltype(**p)>;
    off = (off + 255) & ~(size_t)255;
    if (base) *p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * (n ? n : 1);
  };
  const int64_t m_pad = ((m_cap + 255) / 256) * 256;
  const int64_t nbf = m_pad / 256;
  const int d4 = (d_cap + 3) / 4;
  const int n1 = d_cap + 1;
  // instances with d + 1 <= kGjRegN take the dense Newton solve whatever the
  // batch's largest d: room for the largest dense system and its SYRK tiles
  const int nd = n1 < kGjRegN ? n1 : kGjRegN;
  const int nt = (nd - 1 + kSyrkTile - 1) / kSyrkTile;
  const int64_t ntri = (int64_t)nt * (nt + 1) / 2;
  take(&B.X32, (size_t)d4 * m_pad);
  take(&B.X16, (size_t)((d4 + 1) / 2) * m_pad);
  take(&B.EPS16, m_pad);
  take(&B.E32, m_pad);
  take(&B.R32, m_pad);
  take(&B.Hhi, (size_t)nd * nd);
  take(&B.Hlo, (size_t)nd * nd);
  take(&B.Ainv, (size_t)kAinvLen);
  take(&B.H, (size_t)nd * nd);
  take(&B.slot, m_pad);
  for (int k = 0; k < 2; k++) {
    take(&B.sup_idx[k], sup_cap);
    take(&B.sup_u[k], sup_cap);
    take(&B.sup_v[k], (size_t)sup_cap * d_cap);
    take(&B.sup_vv[k], sup_cap);
  }
  take(&B.part_flag, kMaxPassBlocks);
  take(&B.part, (size_t)kMaxPassBlocks * P_NREC);
  take(&B.part_cnt, (size_t)kMaxPassBlocks * P_NCNT);
  take(&B.cand_off, kMaxPassBlocks + 1);
  take(&B.cand_cnt, kMaxPassBlocks);
  take(&B.unc_cnt, kMaxPassBlocks);
  take(&B.vlb_part, kMaxPassBlocks);
  take(&B.unc_idx, m_pad + 256);
  take(&B.cand_idx, m_pad + 256);
  take(&B.cand_case, m_pad + 256);
  take(&B.cand_a, m_pad + 256);
  take(&B.cand_n, m_pad + 256);
  take(&B.cand_u, m_pad + 256);
  take(&B.S_idx, sup_cap);
  take(&B.S_case, sup_cap);
  take(&B.S_a, sup_cap);
  take(&B.S_n, sup_cap);
  take(&B.S_u, sup_cap);
  take(&B.S_t, sup_cap);
  take(&B.W, (size_t)sup_cap * d_cap);
  if (n1 > kGjRegN) take(&B.W32, (size_t)sup_cap * d_cap);   // CG instances: FP32 rows
  take(&B.svec_part, (size_t)kBatchMaxSvec * (3 * d_cap + 1));
  const size_t hp = (size_t)ntri * kSyrkTile * kSyrkTile;
  take(&B.hpart, hp > (size_t)n1 ? hp : (size_t)n1);
  take(&B.colsum_part, (size_t)((m_cap + kShadowBalls - 1) / kShadowBalls) * d_cap);
  take(&B.fe_ub, m_pad);
  take(&B.fe_lb, m_pad);
  take(&B.fe_blb, nbf);
  take(&B.fe_L, 4);
  take(&B.fq_y32, (size_t)4 * d4 + 4);
  take(&B.feas_part, nbf + 8);
  take(&B.feas_ipart, nbf + 8);
  take(&B.feas_cnt, nbf + 8);
  take(&B.list_tmp, m_pad);
  take(&B.count64, 8);
  take(&B.scal, 8);
  take(&B.wq, sup_cap);
  take(&B.cf32, sup_cap);
  take(&B.st, 1);
  const size_t stride = (size_t)((n1 + 8 + 1) / 2) * 2;
  take(&B.vec_store, 20 * stride + (size_t)(d4 * 4 + 8));
  if (base) {
    double* p = B.vec_store;
    auto vtake = [&](double** q) { *q = p; p += stride; };
    vtake(&B.vec.x); vtake(&B.vec.xt); vtake(&B.vec.xk); vtake(&B.vec.ab); vtake(&B.vec.g);
    vtake(&B.vec.gt); vtake(&B.vec.dx); vtake(&B.vec.ct); vtake(&B.vec.o); vtake(&B.vec.c0);
    vtake(&B.vec.sv); vtake(&B.vec.sw); vtake(&B.vec.st1); vtake(&B.vec.cg_r); vtake(&B.vec.cg_z);
    vtake(&B.vec.cg_p); vtake(&B.vec.cg_ap); vtake(&B.vec.cg_diag);
    B.vec.y32 = reinterpret_cast<float*>(p);
    B.m_cap = m_cap;
    B.d_cap = d_cap;
    B.nblk_cap = nbf;
    B.hpart_cap = (int64_t)(hp > (size_t)n1 ? hp : (size_t)n1);
    *Bp = B;
  }
  return (off + 255) & ~(size_t)255;
}

// Dynamic shared memory of the batch kernel for instances up to d_cap: the
// largest of the screen's query row, the FP64 rows' centre, the feasibility
// sweeps' query, and (dense Newton) the FP64 Cholesky fallback's factor.
size_t batch_smem(int d_cap) {
  const int d4 = (d_cap + 3) / 4;
  size_t sh = 16 * (size_t)(2 * ((d4 + 1) / 2));
  sh = sh > 8 * (size_t)d_cap ? sh : 8 * (size_t)d_cap;
  sh = sh > 16 * (size_t)d4 ? sh : 16 * (size_t)d4;
  const int n = d_cap + 1;
  const int nd = n <= kGjRegN ? n : kGjRegN;   // larger d take the CG path
  const size_t chol = sizeof(double) * (size_t)nd * (nd + 1) / 2;
  return sh > chol ? sh : chol;
}

cudaError_t launch_batch(const BatchArgs& G, int nblocks, size_t smem, cudaStream_t s) {
  cudaError_t e = raise_smem_limit((const void*)k_batch, smem);
  if (e != cudaSuccess) return e;
  k_batch<<<nblocks, 256, smem, s>>>(G);
  return cudaGetLastError();
}

int batch_blocks_per_sm(size_t smem) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, 256, smem);
  return per;
}

}  // namespace meb
