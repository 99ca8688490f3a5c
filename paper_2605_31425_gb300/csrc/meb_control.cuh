// The controller of Algorithms 1 and 2 as block-level device functions.  Each
// runs in the last block of the kernel that produced its inputs (the block
// that takes the last ticket after every block has fenced its writes), so the
// decisions need no kernel launch of their own.  Vector work (length d + 1)
// is spread over the block's 256 threads.
#pragma once
#include "meb_common.cuh"

namespace meb {

// Last-block-done: after a barrier (which makes the block's writes visible
// to thread 0), thread 0 fences at GPU scope (the fence is cumulative, so it
// orders those writes too) and takes a ticket; the block holding the last
// ticket returns true (after an acquire fence) and resets the counter for
// the next launch.
__device__ __forceinline__ bool last_block_ticket(unsigned int* ctr) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(ctr, 1u);
    s_last = (t == gridDim.x - 1);
    if (s_last) *ctr = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// The controller bodies work on a shared-memory copy of the state: its
// scalar logic then waits on shared-memory latency instead of one global
// round trip per field.  No other block of the kernel touches the state
// while the last block runs; the copy is written back whole.
__device__ __forceinline__ DevState* state_in(DevState* g, DevState* s) {
  static_assert(sizeof(DevState) % 4 == 0, "state copied as 32-bit words");
  const unsigned* src = reinterpret_cast<const unsigned*>(g);
  unsigned* dst = reinterpret_cast<unsigned*>(s);
  for (int k = threadIdx.x; k < (int)(sizeof(DevState) / 4); k += blockDim.x)
    dst[k] = __ldcg(src + k);
  __syncthreads();
  return s;
}
__device__ __forceinline__ void state_out(DevState* g, const DevState* s) {
  __syncthreads();
  const unsigned* src = reinterpret_cast<const unsigned*>(s);
  unsigned* dst = reinterpret_cast<unsigned*>(g);
  for (int k = threadIdx.x; k < (int)(sizeof(DevState) / 4); k += blockDim.x) dst[k] = src[k];
}

// Outer update (Algorithm 1): (alpha,beta) -= sigma g, KKT_max, sigma rule.
// Returns the action; thread 0 writes the state.
__device__ __forceinline__ void do_outer(DevState* st, const DevVecs& V, int d, double* sh) {
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
        st->tos = st->tau / sg;
      }
      st->pinf_prev = pinf;
      st->phase = 0;
      st->reuse_lists = 1;
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

// Early line-search rejection (the last block of k_screen): from the screen's certified lower
// bound Psi_lb <= Psi(trial) (only balls with zero multipliers counted), a
// trial with Psi_lb above the Armijo threshold is rejected without its FP64
// rows; the next trial is set as in the controller.
__device__ __forceinline__ void early_body_impl(const Buffers& B, DevState* st, int d, int nb) {
  if (st->phase != 1 || st->eval_only) {
    if (threadIdx.x == 0 && st->action == ACT_TRIAL_EARLY) st->action = ACT_TRIAL;
    return;
  }
  __shared__ double sh[32];
  __shared__ float shf[8];
  __shared__ int s_rej;
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  // FP32 sum of the non-negative block bounds (its relative rounding, below
  // nb 2^-24, is inside the 1% kept below)
  float tf = 0.0f;
  for (int b = threadIdx.x; b < nb; b += 256) tf += B.vlb_part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tf += __shfl_xor_sync(MEB_FULLMASK, tf, o);
  if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = tf;
  __syncthreads();
  float tsum = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; k++) tsum += shf[k];
  const double t = (double)tsum;
  const double dx2 = st->dx2_t;
  if (threadIdx.x == 0) {
    const double sigma = st->sigma, tos = st->tos;
    // FP32 sums of nonnegative terms: keep 1% for their rounding
    const double pi2_lb = 0.99 * t * st->inv_s * st->inv_s * 0.5;
    const double psi_lb = V.xt[0] + 0.5 * sigma * pi2_lb + 0.5 * tos * dx2;
    const double mag = fabs(V.xt[0]) + 0.5 * sigma * pi2_lb + 0.5 * tos * dx2;
    const double allow = 64.0 * st->rnd * fmax(st->psi_mag, mag);
    const double thr = st->psi + st->mu * st->eta * st->gdx + allow;
    int rej = 0;
    if (psi_lb > thr && st->bt < st->max_backtrack) {
      const double eta = st->eta;
      const double den = 2.0 * (psi_lb - st->psi - st->gdx * eta);
      double en = (den > 0.0) ? -st->gdx * eta * eta / den : 0.5 * eta;
      en = fmin(fmax(en, 0.1 * eta), 0.5 * eta);
      st->eta = en;
      st->bt += 1;
      st->tot_bt += 1;
      st->tot_passes += 1;
      st->early_rejects += 1;
      st->last[P_N64] = 0.0;
      st->action = ACT_TRIAL_EARLY;
      rej = 1;
    } else if (st->action == ACT_TRIAL_EARLY) {
      st->action = ACT_TRIAL;   // the trial set by the previous early rejection is evaluated
    }
    s_rej = rej;
  }
  __syncthreads();
  if (s_rej) {
    const double eta = st->eta;
    for (int k = threadIdx.x; k < n1; k += 256) V.xt[k] = V.x[k] + eta * V.dx[k];
    __syncthreads();
    set_trial(st, V, d, sh);
  }
}

__device__ __forceinline__ void early_body(const Buffers& B, int d, int nb) {
  __shared__ DevState s_st;
  DevState* st = state_in(B.st, &s_st);
  early_body_impl(B, st, d, nb);
  state_out(B.st, st);
}

// Controller, part A (the last block of k_rows64): reduce the pass partials,
// form Psi at the trial and take the line-search decision (Algorithm 2).  A rejected trial
// sets the next trial directly; an accepted one (or the first evaluation of an
// outer step) asks for the gradient: action ACT_GRAD.
__device__ __forceinline__ void control_a_body_impl(const Buffers& B, DevState* st, int d,
                                                    int nb) {
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ double sh[32];
  __shared__ double s_last[P_COUNT];
  __shared__ int s_next;
  __shared__ int s_list[kMaxPassBlocks];
  __shared__ int s_wc[8];
  {
    // the blocks that evaluated rows, in block order
    int nlist = 0;
    for (int r0 = 0; r0 < nb; r0 += 256) {
      const int b = r0 + threadIdx.x;
      const bool f = b < nb && B.part_flag[b];
      const unsigned msk = __ballot_sync(MEB_FULLMASK, f);
      if (lane == 0) s_wc[w] = __popc(msk);
      __syncthreads();
      int off = nlist, tot = 0;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        off += (k < w) ? s_wc[k] : 0;
        tot += s_wc[k];
      }
      if (f) s_list[off + __popc(msk & ((1u << lane) - 1u))] = b;
      nlist += tot;
      __syncthreads();
    }
    // warps 0..4: the FP64 sums; warps 5..7: the maxima (on bit patterns) and
    // the counts.  Lanes stride over the list, then a fixed warp tree.
    if (w < P_NSUM) {
      double t = 0.0;
      for (int e = lane; e < nlist; e += 32) t += B.part[(int64_t)s_list[e] * P_NREC + w];
      t = warp_sum(t);
      if (lane == 0) s_last[w] = t;
    } else {
      long long mx = 0;
      unsigned c = 0;
      for (int e = lane; e < nlist; e += 32) {
        const long long b = __double_as_longlong(B.part[(int64_t)s_list[e] * P_NREC + w]);
        mx = b > mx ? b : mx;
        c += (unsigned)B.part_cnt[(int64_t)s_list[e] * P_NCNT + (w - P_NSUM)];
      }
      const double m = warp_max_nonneg(__longlong_as_double(mx));
      c = __reduce_add_sync(MEB_FULLMASK, c);
      if (lane == 0) {
        s_last[w] = m;
        s_last[P_NI + (w - P_NSUM)] = (double)c;
      }
    }
    __syncthreads();
  }
  const double sigma = st->sigma, tos = st->tos;
  const double dx2 = st->dx2_t;
  const double psi_t = V.xt[0] + 0.5 * sigma * s_last[P_PI2] + 0.5 * tos * dx2;
  const double mag_t = fabs(V.xt[0]) + 0.5 * sigma * s_last[P_PI2] + 0.5 * tos * dx2;
  if (threadIdx.x == 0) {
    for (int k = 0; k < P_COUNT; k++) st->last[k] = s_last[k];
    if (!st->reuse_lists) st->screens += 1;
    st->reuse_lists = 0;
    st->tot_passes += 1;
    st->n64_total += (int64_t)s_last[P_N64];
    int nxt = 0;   // 0: gradient at the (accepted) trial; 1: backtrack
    if (st->eval_only) {
      st->psi = psi_t - s_last[P_UV2] / (2.0 * sigma);
      st->accept_mode = 0;
    } else if (st->phase == 1) {
      const double allow = 64.0 * st->rnd * fmax(st->psi_mag, mag_t);
      const bool ok = psi_t <= st->psi + st->mu * st->eta * st->gdx + allow;
      if (ok || st->bt >= st->max_backtrack) {
        st->psi = psi_t; st->psi_mag = mag_t;
        st->ssn_j += 1;
        st->tot_ssn += 1;
        st->accept_mode = (!ok || st->ssn_j >= st->max_ssn) ? 2 : 1;   // 2: outer forced
      } else {
        // next step: minimiser of the quadratic through Psi(0), Psi'(0), Psi(eta),
        // kept in [eta/10, eta/2]
        const double eta = st->eta;
        const double den = 2.0 * (psi_t - st->psi - st->gdx * eta);
        double en = (den > 0.0) ? -st->gdx * eta * eta / den : 0.5 * eta;
        en = fmin(fmax(en, 0.1 * eta), 0.5 * eta);
        st->eta = en;
        st->bt += 1;
        st->tot_bt += 1;
        nxt = 1;
      }
    } else {
      st->psi = psi_t; st->psi_mag = mag_t;
      st->ssn_j = 0;
      st->accept_mode = 1;
    }
    st->action = nxt ? ACT_TRIAL : ACT_GRAD;
    s_next = nxt;
  }
  __syncthreads();
  if (s_next == 1) {
    const double eta = st->eta;
    for (int k = threadIdx.x; k < n1; k += 256) V.xt[k] = V.x[k] + eta * V.dx[k];
    __syncthreads();
    set_trial(st, V, d, sh);
    if (threadIdx.x == 0) st->phase = 1;
  } else {
    // the support S of the accepted point is the concatenation of the pass
    // blocks' candidate segments: their start offsets (exclusive prefix of
    // the counts, 8 per thread) and |S|
    __shared__ int s_tot[8];
    int v[8], run = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int b = 8 * threadIdx.x + q;
      v[q] = (b < nb) ? B.cand_cnt[b] : 0;
      run += v[q];
    }
    int incl = run;   // inclusive scan of the thread totals: warp, then warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(MEB_FULLMASK, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_tot[w] = incl;
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      base += (q < w) ? s_tot[q] : 0;
      total += s_tot[q];
    }
    int off = base + incl - run;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int b = 8 * threadIdx.x + q;
      if (b < nb) B.cand_off[b] = off;
      off += v[q];
    }
    if (threadIdx.x == 0) {
      B.cand_off[nb] = total;
      st->nS = total;
    }
  }
}

__device__ __forceinline__ void control_a_body(const Buffers& B, int d, int nb) {
  __shared__ DevState s_st;
  DevState* st = state_in(B.st, &s_st);
  control_a_body_impl(B, st, d, nb);
  state_out(B.st, st);
}

// Entry e of the 3d + 1 sums over the support blocks' partials (in block
// order): sum v^+ (d), sum w (d), sum t w^2 (d), sum (1 + t).
__device__ __forceinline__ void svec_sum_entry(const Buffers& B, int d, int e, int snb) {
  const DevVecs& V = B.vec;
  const int nsum = 3 * d + 1;
  double a = 0.0;
  for (int k = 0; k < snb; k++) a += B.svec_part[(int64_t)k * nsum + e];
  if (e < d) V.sv[e] = a;
  else if (e < 2 * d) V.sw[e - d] = a;
  else if (e < 3 * d) V.cg_diag[1 + e - 2 * d] = a;   // sum_M t w_j^2 (Jacobi preconditioner)
  else V.st1[0] = a;
}

// Controller, part B (the last block of k_svec, or of k_svec_reduce when that
// kernel summed the partials: `reduced`): the gradient at the accepted point,
// then the relative-type stopping condition (Algorithm 1) and the next action.
__device__ __forceinline__ void control_b_body_impl(const Buffers& B, DevState* st, int d,
                                                    bool reduced = false) {
  const DevVecs& V = B.vec;
  const int n1 = d + 1;
  __shared__ double sh[32];
  if (!reduced) {
    const int snb = st->svec_nb;
    for (int e = threadIdx.x; e < 3 * d + 1; e += 256) svec_sum_entry(B, d, e, snb);
  }
  __syncthreads();
  const double sigma = st->sigma, tau = st->tau, tos = st->tos;
  const double su = st->last[P_SU];
  const bool eval_only = st->eval_only != 0;
  // the gradient at the trial; when it is accepted (not eval_only): x <- xt,
  // g <- gt, and the terms of the stopping condition
  double la = 0.0, g2 = 0.0;
  for (int k = threadIdx.x; k < n1; k += 256) {
    const double xt = V.xt[k];
    const double dk = xt - V.xk[k];
    const double sk = (k == 0) ? su : V.sv[k - 1];
    const double gk = ((k == 0) ? 1.0 : 0.0) - sk + tos * dk;
    V.gt[k] = gk;
    if (!eval_only) {
      V.x[k] = xt;
      V.g[k] = gk;
      la += (V.ab[k] - xt) * gk;
      g2 += gk * gk;
    }
  }
  if (eval_only) {
    if (threadIdx.x == 0) { st->action = ACT_DONE; st->status = 1; }
    return;
  }
  if (threadIdx.x == 0) {
    st->gmag = 1.0 + sigma * st->last[P_ZMAG] + tos * sqrt(st->dx2_t);
    st->phase = 2;
  }
  __syncthreads();
  if (st->accept_mode == 2) {
    do_outer(st, V, d, sh);
    return;
  }
  const double2 lg = block_sum2(la, g2);
  la = lg.x;
  g2 = lg.y;
  const double dk2 = st->dx2_t;   // ||x - xk||^2 with x = xt
  const double lhs = 2.0 * sigma * fabs(la) + sigma * sigma * g2;
  const double rhs = st->rho * (st->last[P_DUV2] + tau * dk2);
  const bool stop = (lhs <= rhs) || (sqrt(g2) <= 8.0 * st->rnd * st->gmag);
  if (stop) {
    do_outer(st, V, d, sh);
    return;
  }
  if (threadIdx.x == 0) {
    st->action = ACT_NEWTON;
    st->bt = 0;
  }
}

__device__ __forceinline__ void control_b_body(const Buffers& B, int d, bool reduced = false) {
  __shared__ DevState s_st;
  DevState* st = state_in(B.st, &s_st);
  control_b_body_impl(B, st, d, reduced);
  state_out(B.st, st);
}

}  // namespace meb
