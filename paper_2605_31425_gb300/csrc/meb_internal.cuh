// Internal declarations shared by the kernels and the C-ABI layer of libmeb.
//
// All solver state lives in device memory (DevState plus the vectors it
// points to); the kernels read and write it, and the host only launches and
// reads back the small action/status fields.
#pragma once
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "../../include/meb.h"

namespace meb {

constexpr int kPassThreads = 256;   // balls per pass block (one per thread)
constexpr int kPassWarps = kPassThreads / 32;
constexpr int kMaxDenseN = 225;     // dense Newton solve for d+1 <= 225 (packed FP64 in smem)
constexpr int kAinvMaxN = 112;      // n = d + 1 of the register Gauss-Jordan solve
constexpr int kAinvLen = 28 * 256;  // float2 entries of its kept FP32 inverse
constexpr int kSvecBlocks = 152;    // blocks of the support-row reduction (one per SM)
constexpr int kSvecBlocksWide = 456;   // the same for rows of d >= 512 (three per SM)
constexpr int kSyrkTile = 32;
constexpr int kSyrkRows = 32;       // support rows per SYRK block

// ball case of the projection onto Q_{d+1}
enum : int { CASE_Z = 0, CASE_I = 1, CASE_M = 2 };

// controller actions
enum : int {
  ACT_NONE = 0,
  ACT_NEWTON = 1,   // assemble H / run CG at the accepted point, then a trial pass
  ACT_TRIAL = 2,    // a new trial point is set (backtrack); next is a pass
  ACT_OUTER = 3,    // outer step: multiplier update, then a pass at x
  ACT_DONE = 4,
  ACT_GRAD = 5,     // trial accepted (or first evaluation): reduce the support rows
  ACT_TRIAL_EARLY = 6,  // trial rejected from the certified lower bound; next trial set
};

// DevState::status: 0 running, 1 converged, 2 iteration cap, 3 a device wait
// gave up (a bulk copy did not complete in time)
constexpr int kStatusWaitTimeout = 3;
constexpr int kStatusTickCap = 4;   // the while-node loop reached its tick cap
constexpr int kStatusSupportCap = 5;   // batched solver: the support outgrew its slot's rows

// per-block partial record of the pass (doubles)
enum : int {
  P_PI2 = 0,   // sum ||Pi(z_i)||^2
  P_SU,        // sum u_i^+
  P_DUV2,      // sum ||(u,v)_i^+ - (u,v)_i||^2
  P_UV2,       // sum ||(u,v)_i||^2 over the current multipliers
  P_ZMAG,      // sum_{I,M} |a_i| + ||b_i||
  P_KP,        // max primal distance to Q
  P_KD,        // max dual distance to Q
  P_KC,        // max complementarity
  P_NI,        // count of case I
  P_NM,        // count of case M
  P_N64,       // rows evaluated in FP64
  P_COUNT
};
// block partial records: P_NREC doubles (the sums P_PI2..P_ZMAG, then the
// maxima P_KP..P_KC) in part[], the three counts as ints in part_cnt[]
constexpr int P_NSUM = 5, P_NREC = 8, P_NCNT = 3;
constexpr int kMaxPassBlocks = 2048;   // cap of the pass grid (controller lists)

struct DevState {
  // problem
  int64_t m, m_pad;
  int d, d4, n1;
  int dense;              // 1: dense Cholesky, 0: CG
  double s, inv_s;        // power-of-two scale
  double sh_s, sh_inv_s;  // scale of the FP16 shadow (s in solves; any power of two in evaluations)
  // parameters (scaled problem)
  double tol, rho, sigma_max, sigma_growth, sigma_ratio, tau, mu;
  double rnd;   // rounding unit of the per-ball rows (FP64, or the FP32 low-precision run)
  int max_outer, max_ssn, max_backtrack, max_cg;
  // iteration state
  double sigma, inv_sigma;
  double tos;                  // tau / sigma
  double psi, psi_mag, gmag;   // at the accepted point x
  double gdx, eta;
  double pinf_prev;
  int outer, ssn_j, bt;
  int tot_ssn, tot_passes, tot_bt, tot_cg;
  int phase;                   // 0: pass evaluates x^k (outer start); 1: a line-search trial
  int action, status;          // status: 0 running, 1 converged, 2 iteration cap
  int sup_cur, nsup;           // current multiplier buffers and their size
  int nS;                      // support (cases I, M) of the last evaluated point
  int svec_nb, svec_rpb;       // blocks / rows per block of the support reduction
  double sigma_prev;           // sigma of the finished outer step (multiplier update)
  int64_t n64_total;
  int chol_fail, eval_only;
  int accept_mode;             // 1: accepted, go to the stop test; 2: accepted, outer forced
  int need_fp64_solve;         // FP32 inverse + refinement failed: FP64 Cholesky
  int force_fp64_solve;        // every dense Newton system by the FP64 Cholesky
  int fp64_solves;             // count of FP64 Cholesky fallbacks
  int gj_inverses;             // count of FP32 Gauss-Jordan inverses
  int gj_reuses;               // Newton systems solved with the kept inverse
  int inv_valid;               // Buffers::Ainv holds the inverse of an H at sigma = kept_sigma
  double kept_sigma;
  int early_rejects;           // trials rejected by the certified lower bound
  int reuse_lists;             // next pass: same point, new multipliers (skip the screen)
  int64_t ticks, max_ticks;    // controller ticks of the device-resident loop and their cap
  int64_t cg_bodies;           // runs of the CG loop body in the tick graph (launch count)
  int screen_log[8];           // profiling: tick t of a graph batch ran a full screen
  unsigned int ctr_screen, ctr_rows, ctr_svec, ctr_slots, ctr_svecr;   // last-block-done tickets
  int screens;                 // full FP32 screens run
  double dx2_t;                // ||xt - xk||^2 of the trial (set with the trial)
  double kkt[5], kkt_max;
  double last[P_COUNT];        // reduced partials of the last pass
  // trial point shadow for the FP32 screen
  double rt_abs;               // trial radius, unscaled
  float rq32, yn32;            // fl32(r_t), an upper bound on ||y32||
  // CG scratch scalars
  double cg_rz, cg_bn, cg_rtol;
  int cg_it, cg_done;
};

// Device vectors of length n1 = d+1 (scaled units unless noted) and more.
struct DevVecs {
  double* x;      // accepted point
  double* xt;     // trial point
  double* xk;     // proximal centre x^k
  double* ab;     // auxiliary (alpha, beta)
  double* g;      // gradient at x
  double* gt;     // gradient at the trial
  double* dx;     // Newton direction
  double* ct;     // trial centre, UNSCALED (c = s * xt[1:])
  double* o;      // origin of the FP32 shadow (the first centre), unscaled
  double* c0;     // initial centre (mean of the centres), unscaled
  float* y32;     // trunc32(ct - o), 4*d4 floats
  double* sv;     // sum of v^+ (d)
  double* sw;     // sum of w over case M (d)
  double* st1;    // [0]: sum_M (1 + t)
  // CG
  double* cg_r; double* cg_z; double* cg_p; double* cg_ap; double* cg_diag;
};

struct Buffers {
  int64_t launches;     // host-side count of kernels launched through these buffers
  const double* C_in;   // centres of the current call (device)
  int64_t m_cap;
  int d_cap;
  int64_t nblk_cap;
  // shadow
  float4* X32;          // [d4][m_pad]
  uint4* X16;           // [ceil(d4/2)][m_pad] FP16 shadow scaled by 1/s (meb_solve)
  float* EPS16;         // [m_pad] per ball: bound eps_i on ||x_i/s - x16_i|| (scaled units)
  float* E32;           // [m_pad] per ball: absolute part E_i of the FP32 shadow error
  float* Hhi;           // [n1 x n1] fl32(H)
  float* Hlo;           // [n1 x n1] fl32(H - Hhi)
  float2* Ainv;         // [kAinvLen] the last FP32 inverse of H (register layout of the
                        // n <= 112 Gauss-Jordan solve); null: none kept
  bool use_x16;         // host side: the screens read X16
  bool bulk;            // host side: FP16 screens through the bulk-copy pipeline
  bool fp64_all;        // host side: no shadow is read; every ball goes through the FP64 rows
  bool lowp;            // host side: rows, support rows and multiplier rows in FP32 from the
                        // FP32 shadow (the low-precision run of the mixed-precision pipeline)
  long long wait_cycles;   // bound of the bulk-copy screen's waits (SM clock cycles; 0: one test)
  float* R32;           // [m_pad]
  // multipliers (double buffered)
  int* slot;            // [m]
  int* sup_idx[2];      // [m]
  double* sup_u[2];     // [m]
  double* sup_v[2];     // [m*d]
  double* sup_vv[2];    // [m] ||v_k||^2, lane-strided FMAs then a warp tree (as the rows sum it)
  // pass outputs
  int* part_flag;       // [nblk]
  int* part_cnt;        // [nblk][P_NCNT]
  int* cand_off;        // [nblk + 1] start of each pass block's candidates in S
  double* part;         // [nblk][P_COUNT]
  int* unc_cnt;         // [nblk] balls each pass block could not certify
  int* unc_idx;         // [ncand] their indices (per-block segments)
  int* unc_slot;        // [ncand] their multiplier slots (-1: none)
  float* vlb_part;      // [nblk] lower-bound partials of the early rejection
  int* cand_cnt;        // [nblk]
  int* cand_idx;        // [m_pad]
  unsigned char* cand_case;
  double* cand_a; double* cand_n; double* cand_u;
  // support list of the last pass (ball order)
  int* S_idx; unsigned char* S_case; double* S_a; double* S_n; double* S_u; double* S_t;
  double* W;            // [m*d] w rows (case M) / b rows (case I)
  float* W32;           // [m*d] the same in FP32 for the CG products (matrix-free path), or null
  double* svec_part;    // [kSvecBlocks or kSvecBlocksWide][3d+1]
  double* hpart;        // SYRK partials
  int64_t hpart_cap;
  double* H;            // [n1*n1] assembled Hessian (eval entry / CG diag)
  double* hq;           // [n1] Hessian-vector product
  double* colsum_part;  // mean-centre partials
  float* fe_ub;         // [m] certified upper bound on r_i + ||c - c_i||
  float* fe_lb;         // [m] certified lower bound
  float* fe_blb;        // [nblk] block maxima of the lower bounds
  float* fe_L;          // [4] max lower bound, query norm bound
  float* fq_y32;        // [4*d4] query shadow of the feasibility pass
  double* feas_part;    // feasibility partials
  int64_t* feas_ipart;
  int* feas_cnt;        // [nblk]
  int64_t* viol;        // [m] compacted indices
  int64_t* list_tmp;    // [m_pad] per-tile lists before compaction
  int64_t* count64;     // [4] device counters
  double* wq;           // [m] w_k . q of the Hessian-vector product
  float* cf32;          // [m] FP32 products: -t_k (w_k . q) / 2 for case M, else 0
  double* scal;         // [8] scalars of the batched solver (r0, r_out, r_alm)
  DevState* st;
  DevVecs vec;
  double* vec_store;
};

// The controller's state at the start of a solve (host or device): problem
// sizes, the parameters of Algorithms 1 and 2 on the scaled problem (scale s),
// the initial penalty; everything else zero.  dense: 1 for the dense Newton
// solve, 0 for CG.
__host__ __device__ inline void state_defaults(DevState& S, int64_t m, int d, const meb_params& P,
                                               double s, int dense) {
  unsigned* w = reinterpret_cast<unsigned*>(&S);
  for (size_t k = 0; k < sizeof(DevState) / 4; k++) w[k] = 0u;
  S.m = m;
  S.m_pad = ((m + 255) / 256) * 256;
  S.d = d;
  S.d4 = (d + 3) / 4;
  S.n1 = d + 1;
  S.dense = dense;
  S.force_fp64_solve = P.newton_fp64 != 0;
  S.s = s;
  S.inv_s = 1.0 / s;
  S.sh_s = s;
  S.sh_inv_s = 1.0 / s;
  S.tol = P.tol;
  S.rho = P.rho;
  S.sigma_max = P.sigma_max;
  S.sigma_growth = P.sigma_growth;
  S.sigma_ratio = P.sigma_ratio;
  S.tau = P.tau;
  S.mu = P.armijo_mu;
  S.rnd = DBL_EPSILON;
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

// Raise (never lower) a kernel's dynamic shared-memory limit; thread-safe.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
// Record / read the last failed launch of this host thread.
void note_launch_failure(const char* what, unsigned grid, size_t smem, cudaError_t e);
const char* launch_failure_note();

// ---- the batched solver (meb_batch.cu) ----
constexpr int kBatchMaxSvec = 16;   // support-row blocks of one batched solve, at most

// One instance of a batch, device view (pointers on the device).
struct BatchItemDev {
  const double* C;
  const double* R;
  int64_t m;
  int d;
  int cfg;             // index of its configuration
  double* c_out;       // [d]
  int64_t* act;        // [act_cap] ascending active indices
  int64_t act_cap;
  int64_t sup_cap;     // support rows it may use: min(m, max(2048, 16 (d + 1)))
};

// Support rows a batched solve of (m, d) may hold (a function of the instance
// alone, so that the choice to fall back never depends on the rest of a batch).
__host__ __device__ inline int64_t batch_support_cap(int64_t m, int d) {
  const int64_t c = 16 * (int64_t)(d + 1) > 2048 ? 16 * (int64_t)(d + 1) : 2048;
  return m < c ? m : c;
}

// Execution choices of one class of instances (picked by the tuner).
struct BatchConfig {
  int half;            // 1: screen the FP16 shadow, 0: the FP32 shadow
  int tiles_per_vb;    // tiles of 256 balls per pass block
  int nsvb;            // blocks of the support-row reduction (<= kBatchMaxSvec)
  int pad;
};

// Results of one instance (the fields of meb_info).
struct BatchOut {
  double r, r_alm, kkt[5], kkt_max, scale;
  int64_t n_active, fp64_rows;
  int32_t status;      // 0 converged, 1 cap, -1 invalid input, kStatusSupportCap, kStatusTickCap
  int32_t outer, ssn, cg, passes, backtracks, inverses, fp64_solves;
};

struct BatchArgs {
  const BatchItemDev* items;   // in queue order (largest first)
  BatchOut* out;
  int n;
  int* next;                   // queue head (zero before the launch)
  const Buffers* slots;        // one per thread block (per item when per_item)
  const BatchConfig* cfg;
  meb_params P;
  int64_t max_ticks;
  int per_item;                // 1: block j solves item j with slot j (no queue)
};

size_t batch_slot_layout(Buffers* B, char* base, int64_t m_cap, int d_cap, int64_t sup_cap);
size_t batch_smem(int d_cap);
int batch_blocks_per_sm(size_t smem);
cudaError_t launch_batch(const BatchArgs& G, int nblocks, size_t smem, cudaStream_t s);

// ---- launch wrappers: streaming kernels (meb_pass.cu) ----
// Launch of a controller-tick kernel with programmatic dependent launch: the
// kernel may be scheduled while its predecessor in the stream finishes; it
// waits (griddepcontrol.wait, pdl_wait) for the predecessor's completion and
// memory before it reads anything.  In a captured graph the dependency
// becomes a programmatic edge.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// screen kernels: 0 FP32 shadow, 1 FP16 shadow (register batches),
// 2 FP16 shadow through a bulk-copy (TMA) pipeline in shared memory,
// 3 no shadow (every ball listed for the FP64 rows: the plain FP64 pass)
int screen_variant(const Buffers& B, int d);
int pass_blocks(int64_t m, int d, int variant, int* tiles_per_block);
cudaError_t prepare_pass(const Buffers& B, int d);
cudaError_t launch_shadow(const double* C, const double* R, int64_t m, int d, Buffers& B,
                          double* o, double* c0, int* bad, cudaStream_t s);
// The two halves of launch_shadow: the sweep over the shadow blocks
// [b0, b1) (64 balls each; rows of those balls only are read) and the mean
// centre once every block has run.
constexpr int kShadowBallsPerBlock = 64;
cudaError_t launch_shadow_blocks(const double* C, const double* R, int64_t m, int d, Buffers& B,
                                 int64_t b0, int64_t b1, int* bad, cudaStream_t s);
cudaError_t launch_shadow_mean(const double* C, int64_t m, int d, Buffers& B, double* o,
                               double* c0, cudaStream_t s);
cudaError_t launch_shadow16(Buffers& B, int64_t m, int d, double inv_s, cudaStream_t s);
cudaError_t launch_pass(const double* C, const double* R, Buffers& B, int64_t m, int d,
                        cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                        int log_slot = -1);
cudaError_t launch_support_rows(const double* C, Buffers& B, int64_t m, int d, cudaStream_t s);
cudaError_t launch_feas_cert(const double* C, const double* R, int64_t m, int d, const double* c,
                             double r, double eps, int mode, int want_max, Buffers& B,
                             double* dmax_out, int64_t* argmax_out, int64_t* nviol_out,
                             cudaStream_t s, bool reuse_bounds = false, int* bad = nullptr);
cudaError_t launch_support_from_dense(const double* U, const double* V, Buffers& B, int64_t m,
                                      int d, cudaStream_t s);
// ---- launch wrappers: solver kernels (meb_solve.cu) ----
cudaError_t launch_tick_control(Buffers& B, int64_t m, int d, cudaStream_t s);
cudaError_t launch_newton_dense(Buffers& B, int d, cudaStream_t s);
int newton_dense_launches(int d);
cudaError_t prepare_newton(int d);
cudaError_t launch_cg_setup(Buffers& B, int d, cudaStream_t s);
cudaError_t launch_cg_iter(Buffers& B, int64_t m, int d, cudaStream_t s);
cudaError_t launch_cg_finish(Buffers& B, int d, cudaStream_t s);
cudaError_t launch_mult_update(const double* C, Buffers& B, int64_t m, int d, cudaStream_t s);
cudaError_t launch_state_init(Buffers& B, int d, cudaStream_t s);
cudaError_t launch_eval_outputs(const double* C, Buffers& B, int64_t m, int d, const double* q,
                                double* Uplus, double* Vplus, double* Hq, double* H,
                                cudaStream_t s);
cudaError_t launch_eval_prepare(Buffers& B, const double* x, const double* xbar, int d,
                                cudaStream_t s);
cudaError_t launch_final_point(Buffers& B, int d, double* c_out, double* r_alm, cudaStream_t s);
cudaError_t launch_mult_out(Buffers& B, int d, int64_t* idx, double* u, double* v, int64_t cap,
                            cudaStream_t s);
cudaError_t launch_gather_rows(const double* C, const double* R, const int64_t* idx, int64_t n,
                               int d, double* Cr, double* Rr, cudaStream_t s);
cudaError_t launch_warm_start(Buffers& B, int d, const double* wx, double sigma,
                              const int64_t* widx, const double* wu, const double* wv, int64_t nw,
                              const int64_t* ired, int64_t nred, cudaStream_t s);
cudaError_t launch_map_idx(int64_t* idx, int64_t n, const int64_t* map, cudaStream_t s);
cudaError_t launch_loop_cond(Buffers& B, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_cg_cond(Buffers& B, cudaGraphConditionalHandle h, cudaStream_t s);
bool support_rows_wide(const Buffers& B, int d);   // support rows over kSvecBlocksWide blocks

}  // namespace meb
