/*
 * meb.h -- C ABI of libmeb: the ripALM minimum-enclosing-ball hot path on one
 * GB300 GPU (sm_103a).
 *
 * Problem (Sec. 1, eq. (MEB)): given m balls B(c_i, r_i) in R^d, find the
 * centre c and the smallest radius r with ||c - c_i|| + r_i <= r for all i.
 * Method: the SOCP form of Sec. 2 (one second-order-cone constraint
 * (r - r_i, c - c_i) in Q_{d+1} per ball), solved by the relative-type
 * inexact proximal augmented Lagrangian method (Algorithm 1, ripALM) with the
 * semismooth Newton inner solver of Algorithm 2, and the a-posteriori
 * feasibility pass of Sec. 4.2.
 *
 * Conventions for every entry point:
 *  - Return 0 on success, a negative MEB_E* code otherwise; no exception
 *    crosses the ABI.  meb_last_error() gives a one-line message.
 *  - Arrays are FP64 unless stated: centres are m x d row-major, radii m.
 *  - flags & MEB_PTR_DEVICE: every array argument is a device pointer on the
 *    context's device; otherwise every array argument is a host pointer and
 *    the library copies it in (and results out) on the context's stream.
 *    Scalar outputs (psi, delta_max, argmax, counts, n_viol, info) are always
 *    host pointers.
 *  - The caller owns every buffer it passes; the library never keeps a
 *    pointer past the call.  The context owns its device scratch (grown on
 *    demand, freed by meb_destroy).
 *  - A context is bound to one device and one stream; use one context per
 *    host thread.  Calls return after the work on the stream is complete.
 *  - Sizes: 1 <= m <= 2^31 - 257, 1 <= d <= 16384.
 */
#ifndef MEB_H
#define MEB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MEB_OK 0
#define MEB_EINVAL (-1)    /* bad size, NULL pointer, non-finite value, r_i < 0, tol <= 0 */
#define MEB_ENOMEM (-2)    /* device allocation failed                                    */
#define MEB_ECUDA (-3)     /* a CUDA call failed (message in meb_last_error)              */
#define MEB_ENOTCONV (-4)  /* iteration cap reached; outputs hold the last iterate        */
#define MEB_ETIMEOUT (-5)  /* a bounded device wait expired (a bulk copy did not land)    */

#define MEB_PTR_DEVICE 1u

typedef struct meb_ctx meb_ctx;

/* Parameters of Algorithms 1 and 2 on the scaled problem (data divided by the
 * power of two s >= r0, r0 = max_i ||c0 - c_i|| + r_i at the mean centre c0). */
typedef struct {
    double tol;          /* KKT_max tolerance (Sec. 5), scaled problem; default 1e-10 */
    double rho;          /* relative-error factor of Algorithm 1, [0,1); 0.5          */
    double sigma0;       /* initial penalty; 10                                        */
    double sigma_max;    /* cap on the penalty; 1e7                                    */
    double sigma_growth; /* sigma *= growth when the primal residual stalls; 10        */
    double sigma_ratio;  /* stall: residual > ratio * previous residual; 0.1           */
    double tau;          /* proximal weight (constant); 10                             */
    double armijo_mu;    /* Armijo sufficient-decrease constant; 1e-4                  */
    double active_theta; /* active set: r - r_i - ||c - c_i|| <= theta r; 2e-6          */
    int32_t max_outer;   /* 500 */
    int32_t max_ssn;     /* 50  */
    int32_t max_backtrack; /* 40 */
    int32_t dense_max_d; /* dense Cholesky Newton solve when d <= this (<= 224); 224    */
    int32_t max_cg;      /* CG iterations per Newton system (d > dense_max_d); 500,
                            at most 20,000 (the device-side CG loop's bound)        */
    int32_t newton_fp64; /* 1: solve every dense Newton system by the FP64 Cholesky   */
                         /* (the reference path; default 0: FP32 Gauss-Jordan with   */
                         /* refinement, FP64 Cholesky only as the fallback)          */
    /* The mixed-precision reduction pipeline of Sec. 4.2 (mixed = 1): a
     * low-precision ripALM (FP32 rows from the FP32 shadow) to tol_lp on all
     * balls; the reduced set I_red = {i : r - r_i - ||c - c_i|| <= tol_red r}
     * at its point (certified, plus every ball with a multiplier); the FP64
     * ripALM on I_red, warm-started from the low-precision point, penalty and
     * multipliers; then the FP64 feasibility pass over all balls, adding the
     * violated ones to I_red and solving again, at most max_readd times.  The
     * result is an FP64 solve to tol of the whole instance. */
    int32_t mixed;       /* 0 */
    int32_t max_readd;   /* 8 */
    double tol_lp;       /* KKT_max tolerance of the low-precision run; 1e-2 (Sec. 5) */
    double tol_red;      /* relative screening threshold; 0 means max(10 KKT_lp, 1e-3) */
} meb_params;

typedef struct {
    double r;            /* returned radius: max_i(||c - c_i|| + r_i) at the returned c */
    double r_alm;        /* ripALM's own radius variable                                */
    double kkt[5];       /* KKT residuals of Sec. 5 at the last iterate, original units */
    double kkt_max;      /* max of the five on the scaled problem (compared with tol)  */
    double delta_max;    /* Delta_max = max_i(r_i + ||c - c_i||) - r_alm (Sec. 4.2)      */
    double scale;        /* s                                                          */
    int64_t n_active;    /* true size of the active set (may exceed active_cap)        */
    int64_t fp64_rows;   /* ball rows evaluated in FP64 over all passes                */
    int32_t outer_iters, ssn_iters, cg_iters, passes, backtracks;
    int32_t status;      /* 0 converged, 1 iteration cap                               */
    int32_t newton_inverses; /* dense Newton systems: FP32 Gauss-Jordan inverses of H  */
    int32_t newton_fp64; /* dense Newton systems that fell back to FP64 Cholesky       */
    int64_t n_reduced;   /* balls of the FP64 solve (m unless params->mixed)           */
    int32_t readd_rounds; /* mixed: FP64 solves after the first (violated balls added) */
    int32_t lowp_passes; /* mixed: passes of the low-precision run                     */
} meb_info;

/* Measurement counters of a context (no counterpart in the paper: they
 * support the roofline report).  kernel_launches counts every kernel the
 * context launched since meb_reset_stats; with profiling on, each full pass
 * over the balls (the per-ball map of Algorithm 2, step 1) is bracketed by
 * CUDA events on the context's stream and its device time summed here. */
typedef struct {
    int64_t kernel_launches;
    int64_t pass_launches;   /* timed pass launches                      */
    double pass_ms;          /* their summed device time, milliseconds   */
    int64_t pass_balls;      /* balls they streamed (m per launch)       */
    int64_t pass_fp64_rows;  /* rows they evaluated in FP64              */
    int64_t pass_bytes;      /* bytes they streamed: per ball the shadow
                                row, 16*ceil(d/8) + 4 (FP16 and its norm,
                                solves) or 16*ceil(d/4) (FP32), + 4
                                (radius) + 4 (multiplier slot)             */
    int64_t batch_instances; /* instances solved by meb_solve_batch      */
    int64_t batch_fallbacks; /* of those, re-solved by the multi-block path */
    double phase_ms[4];      /* with profiling, ticks driven by the host (the
                                matrix-free Newton path, or MEB_OPT_TICK_LOOP
                                1): elapsed device time of the pass (screen
                                and FP64 rows), the support rows and
                                controller, the Newton system (with the host's
                                turnarounds between CG rounds) and the
                                multiplier update, milliseconds            */
} meb_stats;

/* Create a context on `device`, issuing work on `cuda_stream` (a cudaStream_t;
 * NULL: the context creates and owns a non-blocking stream). */
int meb_create(meb_ctx **out, int device, void *cuda_stream);
void meb_destroy(meb_ctx *ctx);
void meb_params_default(meb_params *p);
const char *meb_last_error(const meb_ctx *ctx);

/* Context options (no counterpart in the paper: they select how the same
 * method is executed, and the numbers the tests and the benchmark compare).
 * Each context keeps its own values; a new context starts at the defaults.
 *
 *  MEB_OPT_SCREEN       how every full pass of a solve decides which balls
 *                       need FP64 rows (Algorithm 2, step 1):
 *                       MEB_SCREEN_FP16 (default) certified FP16 shadow,
 *                       register-batched loads; MEB_SCREEN_FP16_BULK the same
 *                       through a bulk-copy (TMA) pipeline; MEB_SCREEN_FP32
 *                       certified FP32 shadow; MEB_SCREEN_FP64 no shadow: every
 *                       ball of every pass and of every feasibility pass is
 *                       evaluated in FP64 (the plain FP64 ripALM).
 *  MEB_OPT_EVAL_SCREEN  the same choice for meb_eval_alm (default FP32); it
 *                       also applies to meb_feas_check when it is MEB_SCREEN_FP64.
 *  MEB_OPT_EVAL_SHADOW_EXP  meb_eval_alm with an FP16 screen builds the shadow
 *                       of (c_i - c_1) / 2^value (any exponent; default 0).
 *                       Values that overflow FP16 are never certified and values
 *                       in its subnormal range carry their absolute error bound,
 *                       so every exponent gives the same results.
 *  MEB_OPT_TICK_LOOP    device-resident loop of a solve: 0 (default) CUDA graphs
 *                       of 8 controller ticks relaunched until the controller
 *                       stops; 1 host-launched ticks; 2 one graph with a
 *                       while-node.  All three give bit-identical results.
 *  MEB_OPT_WAIT_CYCLES  bound, in SM clock cycles, of each wait of the
 *                       bulk-copy screen for its copies (default 2e9, about one
 *                       second); 0 makes each wait a single non-blocking test.
 *                       An expired wait ends the solve with MEB_ETIMEOUT after
 *                       the copies in flight have landed; the context stays
 *                       usable.
 *  MEB_OPT_BATCH_SLOTS  meb_solve_batch's scratch: 0 (default) one slot per
 *                       resident thread block, each sized for the batch's
 *                       largest instance, blocks taking instances from a queue;
 *                       1 one slot per instance sized for it, block k solving
 *                       instance k (scratch = the sum of meb_footprint(.., 1)).
 *                       Results are the same either way.
 *  MEB_OPT_RELEASE_SCRATCH  1: every call frees the context's device scratch
 *                       before it returns (for callers that account device
 *                       memory against a budget); 0 (default) keeps it for the
 *                       next call.
 *  MEB_OPT_BLOCKING_SYNC  1: the calling thread sleeps while it waits for the
 *                       context's stream (a blocking-sync event) instead of
 *                       spinning, for callers that run many contexts from
 *                       more threads than host cores; 0 (default) spins, the
 *                       shortest wake-up.
 * Returns MEB_EINVAL for an unknown option or value. */
#define MEB_OPT_SCREEN 1
#define MEB_OPT_EVAL_SCREEN 2
#define MEB_OPT_EVAL_SHADOW_EXP 3
#define MEB_OPT_TICK_LOOP 4
#define MEB_OPT_WAIT_CYCLES 5
#define MEB_OPT_BATCH_SLOTS 6
#define MEB_OPT_RELEASE_SCRATCH 7
#define MEB_OPT_BLOCKING_SYNC 8
#define MEB_SCREEN_FP16 0
#define MEB_SCREEN_FP16_BULK 1
#define MEB_SCREEN_FP32 2
#define MEB_SCREEN_FP64 3
int meb_set_option(meb_ctx *ctx, int32_t option, int64_t value);

/* Device scratch, in bytes, beyond inputs and outputs: path 0 a meb_solve of
 * (m, d) (the context's buffers), path 1 one instance of meb_solve_batch with
 * MEB_OPT_BATCH_SLOTS = 1.  MEB_EINVAL for sizes out of range. */
int meb_footprint(int64_t m, int32_t d, int32_t path, int64_t *bytes);

/* Turn per-pass event timing on (1) or off (0); reset / read the counters. */
int meb_set_profiling(meb_ctx *ctx, int on);
int meb_reset_stats(meb_ctx *ctx);
int meb_get_stats(meb_ctx *ctx, meb_stats *out);

/* Solve eq. (MEB) (Algorithms 1 + 2, then the feasibility pass of Sec. 4.2).
 * centers m x d, radii m; tol > 0 overrides params->tol (params may be NULL).
 * Outputs: c_out[d]; active_idx[active_cap] ascending indices of
 * {i : r - r_i - ||c - c_i|| <= theta r} (truncated at active_cap, which may be
 * 0 with active_idx NULL); info (may be NULL).  m = 1 returns the ball itself.
 * Host centres of more than 128 MB are copied in chunks of about 64 MB on the
 * context's second stream, the FP32 shadow of each chunk computed on the
 * context's stream under the copy of the next (same results as device
 * inputs); the call returns when both streams are done with the inputs. */
int meb_solve(meb_ctx *ctx, const double *centers, const double *radii, int64_t m, int32_t d,
              double tol, const meb_params *params, unsigned flags, double *c_out,
              int64_t *active_idx, int64_t active_cap, meb_info *info);

/* The multipliers (u_i, v_i) = sigma Pi_Q(z_i) at the point the last
 * meb_solve on this context returned (Algorithm 1's multiplier update at the
 * last accepted point; the KKT residuals info->kkt were evaluated with them).
 * Only balls with a nonzero multiplier are listed, in ascending ball order:
 * idx[k], u[k] and v[k*d .. k*d+d-1] for k < min(cap, *n_sup); *n_sup is the
 * true count.  The multipliers do not depend on the problem's scale.  For
 * m = 1 the list is (0, 1, 0); when every ball is the same point it is every
 * ball with u = 1/m, v = 0.  flags & MEB_PTR_DEVICE: idx, u and v are device
 * pointers; n_sup is a host pointer.  Valid until the next call that computes
 * on the context; MEB_EINVAL if there is no such solve. */
int meb_get_multipliers(meb_ctx *ctx, unsigned flags, int64_t *idx, double *u, double *v,
                        int64_t cap, int64_t *n_sup);

/* A ragged batch of independent instances (no counterpart in the paper, which
 * solves one instance at a time: this is Algorithms 1 + 2 and the Sec. 4.2
 * pass applied to many instances in one launch).  Per instance: centers
 * (m x d row-major) and radii (m) in; c_out (d) and active_idx (the first
 * active_cap ascending indices of the active set, may be NULL with cap 0) out.
 * Pointers follow flags & MEB_PTR_DEVICE like every other call (host arrays
 * are copied in and out by the library). */
typedef struct {
    const double *centers;
    const double *radii;
    int64_t m;
    int32_t d;
    int32_t reserved;
    double *c_out;
    int64_t *active_idx;
    int64_t active_cap;
} meb_batch_item;

/* Solve every instance of the batch (the same method and parameters as
 * meb_solve; tol > 0 overrides params->tol).  One persistent launch: each
 * thread block takes instances from a device queue, largest first, and runs a
 * whole solve of one instance at a time (its passes, controller, Newton
 * systems and final feasibility pass), so an instance's result does not
 * depend on the other instances of the batch or on which block solved it.
 * Instances need 1 <= d <= 4096; the dense Newton solve is used for d <= 111,
 * matrix-free CG above.  Each block holds scratch sized for the batch's
 * largest instance, with room for the support rows of min(m, max(2048,
 * 16 (d + 1))) balls; an instance whose support outgrows it is solved again
 * by meb_solve's multi-block path (counted in meb_stats.batch_fallbacks).
 * infos[n] (host, may be NULL): per instance as meb_solve's info, status 0
 * converged, 1 iteration cap.  Returns MEB_EINVAL if an instance is invalid
 * (sizes, NULL pointers, non-finite values, negative radius: its info has
 * status -1; the others are still solved), MEB_ENOTCONV if one hit its cap. */
int meb_solve_batch(meb_ctx *ctx, int32_t n, const meb_batch_item *items, double tol,
                    const meb_params *params, unsigned flags, meb_info *infos);

/* The batch solver's execution choices per class of d (d <= 4, <= 16, <= 64,
 * <= 128, larger): the screen's shadow (FP32: 4 coordinates per 16-byte load;
 * FP16: 8), the balls per pass block (tiles of 256) and the blocks of the
 * support-row reduction, and the thread blocks per SM of the launch.
 * meb_tune_batch times the candidates on up to `per_class` instances of each
 * class present in the batch (device pointers as flags say) and keeps the
 * fastest in the context for the following meb_solve_batch calls; configs
 * (may be NULL) receives, per class, shadow (0 FP32, 1 FP16), tiles per pass
 * block and support blocks, then the blocks per SM: 5 x 3 + 1 int32.  The
 * choice changes which balls are evaluated in FP64, so results can differ in
 * the last bits between configurations (never beyond the solve tolerance);
 * for a fixed configuration they are deterministic. */
#define MEB_BATCH_CLASSES 5
int meb_tune_batch(meb_ctx *ctx, int32_t n, const meb_batch_item *items, int32_t per_class,
                   unsigned flags, int32_t *configs);

/* Serving (no counterpart in the paper): a request loop that solves MEB
 * instances as they arrive, with continuous batching.  Requests are admitted
 * in arrival order while their device footprint (inputs, outputs and solver
 * scratch, meb_footprint) fits in budget_bytes; admitted small requests are
 * grouped into meb_solve_batch launches by several workers, each on its own
 * context and stream, so a group launched while others run shares the GPU
 * with them; requests with m*d >= large_balls take meb_solve's multi-block
 * path on their own workers.  Each request is solved by exactly the steps it
 * would take alone: its results do not depend on the mix.
 * Zero fields of cfg take the defaults: 64 small workers, 2 large workers,
 * large_balls 2^27, groups of at most 4 requests.  The workers allocate from
 * a stream-ordered memory pool that the process's servers share (one per
 * device), which keeps freed memory (up to the largest budget_bytes) for the
 * next requests and servers and never makes one worker's allocation wait for
 * another worker's work; each worker runs on a stream the process keeps for
 * its index (streams are not created and destroyed per server: that churn
 * halved a later server's throughput); they wait for the GPU asleep
 * (MEB_OPT_BLOCKING_SYNC).  The workers' streams run side by side only on
 * separate hardware queues: set CUDA_DEVICE_MAX_CONNECTIONS (at most 32)
 * before the process first uses CUDA. */
typedef struct {
    int64_t budget_bytes;     /* device memory for admitted requests (required, > 0) */
    int64_t large_balls;      /* m*d at or above which a request is "large"          */
    int32_t small_workers;
    int32_t large_workers;
    int32_t max_group;
    int32_t flags;            /* MEB_SERVER_SPIN_WAITS, MEB_SERVER_DEVICE_POOL, or 0 */
} meb_server_config;
/* workers spin while they wait for the GPU (default: they sleep) */
#define MEB_SERVER_SPIN_WAITS 1u
/* workers allocate from the device's default stream-ordered pool (default:
   the pool the process's servers share) */
#define MEB_SERVER_DEVICE_POOL 2u

typedef struct {
    int64_t submitted, completed, failed;
    int64_t launches;         /* batch launches and multi-block solves             */
    int64_t in_use_bytes;     /* footprint of admitted, unfinished requests        */
    int64_t peak_bytes;       /* its maximum since the server started             */
    int64_t pending;          /* submitted, not yet admitted                       */
} meb_server_stats;

typedef struct meb_server meb_server;

/* Create a server on `device` (params may be NULL: defaults). */
int meb_server_create(meb_server **out, int device, const meb_server_config *cfg,
                      const meb_params *params);
/* Queue one instance (host arrays: centers m x d, radii m; outputs c_out (d),
 * active_idx (first active_cap ascending indices), info).  Returns at once
 * with a ticket; every array must stay valid until the request completes.
 * MEB_EINVAL for bad sizes or NULL pointers; MEB_ENOMEM when the request alone
 * exceeds the budget. */
int meb_server_submit(meb_server *sv, const double *centers, const double *radii, int64_t m,
                      int32_t d, double *c_out, int64_t *active_idx, int64_t active_cap,
                      meb_info *info, int64_t *ticket);
/* Wait up to timeout_s seconds (< 0: no limit) for a request: its return code
 * (as meb_solve's) in *rc and its latency, submit to completion, in
 * *latency_s.  MEB_ETIMEOUT if it has not completed in time (wait again). */
int meb_server_wait(meb_server *sv, int64_t ticket, double timeout_s, int *rc, double *latency_s);
int meb_server_get_stats(meb_server *sv, meb_server_stats *out);
/* Finish every queued request, stop the workers and free the server. */
void meb_server_destroy(meb_server *sv);

/* One evaluation of the prox-AL subproblem (Sec. 4, Algorithm 2 steps 1-2) at
 * x = (r, c) (x[0] = r) with proximal centre xbar, multipliers U (m), V (m x d),
 * penalty sigma > 0, proximal weight tau > 0, on the unscaled data:
 *   psi   = r + sigma/2 sum ||Pi(z_i)||^2 - 1/(2 sigma) sum ||(u_i,v_i)||^2
 *           + tau/(2 sigma) ||x - xbar||^2,
 *   grad  = (1,0) - sum (u_i^+, v_i^+) + tau/sigma (x - xbar)        [d+1]
 *   Uplus, Vplus = sigma Pi(z_i)                                   [m], [m x d]
 *   Hq    = (tau/sigma I + sigma sum P_i) q   if q and Hq non-NULL  [d+1]
 *   H     = tau/sigma I + sigma sum P_i      if H non-NULL         [(d+1)^2]
 *   case_counts[3] = balls in cases Z (||b|| <= -a), I (||b|| <= a), M.
 * Uplus and Vplus must both be given or both be NULL.                      */
int meb_eval_alm(meb_ctx *ctx, const double *centers, const double *radii, int64_t m,
                 int32_t d, const double *x, const double *xbar, const double *U,
                 const double *V, double sigma, double tau, const double *q, unsigned flags,
                 double *psi, double *grad, double *Uplus, double *Vplus, double *Hq, double *H,
                 int64_t *case_counts);

/* The a-posteriori feasibility pass of Sec. 4.2 at the ball (c, r):
 *   delta_max = max_i (r_i + ||c - c_i|| - r), argmax = lowest maximising index,
 *   viol_idx  = ascending { i : r_i + ||c - c_i|| - r > eps } (first viol_cap),
 *   n_viol    = its true size.  viol_idx may be NULL with viol_cap 0.          */
int meb_feas_check(meb_ctx *ctx, const double *centers, const double *radii, int64_t m,
                   int32_t d, const double *c, double r, double eps, unsigned flags,
                   double *delta_max, int64_t *argmax, int64_t *viol_idx, int64_t viol_cap,
                   int64_t *n_viol);

/* Allocation-free variant of meb_feas_check (the paper has no counterpart: it
 * exists for callers that cannot call cudaMalloc, such as engines whose device
 * memory belongs to their own pool or to another framework's caching
 * allocator, and loops that forbid allocation once running).  Same results as
 * meb_feas_check, computed in FP64 from the rows.  No context: the work runs on
 * `cuda_stream` (NULL: the legacy default stream) of the current device, and the
 * call returns after it completes.  centers (m x d), radii (m), c (d) and
 * viol_idx (viol_cap entries, may be NULL with viol_cap 0) are DEVICE pointers on
 * the current device; delta_max, argmax and n_viol are host pointers.
 * Scratch: a fixed static device array (about 37 KB per GPU that loads the
 * library, held until exit); the call allocates and frees nothing.  A negative
 * or non-finite radius, or any non-finite value of a row or of c (so that a
 * ball's value is not finite), returns MEB_EINVAL.  The first
 * call on a device caches the array's device address (cudaGetSymbolAddress):
 * make it before any stream capture on that device.  All calls share the array:
 * calls that overlap on the GPU (several streams or host threads) race.
 * Limits: 1 <= m <= 2^31 - 1, 1 <= d <= 4096; larger sizes return MEB_EINVAL. */
int meb_feas_check_noalloc(const double *centers, const double *radii, int64_t m, int32_t d,
                           const double *c, double r, double eps, void *cuda_stream,
                           double *delta_max, int64_t *argmax, int64_t *viol_idx,
                           int64_t viol_cap, int64_t *n_viol);

#ifdef __cplusplus
}
#endif

#endif /* MEB_H */
