/*
 * meb_oracle.c -- plain CPU FP64 oracle for the ripALM minimum-enclosing-ball
 * method (arxiv 2605.31425).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference the CUDA path is checked against.  Only tests/, the smoke()
 * entry of __graft_entry__.py and the CPU-baseline leg of bench.py may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library, and it includes nothing from it.
 *
 * Everything is FP64.  Loops over the balls of a solve run over fixed chunks
 * of ORC_CHUNK balls in index order; a sum over balls is the sum, in chunk
 * order, of the chunks' sums, each taken in index order.  Chunks may run on
 * several threads (OpenMP, when the compiler has it), and the results do not
 * depend on the thread count (orc_feas_check takes no sums: its results are
 * those of one loop in index order).  orc_eval_alm sums in plain index
 * order.  Each function cites the passage of the paper it follows:
 *
 *   Sec. 2, eq. (MEB-SOCP)   : constraint (r - r_i, c - c_i) in Q_{d+1}
 *   Sec. 2, AL function      : phi_sigma and its gradient
 *   Sec. 2, projection       : closed form of Pi_Q (three cases)
 *   Algorithm 1 (ripALM)     : prox-AL subproblem, relative stop test,
 *                              multiplier update, auxiliary update
 *   Sec. 4 (GPU implementation): batched projection, grad and generalized
 *                              Hessian H = tau/sigma I + sigma sum P_i,
 *                              Hessian-vector product
 *   Algorithm 2 (SSN)        : inner semismooth Newton with Armijo search
 *   Sec. 4.2                 : a-posteriori feasibility check Delta_max, V
 *   Sec. 5                   : KKT_max (five residuals)
 *
 * Readings of points the paper leaves open (all shared, as readings, with
 * the CUDA path; none of them as code):
 *   - scaling: c0 = mean of centres, r0 = max_i(||c0 - c_i|| + r_i),
 *     s = smallest power of two >= r0; ripALM runs on the data divided by s
 *     (exact) and the result is multiplied back by s.
 *   - generalized Jacobian at kinks: the projection's case order (I first,
 *     then Z, else M); I includes a = ||b|| = 0.
 *   - sigma_0 = 10, sigma_{k+1} = min(sigma_max, 10 sigma_k) when the
 *     primal residual max_i dist((r - r_i, c - c_i), Q) is above tol and
 *     did not fall below a tenth of its previous value; tau = 10 constant
 *     (Theorem 1 holds with nu_k = 0).
 *   - the inner loop also stops when ||grad|| is within 8 ulp of the scale
 *     of its own rounding error (nothing left to gain in FP64).
 *   - Armijo: mu = 1e-4, at most max_backtrack reductions, a rounding
 *     allowance of 64 ulp of the summed magnitude of Psi; each reduction
 *     takes the minimiser of the quadratic through Psi(0), Psi'(0) and
 *     Psi(eta), safeguarded to [eta/10, eta/2].
 *   - the returned radius is the max-type value max_i(||c - c_i|| + r_i)
 *     at the returned centre (the a-posteriori feasibility pass, Sec. 4.2).
 *   - active set A = { i : r - r_i - ||c - c_i|| <= theta * r }.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_CHUNK 4096 /* balls per chunk of a solve's sums (see the header) */

static int64_t nchunks(int64_t m) { return (m + ORC_CHUNK - 1) / ORC_CHUNK; }

/* Threads for the chunk loops (1 without OpenMP); n <= 0 leaves the default. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define ORC_CASE_Z 0 /* ||b|| <= -a : projection is 0              */
#define ORC_CASE_I 1 /* ||b|| <=  a : projection is the point      */
#define ORC_CASE_M 2 /* otherwise   : projection onto the boundary */

typedef struct {
    double tol;          /* KKT_max tolerance on the scaled problem          */
    double rho;          /* relative-error factor of Algorithm 1, in [0,1)   */
    double sigma0;       /* initial penalty on the scaled problem            */
    double sigma_max;    /* cap on the penalty                               */
    double sigma_growth; /* factor applied when the primal residual stalls   */
    double sigma_ratio;  /* "stalls": residual above this fraction of the last */
    double tau;          /* proximal weight (constant)                       */
    double armijo_mu;    /* sufficient-decrease constant                     */
    double active_theta; /* active-set threshold, relative to r              */
    int max_outer;
    int max_ssn;
    int max_backtrack;
    int dense_max_d;     /* dense Cholesky if d <= this, else CG             */
    int max_cg;
} orc_params;

typedef struct {
    double r;            /* returned radius (max-type value at c)          */
    double r_alm;        /* ripALM's own radius variable                   */
    double kkt[5];       /* the five KKT residuals, original units         */
    double kkt_max;      /* max of kkt[] on the scaled problem             */
    double delta_max;    /* Delta_max of the ALM ball (r_alm)              */
    double scale;        /* s                                               */
    int64_t n_active;
    int32_t outer_iters, ssn_iters, cg_iters, passes, backtracks;
    int32_t status;      /* 0 converged, 1 iteration cap                   */
} orc_info;

void orc_params_default(orc_params *p)
{
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
    p->dense_max_d = 256;
    p->max_cg = 500;
}

static double dot(const double *x, const double *y, int n)
{
    double s = 0.0;
    for (int j = 0; j < n; j++) s += x[j] * y[j];
    return s;
}

static double nrm(const double *x, int n) { return sqrt(dot(x, x, n)); }

/* ---------------------------------------------------------------------- */
/* Sec. 2: projection onto Q_{d+1} = {(t,s): ||s|| <= t}, closed form.      */
/* Returns the case; writes Pi(a,b) into (pa, pb).                          */
int orc_soc_project(double a, const double *b, int d, double *pa, double *pb)
{
    double n = nrm(b, d);
    if (n <= a) {
        *pa = a;
        for (int j = 0; j < d; j++) pb[j] = b[j];
        return ORC_CASE_I;
    }
    if (n <= -a) {
        *pa = 0.0;
        for (int j = 0; j < d; j++) pb[j] = 0.0;
        return ORC_CASE_Z;
    }
    double f = 0.5 * (a + n);
    *pa = f;
    for (int j = 0; j < d; j++) pb[j] = f * b[j] / n;
    return ORC_CASE_M;
}

/* Euclidean distance of (a,b) to Q_{d+1}: ||z - Pi(z)||.                   */
double orc_soc_dist(double a, const double *b, int d)
{
    double *pb = (double *)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double pa;
    orc_soc_project(a, b, d, &pa, pb);
    double s = (a - pa) * (a - pa);
    for (int j = 0; j < d; j++) s += (b[j] - pb[j]) * (b[j] - pb[j]);
    free(pb);
    return sqrt(s);
}

/* An element P of the Clarke generalized Jacobian of Pi_Q at (a,b), dense
 * (d+1)x(d+1) row-major.  Case I: identity.  Case Z: zero.  Case M: the
 * derivative of (a+n)/2 * (1, b/n), i.e. with w = b/n, t = a/n,
 *   P = 1/2 [[1, w^T], [w, (1+t) I - t w w^T]].                            */
int orc_soc_jacobian(double a, const double *b, int d, double *P)
{
    int n1 = d + 1;
    for (int k = 0; k < n1 * n1; k++) P[k] = 0.0;
    double n = nrm(b, d);
    if (n <= a) {
        for (int k = 0; k < n1; k++) P[k * n1 + k] = 1.0;
        return ORC_CASE_I;
    }
    if (n <= -a) return ORC_CASE_Z;
    double t = a / n;
    P[0] = 0.5;
    for (int j = 0; j < d; j++) {
        double wj = b[j] / n;
        P[0 * n1 + (1 + j)] = 0.5 * wj;
        P[(1 + j) * n1 + 0] = 0.5 * wj;
        for (int l = 0; l < d; l++) {
            double wl = b[l] / n;
            P[(1 + j) * n1 + (1 + l)] = 0.5 * ((j == l ? 1.0 + t : 0.0) - t * wj * wl);
        }
    }
    return ORC_CASE_M;
}

/* ---------------------------------------------------------------------- */
/* Sec. 4 / Algorithm 2, steps 1-2: one evaluation of the prox-AL
 * subproblem at x = (r, c).
 *
 *   z_i   = (r_i - r, c_i - c) + (u_i, v_i)/sigma
 *   (u_i+, v_i+) = sigma * Pi(z_i)
 *   Psi   = r + sigma/2 sum ||Pi(z_i)||^2 - 1/(2 sigma) sum ||(u_i,v_i)||^2
 *           + tau/(2 sigma) ||x - xbar||^2
 *   grad  = (1,0) - sum (u_i+, v_i+) + tau/sigma (x - xbar)
 *   Hq    = tau/sigma q + sigma sum P_i q          (if q != NULL)
 *   H     = tau/sigma I + sigma sum P_i            (if H != NULL)
 * counts[0..2] = number of balls in cases Z, I, M.
 * Uplus/Vplus may be NULL.  U/V may be NULL (zero multipliers).          */
int orc_eval_alm(int64_t m, int d, const double *C, const double *R,
                 const double *x, const double *xbar, const double *U,
                 const double *V, double sigma, double tau, const double *q,
                 double *psi, double *grad, double *Uplus, double *Vplus,
                 double *Hq, double *H, int64_t *counts)
{
    int n1 = d + 1;
    double *b = (double *)malloc(sizeof(double) * (size_t)d);
    double *pb = (double *)malloc(sizeof(double) * (size_t)d);
    double *sv = (double *)calloc((size_t)d, sizeof(double));
    double *hq = q ? (double *)calloc((size_t)n1, sizeof(double)) : NULL;
    double *hs = H ? (double *)calloc((size_t)n1 * n1, sizeof(double)) : NULL;
    double sum_pi2 = 0.0, sum_uv2 = 0.0, su = 0.0;
    int64_t cnt[3] = {0, 0, 0};

    for (int64_t i = 0; i < m; i++) {
        const double *ci = C + i * d;
        double ui = U ? U[i] : 0.0;
        const double *vi = V ? V + i * d : NULL;
        double a = R[i] - x[0] + ui / sigma;
        for (int j = 0; j < d; j++) b[j] = ci[j] - x[1 + j] + (vi ? vi[j] : 0.0) / sigma;
        double pa;
        int cs = orc_soc_project(a, b, d, &pa, pb);
        cnt[cs]++;

        double pi2 = pa * pa + dot(pb, pb, d);
        sum_pi2 += pi2;
        double uv2 = ui * ui + (vi ? dot(vi, vi, d) : 0.0);
        sum_uv2 += uv2;
        su += sigma * pa;
        for (int j = 0; j < d; j++) sv[j] += sigma * pb[j];
        if (Uplus) Uplus[i] = sigma * pa;
        if (Vplus)
            for (int j = 0; j < d; j++) Vplus[i * d + j] = sigma * pb[j];

        if (cs == ORC_CASE_Z || (!q && !H)) continue;
        if (cs == ORC_CASE_I) {
            if (hq)
                for (int k = 0; k < n1; k++) hq[k] += q[k];
            if (hs)
                for (int k = 0; k < n1; k++) hs[k * n1 + k] += 1.0;
            continue;
        }
        /* case M */
        double n = nrm(b, d);
        double t = a / n;
        if (hq) {
            double wq = 0.0;
            for (int j = 0; j < d; j++) wq += (b[j] / n) * q[1 + j];
            hq[0] += 0.5 * (q[0] + wq);
            for (int j = 0; j < d; j++) {
                double wj = b[j] / n;
                hq[1 + j] += 0.5 * (q[0] * wj + (1.0 + t) * q[1 + j] - t * wj * wq);
            }
        }
        if (hs) {
            hs[0] += 0.5;
            for (int j = 0; j < d; j++) {
                double wj = b[j] / n;
                hs[1 + j] += 0.5 * wj;
                hs[(1 + j) * n1] += 0.5 * wj;
                for (int l = 0; l < d; l++) {
                    double wl = b[l] / n;
                    hs[(1 + j) * n1 + (1 + l)] += 0.5 * ((j == l ? 1.0 + t : 0.0) - t * wj * wl);
                }
            }
        }
    }

    double dx2 = 0.0;
    for (int k = 0; k < n1; k++) dx2 += (x[k] - xbar[k]) * (x[k] - xbar[k]);
    if (psi)
        *psi = x[0] + 0.5 * sigma * sum_pi2 - sum_uv2 / (2.0 * sigma) + tau / (2.0 * sigma) * dx2;
    if (grad) {
        grad[0] = 1.0 - su + tau / sigma * (x[0] - xbar[0]);
        for (int j = 0; j < d; j++) grad[1 + j] = -sv[j] + tau / sigma * (x[1 + j] - xbar[1 + j]);
    }
    if (Hq)
        for (int k = 0; k < n1; k++) Hq[k] = tau / sigma * q[k] + sigma * hq[k];
    if (H)
        for (int k = 0; k < n1 * n1; k++)
            H[k] = sigma * hs[k] + ((k / n1) == (k % n1) ? tau / sigma : 0.0);
    if (counts) {
        counts[0] = cnt[0];
        counts[1] = cnt[1];
        counts[2] = cnt[2];
    }
    free(b);
    free(pb);
    free(sv);
    free(hq);
    free(hs);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Sec. 4.2: a-posteriori feasibility check against all balls.
 *   Delta_max = max_i (r_i + ||c - c_i|| - r),  argmax = lowest index,
 *   V = { i : r_i + ||c - c_i|| - r > eps } in ascending order
 * (written up to cap entries; *n_viol is the true count).                 */
int orc_feas_check(int64_t m, int d, const double *C, const double *R,
                   const double *c, double r, double eps, double *delta_max,
                   int64_t *argmax, int64_t *viol, int64_t cap, int64_t *n_viol)
{
    /* per ball, in chunks: e_i and whether it is violated; then the maximum
     * (lowest index on ties: chunks are merged in order with a strict >) and
     * the list, in index order */
    int64_t nc = nchunks(m);
    double *cbest = (double *)malloc(sizeof(double) * (size_t)nc);
    int64_t *carg = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    unsigned char *in = (unsigned char *)malloc((size_t)m);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nc; ch++) {
        double best = -INFINITY;
        int64_t arg = -1;
        int64_t i1 = (ch + 1) * ORC_CHUNK < m ? (ch + 1) * ORC_CHUNK : m;
        for (int64_t i = ch * ORC_CHUNK; i < i1; i++) {
            double s = 0.0;
            for (int j = 0; j < d; j++) {
                double t = c[j] - C[i * d + j];
                s += t * t;
            }
            double e = R[i] + sqrt(s) - r;
            if (e > best) {
                best = e;
                arg = i;
            }
            in[i] = e > eps;
        }
        cbest[ch] = best;
        carg[ch] = arg;
    }
    double best = -INFINITY;
    int64_t arg = -1, nv = 0;
    for (int64_t ch = 0; ch < nc; ch++)
        if (cbest[ch] > best) {
            best = cbest[ch];
            arg = carg[ch];
        }
    for (int64_t i = 0; i < m; i++)
        if (in[i]) {
            if (viol && nv < cap) viol[nv] = i;
            nv++;
        }
    if (delta_max) *delta_max = best;
    if (argmax) *argmax = arg;
    if (n_viol) *n_viol = nv;
    free(cbest);
    free(carg);
    free(in);
    return 0;
}

/* Sec. 5: the five KKT residuals at (r, c) with multipliers (U, V):
 *   k[0] = |1 - sum u_i|
 *   k[1] = ||sum v_i||
 *   k[2] = max_i dist((r - r_i, c - c_i), Q)
 *   k[3] = max_i dist((u_i, v_i), Q)
 *   k[4] = max_i |(r - r_i) u_i + <c - c_i, v_i>|                        */
int orc_kkt(int64_t m, int d, const double *C, const double *R, double r,
            const double *c, const double *U, const double *V, double *k)
{
    /* per chunk: sum u, sum v (d), and the three maxima; then the chunk sums
     * in chunk order and the maxima over chunks */
    int64_t nc = nchunks(m);
    int w = d + 4;
    double *part = (double *)calloc((size_t)nc * w, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nc; ch++) {
        double *p = part + ch * w; /* [0] sum u, [1..d] sum v, [d+1..d+3] maxima */
        double *b = (double *)malloc(sizeof(double) * (size_t)d);
        int64_t i1 = (ch + 1) * ORC_CHUNK < m ? (ch + 1) * ORC_CHUNK : m;
        for (int64_t i = ch * ORC_CHUNK; i < i1; i++) {
            p[0] += U[i];
            for (int j = 0; j < d; j++) p[1 + j] += V[i * d + j];
            for (int j = 0; j < d; j++) b[j] = c[j] - C[i * d + j];
            double dp = orc_soc_dist(r - R[i], b, d);
            if (dp > p[d + 1]) p[d + 1] = dp;
            double dd = orc_soc_dist(U[i], V + i * d, d);
            if (dd > p[d + 2]) p[d + 2] = dd;
            double cp = fabs((r - R[i]) * U[i] + dot(b, V + i * d, d));
            if (cp > p[d + 3]) p[d + 3] = cp;
        }
        free(b);
    }
    double su = 0.0, pinf = 0.0, dinf = 0.0, comp = 0.0;
    double *sv = (double *)calloc((size_t)d, sizeof(double));
    for (int64_t ch = 0; ch < nc; ch++) {
        const double *p = part + ch * w;
        su += p[0];
        for (int j = 0; j < d; j++) sv[j] += p[1 + j];
        if (p[d + 1] > pinf) pinf = p[d + 1];
        if (p[d + 2] > dinf) dinf = p[d + 2];
        if (p[d + 3] > comp) comp = p[d + 3];
    }
    k[0] = fabs(1.0 - su);
    k[1] = nrm(sv, d);
    k[2] = pinf;
    k[3] = dinf;
    k[4] = comp;
    free(sv);
    free(part);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Dense Cholesky solve of the SPD system H x = rhs (n x n, row-major).
 * Returns 0, or 1 if a pivot is not positive.                              */
static int chol_solve(int n, const double *H, const double *rhs, double *x)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)n * n);
    memcpy(L, H, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; j++) {
        double s = L[j * n + j];
        for (int k = 0; k < j; k++) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) {
            free(L);
            return 1;
        }
        double ljj = sqrt(s);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = L[i * n + j];
            for (int k = 0; k < j; k++) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / ljj;
        }
    }
    for (int i = 0; i < n; i++) { /* L y = rhs */
        double t = rhs[i];
        for (int k = 0; k < i; k++) t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) { /* L^T x = y */
        double t = x[i];
        for (int k = i + 1; k < n; k++) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
    free(L);
    return 0;
}

/* Data of one SSN iterate kept for the Newton system: the support (cases I
 * and M) with, for case M, w_i = b_i/||b_i|| and t_i = a_i/||b_i||.       */
typedef struct {
    int64_t n;      /* support size      */
    int64_t cap;
    int *cs;        /* case per entry    */
    double *t;      /* t_i (case M)      */
    double *w;      /* w_i rows (case M) */
} support_t;

/* Psi, grad, multipliers and the support at x on the scaled data.  The
 * constant -1/(2 sigma) sum ||(u,v)||^2 is left out of psi (it does not
 * depend on x); *psi_mag is the summed magnitude of the terms of psi and
 * *g_mag = 1 + sigma sum_{I,M} |z_i| + tau/sigma ||x - xbar||, the scale of
 * the rounding error of grad (sigma Pi(z_i) loses |z_i| eps absolutely).  */
static void eval_point(int64_t m, int d, const double *C, const double *R,
                       const double *x, const double *xbar, const double *U,
                       const double *V, double sigma, double tau, double *psi,
                       double *psi_mag, double *g_mag, double *grad, double *Up,
                       double *Vp, support_t *S)
{
    /* per chunk: sum ||Pi(z_i)||^2, sum u+, sum_{I,M} |a_i| + ||b_i||, sum v+ (d);
     * the case of every ball */
    int64_t nc = nchunks(m);
    int w = d + 3;
    double *part = (double *)calloc((size_t)nc * w, sizeof(double));
    unsigned char *cs_all = (unsigned char *)malloc((size_t)m);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nc; ch++) {
        double *p = part + ch * w;
        double *b = (double *)malloc(sizeof(double) * (size_t)d);
        double *pb = (double *)malloc(sizeof(double) * (size_t)d);
        int64_t i1 = (ch + 1) * ORC_CHUNK < m ? (ch + 1) * ORC_CHUNK : m;
        for (int64_t i = ch * ORC_CHUNK; i < i1; i++) {
            double a = R[i] - x[0] + U[i] / sigma;
            for (int j = 0; j < d; j++) b[j] = C[i * d + j] - x[1 + j] + V[i * d + j] / sigma;
            double pa;
            int cs = orc_soc_project(a, b, d, &pa, pb);
            cs_all[i] = (unsigned char)cs;
            p[0] += pa * pa + dot(pb, pb, d);
            p[1] += sigma * pa;
            for (int j = 0; j < d; j++) p[3 + j] += sigma * pb[j];
            Up[i] = sigma * pa;
            for (int j = 0; j < d; j++) Vp[i * d + j] = sigma * pb[j];
            if (cs != ORC_CASE_Z) p[2] += fabs(a) + nrm(b, d);
        }
        free(b);
        free(pb);
    }
    double sum_pi2 = 0.0, su = 0.0, zmag = 0.0;
    double *sv = (double *)calloc((size_t)d, sizeof(double));
    for (int64_t ch = 0; ch < nc; ch++) {
        const double *p = part + ch * w;
        sum_pi2 += p[0];
        su += p[1];
        zmag += p[2];
        for (int j = 0; j < d; j++) sv[j] += p[3 + j];
    }
    /* the support (cases I and M) in ball order; for case M, w_i = b_i/||b_i||
     * and t_i = a_i/||b_i|| */
    double *b = (double *)malloc(sizeof(double) * (size_t)d);
    S->n = 0;
    for (int64_t i = 0; i < m; i++) {
        int cs = cs_all[i];
        if (cs == ORC_CASE_Z) continue;
        int64_t k = S->n++;
        S->cs[k] = cs;
        if (cs == ORC_CASE_M) {
            double a = R[i] - x[0] + U[i] / sigma;
            for (int j = 0; j < d; j++) b[j] = C[i * d + j] - x[1 + j] + V[i * d + j] / sigma;
            double n = nrm(b, d);
            S->t[k] = a / n;
            for (int j = 0; j < d; j++) S->w[k * d + j] = b[j] / n;
        }
    }
    double dx2 = 0.0;
    for (int k = 0; k <= d; k++) dx2 += (x[k] - xbar[k]) * (x[k] - xbar[k]);
    *psi = x[0] + 0.5 * sigma * sum_pi2 + tau / (2.0 * sigma) * dx2;
    *psi_mag = fabs(x[0]) + 0.5 * sigma * sum_pi2 + tau / (2.0 * sigma) * dx2;
    *g_mag = 1.0 + sigma * zmag + tau / sigma * sqrt(dx2);
    grad[0] = 1.0 - su + tau / sigma * (x[0] - xbar[0]);
    for (int j = 0; j < d; j++) grad[1 + j] = -sv[j] + tau / sigma * (x[1 + j] - xbar[1 + j]);
    free(b);
    free(sv);
    free(part);
    free(cs_all);
}

/* sum_i ||(Up_i, Vp_i) - (U_i, V_i)||^2 in chunks (the stop test of Algorithm 1). */
static double duv2_sum(int64_t m, int d, const double *Up, const double *U, const double *Vp,
                       const double *V)
{
    int64_t nc = nchunks(m);
    double *part = (double *)calloc((size_t)nc, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nc; ch++) {
        double t2 = 0.0;
        int64_t i1 = (ch + 1) * ORC_CHUNK < m ? (ch + 1) * ORC_CHUNK : m;
        for (int64_t i = ch * ORC_CHUNK; i < i1; i++) {
            t2 += (Up[i] - U[i]) * (Up[i] - U[i]);
            for (int jj = 0; jj < d; jj++) {
                double t = Vp[i * d + jj] - V[i * d + jj];
                t2 += t * t;
            }
        }
        part[ch] = t2;
    }
    double s = 0.0;
    for (int64_t ch = 0; ch < nc; ch++) s += part[ch];
    free(part);
    return s;
}

/* max_i (||c - c_i|| + r_i) in chunks (the max-type value, Sec. 1). */
static double max_type_value(int64_t m, int d, const double *C, const double *R,
                             const double *c)
{
    int64_t nc = nchunks(m);
    double *part = (double *)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nc; ch++) {
        double best = -INFINITY;
        int64_t i1 = (ch + 1) * ORC_CHUNK < m ? (ch + 1) * ORC_CHUNK : m;
        for (int64_t i = ch * ORC_CHUNK; i < i1; i++) {
            double q = 0.0;
            for (int j = 0; j < d; j++) q += (c[j] - C[i * d + j]) * (c[j] - C[i * d + j]);
            double e = sqrt(q) + R[i];
            if (e > best) best = e;
        }
        part[ch] = best;
    }
    double best = -INFINITY;
    for (int64_t ch = 0; ch < nc; ch++)
        if (part[ch] > best) best = part[ch];
    free(part);
    return best;
}

/* y = (tau/sigma I + sigma sum P_i) q using the stored support.            */
static void hess_vec(int d, const support_t *S, double sigma, double tau,
                     const double *q, double *y)
{
    int n1 = d + 1;
    for (int k = 0; k < n1; k++) y[k] = 0.0;
    for (int64_t s = 0; s < S->n; s++) {
        if (S->cs[s] == ORC_CASE_I) {
            for (int k = 0; k < n1; k++) y[k] += q[k];
            continue;
        }
        const double *w = S->w + s * d;
        double t = S->t[s];
        double wq = dot(w, q + 1, d);
        y[0] += 0.5 * (q[0] + wq);
        for (int j = 0; j < d; j++) y[1 + j] += 0.5 * (q[0] * w[j] + (1.0 + t) * q[1 + j] - t * w[j] * wq);
    }
    for (int k = 0; k < n1; k++) y[k] = tau / sigma * q[k] + sigma * y[k];
}

/* H = tau/sigma I + sigma sum P_i, dense, from the stored support.        */
static void hess_dense(int d, const support_t *S, double sigma, double tau, double *H)
{
    int n1 = d + 1;
    for (int k = 0; k < n1 * n1; k++) H[k] = 0.0;
    for (int64_t s = 0; s < S->n; s++) {
        if (S->cs[s] == ORC_CASE_I) {
            for (int k = 0; k < n1; k++) H[k * n1 + k] += 1.0;
            continue;
        }
        const double *w = S->w + s * d;
        double t = S->t[s];
        H[0] += 0.5;
        for (int j = 0; j < d; j++) {
            H[1 + j] += 0.5 * w[j];
            H[(1 + j) * n1] += 0.5 * w[j];
            for (int l = 0; l < d; l++)
                H[(1 + j) * n1 + (1 + l)] += 0.5 * ((j == l ? 1.0 + t : 0.0) - t * w[j] * w[l]);
        }
    }
    for (int k = 0; k < n1 * n1; k++) H[k] *= sigma;
    for (int k = 0; k < n1; k++) H[k * n1 + k] += tau / sigma;
}

/* Conjugate gradients with the Jacobi preconditioner on H x = rhs;
 * stops at ||H x - rhs|| <= rtol ||rhs||.  Returns the iteration count.   */
static int cg_solve(int d, const support_t *S, double sigma, double tau,
                    const double *rhs, double rtol, int maxit, double *x)
{
    int n1 = d + 1;
    double *r = (double *)malloc(sizeof(double) * n1);
    double *z = (double *)malloc(sizeof(double) * n1);
    double *p = (double *)malloc(sizeof(double) * n1);
    double *Ap = (double *)malloc(sizeof(double) * n1);
    double *dg = (double *)malloc(sizeof(double) * n1);
    /* diagonal of H */
    for (int k = 0; k < n1; k++) dg[k] = 0.0;
    for (int64_t s = 0; s < S->n; s++) {
        if (S->cs[s] == ORC_CASE_I) {
            for (int k = 0; k < n1; k++) dg[k] += 1.0;
            continue;
        }
        const double *w = S->w + s * d;
        double t = S->t[s];
        dg[0] += 0.5;
        for (int j = 0; j < d; j++) dg[1 + j] += 0.5 * ((1.0 + t) - t * w[j] * w[j]);
    }
    for (int k = 0; k < n1; k++) dg[k] = tau / sigma + sigma * dg[k];

    for (int k = 0; k < n1; k++) {
        x[k] = 0.0;
        r[k] = rhs[k];
        z[k] = r[k] / dg[k];
        p[k] = z[k];
    }
    double rz = dot(r, z, n1);
    double bn = nrm(rhs, n1);
    int it = 0;
    if (bn == 0.0) goto done;
    for (it = 0; it < maxit; it++) {
        if (nrm(r, n1) <= rtol * bn) break;
        hess_vec(d, S, sigma, tau, p, Ap);
        double alpha = rz / dot(p, Ap, n1);
        for (int k = 0; k < n1; k++) {
            x[k] += alpha * p[k];
            r[k] -= alpha * Ap[k];
        }
        for (int k = 0; k < n1; k++) z[k] = r[k] / dg[k];
        double rz1 = dot(r, z, n1);
        double beta = rz1 / rz;
        rz = rz1;
        for (int k = 0; k < n1; k++) p[k] = z[k] + beta * p[k];
    }
done:
    free(r);
    free(z);
    free(p);
    free(Ap);
    free(dg);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 (ripALM) with Algorithm 2 (SSN) as the inner solver, on the
 * scaled data.  Outputs: c_out[d], info, and optionally the multipliers
 * U_out[m], V_out[m*d] and the active set (ascending, up to cap).        */
int orc_solve(int64_t m, int d, const double *C0, const double *R0,
              const orc_params *prm_in, double *c_out, double *U_out,
              double *V_out, int64_t *active, int64_t cap, orc_info *info)
{
    orc_params prm;
    if (prm_in) prm = *prm_in; else orc_params_default(&prm);
    memset(info, 0, sizeof(*info));
    if (m < 1 || d < 1) return -1;
    int n1 = d + 1;

    /* m = 1: the ball itself. */
    if (m == 1) {
        for (int j = 0; j < d; j++) c_out[j] = C0[j];
        info->r = info->r_alm = R0[0];
        info->scale = 1.0;
        if (U_out) U_out[0] = 1.0;
        if (V_out) for (int j = 0; j < d; j++) V_out[j] = 0.0;
        if (active && cap > 0) active[0] = 0;
        info->n_active = 1;
        return 0;
    }

    /* Initial point: mean centre (chunk sums in chunk order), radius of the
     * max-type value there. */
    double *c0 = (double *)calloc((size_t)d, sizeof(double));
    {
        int64_t nc = nchunks(m);
        double *part = (double *)calloc((size_t)nc * d, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t ch = 0; ch < nc; ch++) {
            int64_t i1 = (ch + 1) * ORC_CHUNK < m ? (ch + 1) * ORC_CHUNK : m;
            for (int64_t i = ch * ORC_CHUNK; i < i1; i++)
                for (int j = 0; j < d; j++) part[ch * d + j] += C0[i * d + j];
        }
        for (int64_t ch = 0; ch < nc; ch++)
            for (int j = 0; j < d; j++) c0[j] += part[ch * d + j];
        free(part);
    }
    for (int j = 0; j < d; j++) c0[j] /= (double)m;
    double r0 = max_type_value(m, d, C0, R0, c0);
    if (r0 == 0.0) { /* every ball is the same point */
        for (int j = 0; j < d; j++) c_out[j] = c0[j];
        info->r = info->r_alm = 0.0;
        info->scale = 1.0;
        if (U_out) for (int64_t i = 0; i < m; i++) U_out[i] = 1.0 / (double)m;
        if (V_out) memset(V_out, 0, sizeof(double) * (size_t)m * d);
        int64_t na = 0;
        for (int64_t i = 0; i < m; i++) { if (active && na < cap) active[na] = i; na++; }
        info->n_active = na;
        free(c0);
        return 0;
    }
    int ex;
    frexp(r0, &ex);
    double s = ldexp(1.0, ex); /* power of two, r0 <= s < 2 r0 */
    if (s / 2.0 >= r0) s /= 2.0;

    /* Scaled data. */
    double *C = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *R = (double *)malloc(sizeof(double) * (size_t)m);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m * d; i++) C[i] = C0[i] / s;
    for (int64_t i = 0; i < m; i++) R[i] = R0[i] / s;

    double *U = (double *)calloc((size_t)m, sizeof(double));
    double *V = (double *)calloc((size_t)m * d, sizeof(double));
    double *Up = (double *)malloc(sizeof(double) * (size_t)m);
    double *Vp = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *Ut = (double *)malloc(sizeof(double) * (size_t)m);
    double *Vt = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *x = (double *)malloc(sizeof(double) * n1);
    double *xk = (double *)malloc(sizeof(double) * n1);
    double *ab = (double *)malloc(sizeof(double) * n1);
    double *g = (double *)malloc(sizeof(double) * n1);
    double *gt = (double *)malloc(sizeof(double) * n1);
    double *xt = (double *)malloc(sizeof(double) * n1);
    double *dx = (double *)malloc(sizeof(double) * n1);
    double *rhs = (double *)malloc(sizeof(double) * n1);
    double *H = (d <= prm.dense_max_d) ? (double *)malloc(sizeof(double) * n1 * n1) : NULL;
    support_t S, St;
    S.cap = St.cap = m;
    S.cs = (int *)malloc(sizeof(int) * (size_t)m);
    S.t = (double *)malloc(sizeof(double) * (size_t)m);
    S.w = (double *)malloc(sizeof(double) * (size_t)m * d);
    St.cs = (int *)malloc(sizeof(int) * (size_t)m);
    St.t = (double *)malloc(sizeof(double) * (size_t)m);
    St.w = (double *)malloc(sizeof(double) * (size_t)m * d);

    x[0] = r0 / s;
    for (int j = 0; j < d; j++) x[1 + j] = c0[j] / s;
    for (int k = 0; k < n1; k++) ab[k] = x[k];
    double sigma = prm.sigma0, tau = prm.tau;
    double pinf_prev = INFINITY;
    double kk[5] = {0, 0, 0, 0, 0};
    int status = 1;
    int outer = 0, ssn_total = 0, cg_total = 0, passes = 0, backtracks = 0;

    for (outer = 0; outer < prm.max_outer; outer++) {
        for (int k = 0; k < n1; k++) xk[k] = x[k];
        /* ---- Algorithm 2 from x^k ---- */
        double psi, mag, gmag;
        eval_point(m, d, C, R, x, xk, U, V, sigma, tau, &psi, &mag, &gmag, g, Up, Vp, &S);
        passes++;
        for (int j = 0; j < prm.max_ssn; j++) {
            /* relative-type stopping condition on the tentative quantities */
            double lhs_a = 0.0, g2 = 0.0, dxk2 = 0.0, duv2 = 0.0;
            for (int k = 0; k < n1; k++) {
                lhs_a += (ab[k] - x[k]) * g[k];
                g2 += g[k] * g[k];
                dxk2 += (x[k] - xk[k]) * (x[k] - xk[k]);
            }
            duv2 = duv2_sum(m, d, Up, U, Vp, V);
            double lhs = 2.0 * sigma * fabs(lhs_a) + sigma * sigma * g2;
            double rhs_v = prm.rho * (duv2 + tau * dxk2);
            if (lhs <= rhs_v) break;
            /* safeguard: g is at the rounding level of its own terms */
            if (sqrt(g2) <= 8.0 * 2.220446049250313e-16 * gmag) break;

            /* Newton direction H dx = -g */
            for (int k = 0; k < n1; k++) rhs[k] = -g[k];
            if (H) {
                hess_dense(d, &S, sigma, tau, H);
                if (chol_solve(n1, H, rhs, dx)) break;
            } else {
                double gn = sqrt(g2);
                double rt = gn < 0.01 ? sqrt(gn) : 0.1;
                cg_total += cg_solve(d, &S, sigma, tau, rhs, rt, prm.max_cg, dx);
            }
            ssn_total++;
            double gdx = dot(g, dx, n1);
            /* Armijo line search on Psi */
            double eta = 1.0, psit = 0.0, magt = 0.0, gmagt = 0.0;
            int ok = 0;
            for (int bt = 0; bt <= prm.max_backtrack; bt++) {
                for (int k = 0; k < n1; k++) xt[k] = x[k] + eta * dx[k];
                eval_point(m, d, C, R, xt, xk, U, V, sigma, tau, &psit, &magt, &gmagt, gt, Ut, Vt, &St);
                passes++;
                double allow = 64.0 * 2.220446049250313e-16 * (mag > magt ? mag : magt);
                if (psit <= psi + prm.armijo_mu * eta * gdx + allow) { ok = 1; break; }
                if (bt == prm.max_backtrack) break;
                {
                    /* next step: minimiser of the quadratic through Psi(0),
                     * Psi'(0) = g.dx and Psi(eta), kept in [eta/10, eta/2] */
                    double den = 2.0 * (psit - psi - gdx * eta);
                    double en = (den > 0.0) ? -gdx * eta * eta / den : 0.5 * eta;
                    if (en < 0.1 * eta) en = 0.1 * eta;
                    if (en > 0.5 * eta) en = 0.5 * eta;
                    eta = en;
                }
                backtracks++;
            }
            /* accept the last trial (ok or not) */
            {
                double *tp;
                support_t tS;
                for (int k = 0; k < n1; k++) { x[k] = xt[k]; g[k] = gt[k]; }
                psi = psit; mag = magt; gmag = gmagt;
                tp = Up; Up = Ut; Ut = tp;
                tp = Vp; Vp = Vt; Vt = tp;
                tS = S; S = St; St = tS;
            }
            if (!ok) break;
        }
        /* multiplier and auxiliary updates */
        for (int k = 0; k < n1; k++) ab[k] -= sigma * g[k];
        { double *tp = U; U = Up; Up = tp; tp = V; V = Vp; Vp = tp; }

        /* KKT_max on the scaled problem */
        orc_kkt(m, d, C, R, x[0], x + 1, U, V, kk);
        double kmax = 0.0;
        for (int k = 0; k < 5; k++) if (kk[k] > kmax) kmax = kk[k];
        if (getenv("MEB_ORACLE_TRACE"))
            fprintf(stderr, "outer %d sigma %.3e ssn_total %d passes %d kkt %.2e %.2e %.2e %.2e %.2e r %.15g\n",
                    outer, sigma, ssn_total, passes, kk[0], kk[1], kk[2], kk[3], kk[4], x[0] * s);
        if (kmax <= prm.tol) { status = 0; outer++; break; }
        if (kk[2] > prm.tol && kk[2] > prm.sigma_ratio * pinf_prev) {
            sigma *= prm.sigma_growth;
            if (sigma > prm.sigma_max) sigma = prm.sigma_max;
        }
        pinf_prev = kk[2];
    }

    /* Sec. 4.2 check at the ALM ball, then the max-type radius at c. */
    double *cc = (double *)malloc(sizeof(double) * (size_t)d);
    for (int j = 0; j < d; j++) cc[j] = x[1 + j] * s;
    double r_alm = x[0] * s;
    double dmax;
    int64_t amax;
    orc_feas_check(m, d, C0, R0, cc, r_alm, 0.0, &dmax, &amax, NULL, 0, NULL);
    double r_out = r_alm + dmax;
    /* r_out is max_i(||c - c_i|| + r_i); recompute it directly */
    r_out = max_type_value(m, d, C0, R0, cc);
    /* active set: slack r - r_i - ||c - c_i|| <= theta r, in index order */
    unsigned char *act = (unsigned char *)malloc((size_t)m);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++) {
        double q = 0.0;
        for (int j = 0; j < d; j++) q += (cc[j] - C0[i * d + j]) * (cc[j] - C0[i * d + j]);
        double slack = r_out - R0[i] - sqrt(q);
        act[i] = slack <= prm.active_theta * r_out;
    }
    int64_t na = 0;
    for (int64_t i = 0; i < m; i++) {
        if (act[i]) {
            if (active && na < cap) active[na] = i;
            na++;
        }
    }
    free(act);
    for (int j = 0; j < d; j++) c_out[j] = cc[j];
    if (U_out) memcpy(U_out, U, sizeof(double) * (size_t)m);
    if (V_out) memcpy(V_out, V, sizeof(double) * (size_t)m * d);

    info->r = r_out;
    info->r_alm = r_alm;
    info->kkt[0] = kk[0];
    info->kkt[1] = kk[1];
    info->kkt[2] = kk[2] * s;
    info->kkt[3] = kk[3];
    info->kkt[4] = kk[4] * s;
    info->kkt_max = 0.0;
    for (int k = 0; k < 5; k++) if (kk[k] > info->kkt_max) info->kkt_max = kk[k];
    info->delta_max = dmax;
    info->scale = s;
    info->n_active = na;
    info->outer_iters = outer;
    info->ssn_iters = ssn_total;
    info->cg_iters = cg_total;
    info->passes = passes;
    info->backtracks = backtracks;
    info->status = status;

    free(cc); free(c0); free(C); free(R); free(U); free(V); free(Up); free(Vp);
    free(Ut); free(Vt); free(x); free(xk); free(ab); free(g); free(gt); free(xt);
    free(dx); free(rhs); free(H);
    free(S.cs); free(S.t); free(S.w); free(St.cs); free(St.t); free(St.w);
    return status == 0 ? 0 : 1;
}
