/*
 * FP64 CPU oracle for (pipelined) BiCGStab -- TEST INFRASTRUCTURE ONLY.
 *
 * Cools & Vanroose, "The communication-hiding pipelined BiCGStab method for
 * the parallel solution of large unsymmetric linear systems" (arXiv:1612.01395).
 *
 * This file is the plain, slow, single-threaded reference that the CUDA path
 * is checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code with the CUDA library.
 *
 * Every routine follows the paper's algorithm step by step, in the paper's
 * notation, with no blocking, fusion or reordering:
 *   o_bicgstab    Algorithm 7 (standard BiCGStab, Section 3.1)
 *   o_cabicgstab  Algorithm 8 (communication-avoiding BiCGStab, Section 3.2)
 *   o_pbicgstab   Algorithm 9 (pipelined BiCGStab, Section 3.3) with the
 *                 residual replacement of Section 4.2, and the eq. (5)
 *                 variant of alpha as a test option.
 * Dot products are summed left to right (i = 0..n-1); a CSR row is summed in
 * storage order. Build with -ffp-contract=off so that no multiply-add is fused
 * and results are the same on every host.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *  - r0 denotes both the initial residual and the fixed shadow vector in every
 *    (r0, .) dot product; residual replacement never changes the shadow.
 *  - p_{-1}, s_{-1}, z_{-1}, v_{-1} and omega_{-1} are zero (they are multiplied
 *    by beta_{-1} = 0).
 *  - Stopping: ||r_{i+1}|| <= rtol ||r_0|| on the recursive residual, tested
 *    once per iteration after the second reduction; (r, r) is an extra dot.
 *    A half step (x += alpha p) is taken when ||q_i|| <= rtol ||r_0||, using an
 *    extra dot (q, q) in the first reduction.
 *  - Breakdown: a zero denominator of alpha, (y, y) = 0 with q != 0, omega = 0,
 *    or (r0, r_{i+1}) = 0 stops with status BREAKDOWN; a non-finite reduced
 *    scalar stops with status NONFINITE. x is left at the last full iterate.
 *  - Residual replacement "at iteration i" (k > 0, i > 0, i mod k == 0, fewer
 *    than max_rr replacements so far) resets r_i, w_i, s_i, z_i with 4 SpMVs
 *    (Section 4.2). Default placement (rr_placement = 0): r_i := b - A x_i and
 *    w_i := A r_i right after x_i, r_i, w_i are formed in iteration i-1 and
 *    before the second reduction, so (r0, r_i), (r0, w_i), ||r_i||, t_i = A w_i
 *    and alpha_i are computed from the replaced vectors; then s_i := A p_i and
 *    z_i := A s_i replace the s and z recurrences after p_i is formed.
 *    rr_placement = 1 is the literal alternative (all four after p_i, with
 *    t_i, v_{i-1}, rho_i and alpha_i left stale); it is kept only so a test
 *    can show that it destabilises the iteration.
 *  - fixed_iters > 0 runs exactly that many iterations and ignores rtol
 *    (breakdown still stops), so two implementations can be compared step by step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The parity build is single-threaded (no -fopenmp: the pragmas below are
 * ignored and every loop runs in the order written). A second build with
 * -fopenmp splits the row loops of the SpMV and the vector updates over
 * threads and sums dot products per thread, for timing the oracle on all host
 * cores; only that build's dot products are summed in another order. */
int o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

enum { O_CONVERGED = 0, O_NOT_CONVERGED = 1, O_BREAKDOWN = 2, O_NONFINITE = 3, O_ERR_ARG = 4, O_ERR_OOM = 5 };

typedef struct {
    int32_t iters;          /* iterations performed; a half step counts as one */
    int32_t status;         /* O_* above */
    int32_t half_step;      /* 1 when the last iteration stopped at x + alpha p */
    int32_t n_replacements; /* residual replacement steps performed */
    double nr0;             /* ||r_0||_2 */
    double rel_res_rec;     /* recursive ||r|| / ||r_0|| at exit */
    double rel_res_true;    /* ||b - A x|| / ||r_0|| at exit */
    double flops;           /* instrumented AXPY + dot-product flops of the
                               paper's operations (Table 1), excluding the
                               stopping norms, summed over all iterations */
    int32_t spmvs;          /* SpMVs performed, including initialisation */
    int32_t pad;
} o_info;

typedef struct {
    int32_t n;
    const int32_t *rowptr;
    const int32_t *col;
    const double *val;
} o_csr;

/* ---------------------------------------------------------------------------
 * The three building blocks the paper names (Section 1): SpMV, dot product,
 * AXPY. Each updates the flop counter with the paper's Table 1 convention:
 * a dot product or an AXPY y = x + a z costs 2N flops.
 * ------------------------------------------------------------------------- */
typedef struct {
    double flops;
    int32_t spmvs;
} o_count;

/* y = A x, row i summed over its stored entries in order */
static void spmv(const o_csr *A, const double *x, double *y, o_count *c)
{
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < A->n; i++) {
        double acc = 0.0;
        for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; e++)
            acc = acc + A->val[e] * x[A->col[e]];
        y[i] = acc;
    }
    if (c) c->spmvs += 1;
}

/* (a, b) summed left to right */
static double dot(int32_t n, const double *a, const double *b, o_count *c)
{
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int32_t i = 0; i < n; i++) acc = acc + a[i] * b[i];
    if (c) c->flops += 2.0 * n;
    return acc;
}

/* out = x + alpha * z (out may alias x or z) */
static void axpy(int32_t n, double *out, const double *x, double alpha, const double *z, o_count *c)
{
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; i++) out[i] = x[i] + alpha * z[i];
    if (c) c->flops += 2.0 * n;
}

static double norm2(int32_t n, const double *a) { return sqrt(dot(n, a, a, NULL)); }

static int finite_all(int cnt, const double *v)
{
    for (int k = 0; k < cnt; k++)
        if (!isfinite(v[k])) return 0;
    return 1;
}

/* res = b - A x, and its norm */
static double true_residual(const o_csr *A, const double *b, const double *x, double *res)
{
    spmv(A, x, res, NULL);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < A->n; i++) res[i] = b[i] - res[i];
    return norm2(A->n, res);
}

void o_spmv(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
            const double *x, double *y)
{
    o_csr A = {n, rowptr, col, val};
    spmv(&A, x, y, NULL);
}

double o_dot(int32_t n, const double *a, const double *b) { return dot(n, a, b, NULL); }

/* Shared bookkeeping of the three solvers: history and traces. */
typedef struct {
    double *hist;     /* [maxit+1] or NULL: ||r_i|| (recursive) */
    double *trace_x;  /* [(maxit+1) * n] or NULL: x_i */
    double *trace_r;  /* [(maxit+1) * n] or NULL: r_i (recursive) */
} o_trace;

static void record(const o_trace *tr, int32_t i, int32_t n, double nr, const double *x, const double *r)
{
    if (tr->hist) tr->hist[i] = nr;
    if (tr->trace_x) memcpy(tr->trace_x + (size_t)i * n, x, sizeof(double) * n);
    if (tr->trace_r) memcpy(tr->trace_r + (size_t)i * n, r, sizeof(double) * n);
}

static void finish(const o_csr *A, const double *b, const double *x, double *tmp,
                   double nr_rec, o_info *info, const o_count *cnt)
{
    double nt = true_residual(A, b, x, tmp);
    info->rel_res_rec = info->nr0 > 0 ? nr_rec / info->nr0 : 0.0;
    info->rel_res_true = info->nr0 > 0 ? nt / info->nr0 : nt;
    info->flops = cnt->flops;
    info->spmvs = cnt->spmvs;
}

/* ===========================================================================
 * Algorithm 7: standard BiCGStab (Section 3.1).
 * ========================================================================= */
int o_bicgstab(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
               const double *b, double *x, double rtol, int32_t maxit, int32_t fixed_iters,
               double *hist, double *trace_x, double *trace_r, o_info *info)
{
    o_csr A = {n, rowptr, col, val};
    o_trace tr = {hist, trace_x, trace_r};
    o_count cnt = {0.0, 0};
    memset(info, 0, sizeof(*info));
    if (n < 0 || maxit < 0) return info->status = O_ERR_ARG;
    double *mem = (double *)calloc((size_t)7 * (n > 0 ? n : 1), sizeof(double));
    if (!mem) return info->status = O_ERR_OOM;
    double *r = mem, *r0 = r + n, *p = r0 + n, *s = p + n, *q = s + n, *y = q + n, *tmp = y + n;
    int32_t limit = fixed_iters > 0 ? fixed_iters : maxit;

    /* r_0 := b - A x_0; p_0 := r_0 */
    spmv(&A, x, tmp, &cnt);
    for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
    memcpy(r0, r, sizeof(double) * n);
    memcpy(p, r, sizeof(double) * n);
    double rho = dot(n, r0, r, NULL); /* (r0, r_0) */
    double nr = norm2(n, r);
    info->nr0 = nr;
    record(&tr, 0, n, nr, x, r);
    double tol = rtol * info->nr0;
    info->status = O_NOT_CONVERGED;
    if (info->nr0 == 0.0) { info->status = O_CONVERGED; finish(&A, b, x, tmp, nr, info, &cnt); free(mem); return info->status; }

    int32_t i;
    for (i = 0; i < limit; i++) {
        /* s_i := A p_i */
        spmv(&A, p, s, &cnt);
        /* alpha_i := (r0, r_i) / (r0, s_i) */
        double r0s = dot(n, r0, s, &cnt);
        if (!isfinite(r0s)) { info->status = O_NONFINITE; break; }
        if (r0s == 0.0) { info->status = O_BREAKDOWN; break; }
        double alpha = rho / r0s;
        /* q_i := r_i - alpha_i s_i */
        axpy(n, q, r, -alpha, s, &cnt);
        /* y_i := A q_i */
        spmv(&A, q, y, &cnt);
        /* omega_i := (q_i, y_i) / (y_i, y_i); (q, q) for the half step */
        double qy = dot(n, q, y, &cnt), yy = dot(n, y, y, &cnt), qq = dot(n, q, q, NULL);
        double d1[3] = {qy, yy, qq};
        if (!finite_all(3, d1)) { info->status = O_NONFINITE; break; }
        if ((fixed_iters <= 0 && sqrt(qq) <= tol) || yy == 0.0) {
            if (yy == 0.0 && qq != 0.0 && !(fixed_iters <= 0 && sqrt(qq) <= tol)) { info->status = O_BREAKDOWN; break; }
            axpy(n, x, x, alpha, p, &cnt); /* half step: x_{i+1/2} = x_i + alpha_i p_i */
            nr = sqrt(qq);
            info->half_step = 1;
            info->status = O_CONVERGED;
            record(&tr, i + 1, n, nr, x, q);
            i++;
            break;
        }
        double omega = qy / yy;
        if (omega == 0.0) { info->status = O_BREAKDOWN; break; }
        /* x_{i+1} := x_i + alpha_i p_i + omega_i q_i */
        axpy(n, x, x, alpha, p, &cnt);
        axpy(n, x, x, omega, q, &cnt);
        /* r_{i+1} := q_i - omega_i y_i */
        axpy(n, r, q, -omega, y, &cnt);
        /* beta_i := (alpha_i / omega_i) (r0, r_{i+1}) / (r0, r_i) */
        double rho_new = dot(n, r0, r, &cnt);
        double rr = dot(n, r, r, NULL);
        double d2[2] = {rho_new, rr};
        nr = sqrt(rr);
        record(&tr, i + 1, n, nr, x, r);
        if (!finite_all(2, d2)) { info->status = O_NONFINITE; i++; break; }
        if (fixed_iters <= 0 && nr <= tol) { info->status = O_CONVERGED; i++; break; }
        if (rho_new == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        double beta = (alpha / omega) * (rho_new / rho);
        rho = rho_new;
        /* p_{i+1} := r_{i+1} + beta_i (p_i - omega_i s_i) */
        axpy(n, p, p, -omega, s, &cnt);
        axpy(n, p, r, beta, p, &cnt);
    }
    if (fixed_iters > 0 && info->status == O_NOT_CONVERGED && i == limit) info->status = O_CONVERGED;
    info->iters = i;
    finish(&A, b, x, tmp, nr, info, &cnt);
    free(mem);
    return info->status;
}

/* ===========================================================================
 * Algorithm 8: communication-avoiding BiCGStab (Section 3.2), alpha by eq. (3).
 * ========================================================================= */
int o_cabicgstab(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                 const double *b, double *x, double rtol, int32_t maxit, int32_t fixed_iters,
                 double *hist, double *trace_x, double *trace_r, o_info *info)
{
    o_csr A = {n, rowptr, col, val};
    o_trace tr = {hist, trace_x, trace_r};
    o_count cnt = {0.0, 0};
    memset(info, 0, sizeof(*info));
    if (n < 0 || maxit < 0) return info->status = O_ERR_ARG;
    double *mem = (double *)calloc((size_t)10 * (n > 0 ? n : 1), sizeof(double));
    if (!mem) return info->status = O_ERR_OOM;
    double *r = mem, *r0 = r + n, *w = r0 + n, *p = w + n, *s = p + n, *z = s + n, *q = z + n, *y = q + n,
           *tmp = y + n;
    int32_t limit = fixed_iters > 0 ? fixed_iters : maxit;

    /* r_0 := b - A x_0; w_0 := A r_0; alpha_0 := (r0, r0)/(r0, w0); beta_{-1} := 0 */
    spmv(&A, x, tmp, &cnt);
    for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
    memcpy(r0, r, sizeof(double) * n);
    spmv(&A, r, w, &cnt);
    double rho = dot(n, r0, r, NULL);
    double r0w = dot(n, r0, w, NULL);
    double nr = norm2(n, r);
    info->nr0 = nr;
    record(&tr, 0, n, nr, x, r);
    double tol = rtol * info->nr0;
    info->status = O_NOT_CONVERGED;
    if (info->nr0 == 0.0) { info->status = O_CONVERGED; finish(&A, b, x, tmp, nr, info, &cnt); free(mem); return info->status; }
    if (r0w == 0.0 || !isfinite(r0w)) { info->status = isfinite(r0w) ? O_BREAKDOWN : O_NONFINITE; finish(&A, b, x, tmp, nr, info, &cnt); free(mem); return info->status; }
    double alpha = rho / r0w, beta = 0.0, omega = 0.0;

    int32_t i;
    for (i = 0; i < limit; i++) {
        /* p_i := r_i + beta_{i-1} (p_{i-1} - omega_{i-1} s_{i-1}) */
        axpy(n, p, p, -omega, s, &cnt);
        axpy(n, p, r, beta, p, &cnt);
        /* s_i := w_i + beta_{i-1} (s_{i-1} - omega_{i-1} z_{i-1}) */
        axpy(n, s, s, -omega, z, &cnt);
        axpy(n, s, w, beta, s, &cnt);
        /* z_i := A s_i */
        spmv(&A, s, z, &cnt);
        /* q_i := r_i - alpha_i s_i; y_i := w_i - alpha_i z_i */
        axpy(n, q, r, -alpha, s, &cnt);
        axpy(n, y, w, -alpha, z, &cnt);
        /* omega_i */
        double qy = dot(n, q, y, &cnt), yy = dot(n, y, y, &cnt), qq = dot(n, q, q, NULL);
        double d1[3] = {qy, yy, qq};
        if (!finite_all(3, d1)) { info->status = O_NONFINITE; break; }
        if ((fixed_iters <= 0 && sqrt(qq) <= tol) || yy == 0.0) {
            if (yy == 0.0 && qq != 0.0 && !(fixed_iters <= 0 && sqrt(qq) <= tol)) { info->status = O_BREAKDOWN; break; }
            axpy(n, x, x, alpha, p, &cnt);
            nr = sqrt(qq);
            info->half_step = 1;
            info->status = O_CONVERGED;
            record(&tr, i + 1, n, nr, x, q);
            i++;
            break;
        }
        omega = qy / yy;
        if (omega == 0.0) { info->status = O_BREAKDOWN; break; }
        /* x and r updates */
        axpy(n, x, x, alpha, p, &cnt);
        axpy(n, x, x, omega, q, &cnt);
        axpy(n, r, q, -omega, y, &cnt);
        /* w_{i+1} := A r_{i+1} */
        spmv(&A, r, w, &cnt);
        /* (r0, r_{i+1}); (r0, w_{i+1}); (r0, s_i); (r0, z_i) */
        double rho_new = dot(n, r0, r, &cnt), r0w_new = dot(n, r0, w, &cnt);
        double r0s = dot(n, r0, s, &cnt), r0z = dot(n, r0, z, &cnt);
        double rr = dot(n, r, r, NULL);
        double d2[5] = {rho_new, r0w_new, r0s, r0z, rr};
        nr = sqrt(rr);
        record(&tr, i + 1, n, nr, x, r);
        if (!finite_all(5, d2)) { info->status = O_NONFINITE; i++; break; }
        if (fixed_iters <= 0 && nr <= tol) { info->status = O_CONVERGED; i++; break; }
        if (rho_new == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        /* beta_i, alpha_{i+1} by eq. (3) */
        beta = (alpha / omega) * (rho_new / rho);
        double den = r0w_new + beta * r0s - beta * omega * r0z;
        if (den == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        alpha = rho_new / den;
        rho = rho_new;
    }
    if (fixed_iters > 0 && info->status == O_NOT_CONVERGED && i == limit) info->status = O_CONVERGED;
    info->iters = i;
    finish(&A, b, x, tmp, nr, info, &cnt);
    free(mem);
    return info->status;
}

/* ===========================================================================
 * Algorithm 9: pipelined BiCGStab (Section 3.3) + residual replacement
 * (Section 4.2). Vectors: x (caller), r, r0, p, s, z, q, y, w, t, v -- the 11
 * of Table 1. `work` may be NULL or point to 10*n doubles that receive
 * r, r0, p, s, z, q, y, w, t, v (in that order) at exit, for invariant tests.
 * ========================================================================= */
int o_pbicgstab(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                const double *b, double *x, double rtol, int32_t maxit, int32_t fixed_iters,
                int32_t replace_period, int32_t max_replacements, int32_t alpha_eq5,
                int32_t rr_placement, double *hist, double *trace_x, double *trace_r, double *work, o_info *info)
{
    o_csr A = {n, rowptr, col, val};
    o_trace tr = {hist, trace_x, trace_r};
    o_count cnt = {0.0, 0};
    memset(info, 0, sizeof(*info));
    if (n < 0 || maxit < 0) return info->status = O_ERR_ARG;
    double *mem = (double *)calloc((size_t)11 * (n > 0 ? n : 1), sizeof(double));
    if (!mem) return info->status = O_ERR_OOM;
    double *r = mem, *r0 = r + n, *p = r0 + n, *s = p + n, *z = s + n, *q = z + n, *y = q + n, *w = y + n,
           *t = w + n, *v = t + n, *tmp = v + n;
    int32_t limit = fixed_iters > 0 ? fixed_iters : maxit;

    /* r_0 := b - A x_0; w_0 := A r_0; t_0 := A w_0;
     *         alpha_0 := (r0, r0)/(r0, w0); beta_{-1} := 0 */
    spmv(&A, x, tmp, &cnt);
    for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
    memcpy(r0, r, sizeof(double) * n);
    spmv(&A, r, w, &cnt);
    spmv(&A, w, t, &cnt);
    double rho = dot(n, r0, r, NULL);
    double r0w = dot(n, r0, w, NULL);
    double nr = norm2(n, r);
    info->nr0 = nr;
    record(&tr, 0, n, nr, x, r);
    double tol = rtol * info->nr0;
    info->status = O_NOT_CONVERGED;
    int32_t i = 0;
    double alpha = 0.0, beta = 0.0, omega = 0.0;
    int replaced_rw = 0;
    if (info->nr0 == 0.0) { info->status = O_CONVERGED; goto out; }
    if (r0w == 0.0 || !isfinite(r0w)) { info->status = isfinite(r0w) ? O_BREAKDOWN : O_NONFINITE; goto out; }
    alpha = rho / r0w;

    for (i = 0; i < limit; i++) {
        /* p_i := r_i + beta_{i-1} (p_{i-1} - omega_{i-1} s_{i-1}) */
        axpy(n, p, p, -omega, s, &cnt);
        axpy(n, p, r, beta, p, &cnt);
        int late = rr_placement == 1 && replace_period > 0 && i > 0 && i % replace_period == 0 &&
                   (max_replacements < 0 || info->n_replacements < max_replacements);
        if (replaced_rw) {
            /* Section 4.2, second part: s_i := A p_i; z_i := A s_i */
            spmv(&A, p, s, &cnt);
            spmv(&A, s, z, &cnt);
        } else if (late) {
            /* literal alternative: r_i := b - A x_i; w_i := A r_i; s_i := A p_i; z_i := A s_i */
            spmv(&A, x, tmp, &cnt);
            for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
            spmv(&A, r, w, &cnt);
            spmv(&A, p, s, &cnt);
            spmv(&A, s, z, &cnt);
            info->n_replacements++;
        } else {
            /* s_i := w_i + beta_{i-1} (s_{i-1} - omega_{i-1} z_{i-1}) */
            axpy(n, s, s, -omega, z, &cnt);
            axpy(n, s, w, beta, s, &cnt);
            /* z_i := t_i + beta_{i-1} (z_{i-1} - omega_{i-1} v_{i-1}) */
            axpy(n, z, z, -omega, v, &cnt);
            axpy(n, z, t, beta, z, &cnt);
        }
        /* q_i := r_i - alpha_i s_i; y_i := w_i - alpha_i z_i */
        axpy(n, q, r, -alpha, s, &cnt);
        axpy(n, y, w, -alpha, z, &cnt);
        /* begin reduction (q_i, y_i); (y_i, y_i)  [+ (q_i, q_i)] */
        double qy = dot(n, q, y, &cnt), yy = dot(n, y, y, &cnt), qq = dot(n, q, q, NULL);
        /* v_i := A z_i */
        spmv(&A, z, v, &cnt);
        /* end reduction; omega_i := (q_i, y_i) / (y_i, y_i) */
        double d1[3] = {qy, yy, qq};
        if (!finite_all(3, d1)) { info->status = O_NONFINITE; break; }
        if ((fixed_iters <= 0 && sqrt(qq) <= tol) || yy == 0.0) {
            if (yy == 0.0 && qq != 0.0 && !(fixed_iters <= 0 && sqrt(qq) <= tol)) { info->status = O_BREAKDOWN; break; }
            axpy(n, x, x, alpha, p, &cnt);
            nr = sqrt(qq);
            info->half_step = 1;
            info->status = O_CONVERGED;
            record(&tr, i + 1, n, nr, x, q);
            i++;
            break;
        }
        omega = qy / yy;
        if (omega == 0.0) { info->status = O_BREAKDOWN; break; }
        /* x_{i+1} := x_i + alpha_i p_i + omega_i q_i */
        axpy(n, x, x, alpha, p, &cnt);
        axpy(n, x, x, omega, q, &cnt);
        /* r_{i+1} := q_i - omega_i y_i */
        axpy(n, r, q, -omega, y, &cnt);
        /* w_{i+1} := y_i - omega_i (t_i - alpha_i v_i) */
        axpy(n, tmp, t, -alpha, v, &cnt);
        axpy(n, w, y, -omega, tmp, &cnt);
        /* Section 4.2, first part (default placement): r_{i+1} := b - A x_{i+1};
         * w_{i+1} := A r_{i+1}, before the second reduction */
        replaced_rw = rr_placement == 0 && replace_period > 0 && (i + 1) % replace_period == 0 &&
                      (max_replacements < 0 || info->n_replacements < max_replacements);
        if (replaced_rw) {
            spmv(&A, x, tmp, &cnt);
            for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
            spmv(&A, r, w, &cnt);
            info->n_replacements++;
        }
        /* begin reduction (r0, r_{i+1}); (r0, w_{i+1}); (r0, s_i); (r0, z_i)  [+ (r, r)] */
        double rho_new = dot(n, r0, r, &cnt), r0w_new = dot(n, r0, w, &cnt);
        double r0s = dot(n, r0, s, &cnt), r0z = dot(n, r0, z, &cnt);
        double rr = dot(n, r, r, NULL);
        /* t_{i+1} := A w_{i+1} */
        spmv(&A, w, t, &cnt);
        /* end reduction */
        double d2[5] = {rho_new, r0w_new, r0s, r0z, rr};
        nr = sqrt(rr);
        record(&tr, i + 1, n, nr, x, r);
        if (!finite_all(5, d2)) { info->status = O_NONFINITE; i++; break; }
        if (fixed_iters <= 0 && nr <= tol) { info->status = O_CONVERGED; i++; break; }
        if (rho_new == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        /* beta_i := (alpha_i / omega_i) (r0, r_{i+1}) / (r0, r_i) */
        beta = (alpha / omega) * (rho_new / rho);
        /* alpha_{i+1} by eq. (3), or by eq. (5) as a test variant */
        if (alpha_eq5) {
            double inv = 1.0 / omega + r0w_new / rho_new - beta * omega * (r0z / rho_new);
            if (inv == 0.0) { info->status = O_BREAKDOWN; i++; break; }
            alpha = 1.0 / inv;
        } else {
            double den = r0w_new + beta * r0s - beta * omega * r0z;
            if (den == 0.0) { info->status = O_BREAKDOWN; i++; break; }
            alpha = rho_new / den;
        }
        rho = rho_new;
    }
    if (fixed_iters > 0 && info->status == O_NOT_CONVERGED && i == limit) info->status = O_CONVERGED;
out:
    info->iters = i;
    if (work) {
        double *src[10] = {r, r0, p, s, z, q, y, w, t, v};
        for (int k = 0; k < 10; k++) memcpy(work + (size_t)k * n, src[k], sizeof(double) * n);
    }
    finish(&A, b, x, tmp, nr, info, &cnt);
    free(mem);
    return info->status;
}

/* ===========================================================================
 * Preconditioned variants (Section 3.6) with a diagonal preconditioner:
 * M^{-1} u = minv .* u (Jacobi when minv = 1 / diag(A)). Right
 * preconditioning: A M^{-1} y = b, x = M^{-1} y.
 * ========================================================================= */
static void prec(int32_t n, double *out, const double *minv, const double *in)
{
    for (int32_t i = 0; i < n; i++) out[i] = minv[i] * in[i];
}

/* Algorithm 10: preconditioned BiCGStab. */
int o_bicgstab_prec(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *minv,
                    const double *b, double *x, double rtol, int32_t maxit, int32_t fixed_iters,
                    double *hist, double *trace_x, double *trace_r, o_info *info)
{
    o_csr A = {n, rowptr, col, val};
    o_trace tr = {hist, trace_x, trace_r};
    o_count cnt = {0.0, 0};
    memset(info, 0, sizeof(*info));
    if (n < 0 || maxit < 0 || !minv) return info->status = O_ERR_ARG;
    double *mem = (double *)calloc((size_t)10 * (n > 0 ? n : 1), sizeof(double));
    if (!mem) return info->status = O_ERR_OOM;
    double *r = mem, *r0 = r + n, *p = r0 + n, *ph = p + n, *s = ph + n, *q = s + n, *qh = q + n, *y = qh + n,
           *tmp = y + n;
    int32_t limit = fixed_iters > 0 ? fixed_iters : maxit;

    /* r_0 := b - A x_0; p_0 := r_0 */
    spmv(&A, x, tmp, &cnt);
    for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
    memcpy(r0, r, sizeof(double) * n);
    memcpy(p, r, sizeof(double) * n);
    double rho = dot(n, r0, r, NULL);
    double nr = norm2(n, r);
    info->nr0 = nr;
    record(&tr, 0, n, nr, x, r);
    double tol = rtol * info->nr0;
    info->status = O_NOT_CONVERGED;
    if (info->nr0 == 0.0) { info->status = O_CONVERGED; finish(&A, b, x, tmp, nr, info, &cnt); free(mem); return info->status; }

    int32_t i;
    for (i = 0; i < limit; i++) {
        /* p^_i := M^{-1} p_i; s_i := A p^_i */
        prec(n, ph, minv, p);
        spmv(&A, ph, s, &cnt);
        double r0s = dot(n, r0, s, &cnt);
        if (!isfinite(r0s)) { info->status = O_NONFINITE; break; }
        if (r0s == 0.0) { info->status = O_BREAKDOWN; break; }
        double alpha = rho / r0s;
        /* q_i := r_i - alpha_i s_i; q^_i := M^{-1} q_i; y_i := A q^_i */
        axpy(n, q, r, -alpha, s, &cnt);
        prec(n, qh, minv, q);
        spmv(&A, qh, y, &cnt);
        double qy = dot(n, q, y, &cnt), yy = dot(n, y, y, &cnt), qq = dot(n, q, q, NULL);
        double d1[3] = {qy, yy, qq};
        if (!finite_all(3, d1)) { info->status = O_NONFINITE; break; }
        if ((fixed_iters <= 0 && sqrt(qq) <= tol) || yy == 0.0) {
            if (yy == 0.0 && qq != 0.0 && !(fixed_iters <= 0 && sqrt(qq) <= tol)) { info->status = O_BREAKDOWN; break; }
            axpy(n, x, x, alpha, ph, &cnt);
            nr = sqrt(qq);
            info->half_step = 1;
            info->status = O_CONVERGED;
            record(&tr, i + 1, n, nr, x, q);
            i++;
            break;
        }
        double omega = qy / yy;
        if (omega == 0.0) { info->status = O_BREAKDOWN; break; }
        /* x_{i+1} := x_i + alpha_i p^_i + omega_i q^_i; r_{i+1} := q_i - omega_i y_i */
        axpy(n, x, x, alpha, ph, &cnt);
        axpy(n, x, x, omega, qh, &cnt);
        axpy(n, r, q, -omega, y, &cnt);
        double rho_new = dot(n, r0, r, &cnt);
        double rr = dot(n, r, r, NULL);
        double d2[2] = {rho_new, rr};
        nr = sqrt(rr);
        record(&tr, i + 1, n, nr, x, r);
        if (!finite_all(2, d2)) { info->status = O_NONFINITE; i++; break; }
        if (fixed_iters <= 0 && nr <= tol) { info->status = O_CONVERGED; i++; break; }
        if (rho_new == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        double beta = (alpha / omega) * (rho_new / rho);
        rho = rho_new;
        /* p_{i+1} := r_{i+1} + beta_i (p_i - omega_i s_i) */
        axpy(n, p, p, -omega, s, &cnt);
        axpy(n, p, r, beta, p, &cnt);
    }
    if (fixed_iters > 0 && info->status == O_NOT_CONVERGED && i == limit) info->status = O_CONVERGED;
    info->iters = i;
    finish(&A, b, x, tmp, nr, info, &cnt);
    free(mem);
    return info->status;
}

/* Algorithm 11: preconditioned pipelined BiCGStab, with the residual
 * replacement of Section 4.2 in the split placement used by o_pbicgstab:
 * r_i := b - A x_i, r^_i := M^{-1} r_i, w_i := A r^_i before the second
 * reduction of iteration i-1 (so w^_i = M^{-1} w_i and t_i = A w^_i follow
 * from the replaced w_i), and s_i := A p^_i, s^_i := M^{-1} s_i,
 * z_i := A s^_i after p^_i. 4 SpMVs and 2 preconditioner applications. */
int o_pbicgstab_prec(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *minv,
                     const double *b, double *x, double rtol, int32_t maxit, int32_t fixed_iters,
                     int32_t replace_period, int32_t max_replacements,
                     double *hist, double *trace_x, double *trace_r, o_info *info)
{
    o_csr A = {n, rowptr, col, val};
    o_trace tr = {hist, trace_x, trace_r};
    o_count cnt = {0.0, 0};
    memset(info, 0, sizeof(*info));
    if (n < 0 || maxit < 0 || !minv) return info->status = O_ERR_ARG;
    double *mem = (double *)calloc((size_t)17 * (n > 0 ? n : 1), sizeof(double));
    if (!mem) return info->status = O_ERR_OOM;
    double *r = mem, *rh = r + n, *r0 = rh + n, *ph = r0 + n, *s = ph + n, *sh = s + n, *z = sh + n, *zh = z + n,
           *q = zh + n, *qh = q + n, *y = qh + n, *w = y + n, *wh = w + n, *t = wh + n, *v = t + n, *tmp = v + n;
    int32_t limit = fixed_iters > 0 ? fixed_iters : maxit;

    /* r_0 := b - A x_0; r^_0 := M^{-1} r_0; w_0 := A r^_0; w^_0 := M^{-1} w_0; t_0 := A w^_0;
     * alpha_0 := (r0, r0) / (r0, w0); beta_{-1} := 0 */
    spmv(&A, x, tmp, &cnt);
    for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
    memcpy(r0, r, sizeof(double) * n);
    prec(n, rh, minv, r);
    spmv(&A, rh, w, &cnt);
    prec(n, wh, minv, w);
    spmv(&A, wh, t, &cnt);
    double rho = dot(n, r0, r, NULL);
    double r0w = dot(n, r0, w, NULL);
    double nr = norm2(n, r);
    info->nr0 = nr;
    record(&tr, 0, n, nr, x, r);
    double tol = rtol * info->nr0;
    info->status = O_NOT_CONVERGED;
    int32_t i = 0;
    double alpha = 0.0, beta = 0.0, omega = 0.0;
    int replaced = 0;
    if (info->nr0 == 0.0) { info->status = O_CONVERGED; goto out; }
    if (r0w == 0.0 || !isfinite(r0w)) { info->status = isfinite(r0w) ? O_BREAKDOWN : O_NONFINITE; goto out; }
    alpha = rho / r0w;

    for (i = 0; i < limit; i++) {
        /* p^_i := r^_i + beta (p^_{i-1} - omega s^_{i-1}) */
        axpy(n, ph, ph, -omega, sh, &cnt);
        axpy(n, ph, rh, beta, ph, &cnt);
        if (replaced) {
            spmv(&A, ph, s, &cnt);
            prec(n, sh, minv, s);
            spmv(&A, sh, z, &cnt);
        } else {
            /* s_i := w_i + beta (s_{i-1} - omega z_{i-1}); s^_i := w^_i + beta (s^_{i-1} - omega z^_{i-1});
             * z_i := t_i + beta (z_{i-1} - omega v_{i-1}) */
            axpy(n, s, s, -omega, z, &cnt);
            axpy(n, s, w, beta, s, &cnt);
            axpy(n, sh, sh, -omega, zh, &cnt);
            axpy(n, sh, wh, beta, sh, &cnt);
            axpy(n, z, z, -omega, v, &cnt);
            axpy(n, z, t, beta, z, &cnt);
        }
        /* q_i := r_i - alpha s_i; q^_i := r^_i - alpha s^_i; y_i := w_i - alpha z_i */
        axpy(n, q, r, -alpha, s, &cnt);
        axpy(n, qh, rh, -alpha, sh, &cnt);
        axpy(n, y, w, -alpha, z, &cnt);
        double qy = dot(n, q, y, &cnt), yy = dot(n, y, y, &cnt), qq = dot(n, q, q, NULL);
        /* z^_i := M^{-1} z_i; v_i := A z^_i */
        prec(n, zh, minv, z);
        spmv(&A, zh, v, &cnt);
        double d1[3] = {qy, yy, qq};
        if (!finite_all(3, d1)) { info->status = O_NONFINITE; break; }
        if ((fixed_iters <= 0 && sqrt(qq) <= tol) || yy == 0.0) {
            if (yy == 0.0 && qq != 0.0 && !(fixed_iters <= 0 && sqrt(qq) <= tol)) { info->status = O_BREAKDOWN; break; }
            axpy(n, x, x, alpha, ph, &cnt);
            nr = sqrt(qq);
            info->half_step = 1;
            info->status = O_CONVERGED;
            record(&tr, i + 1, n, nr, x, q);
            i++;
            break;
        }
        omega = qy / yy;
        if (omega == 0.0) { info->status = O_BREAKDOWN; break; }
        /* x_{i+1} := x_i + alpha p^_i + omega q^_i; r_{i+1} := q_i - omega y_i;
         * r^_{i+1} := q^_i - omega (w^_i - alpha z^_i); w_{i+1} := y_i - omega (t_i - alpha v_i) */
        axpy(n, x, x, alpha, ph, &cnt);
        axpy(n, x, x, omega, qh, &cnt);
        axpy(n, r, q, -omega, y, &cnt);
        axpy(n, tmp, wh, -alpha, zh, &cnt);
        axpy(n, rh, qh, -omega, tmp, &cnt);
        axpy(n, tmp, t, -alpha, v, &cnt);
        axpy(n, w, y, -omega, tmp, &cnt);
        replaced = replace_period > 0 && (i + 1) % replace_period == 0 &&
                   (max_replacements < 0 || info->n_replacements < max_replacements);
        if (replaced) {
            spmv(&A, x, tmp, &cnt);
            for (int32_t j = 0; j < n; j++) r[j] = b[j] - tmp[j];
            prec(n, rh, minv, r);
            spmv(&A, rh, w, &cnt);
            info->n_replacements++;
        }
        double rho_new = dot(n, r0, r, &cnt), r0w_new = dot(n, r0, w, &cnt);
        double r0s = dot(n, r0, s, &cnt), r0z = dot(n, r0, z, &cnt);
        double rr = dot(n, r, r, NULL);
        /* w^_{i+1} := M^{-1} w_{i+1}; t_{i+1} := A w^_{i+1} */
        prec(n, wh, minv, w);
        spmv(&A, wh, t, &cnt);
        double d2[5] = {rho_new, r0w_new, r0s, r0z, rr};
        nr = sqrt(rr);
        record(&tr, i + 1, n, nr, x, r);
        if (!finite_all(5, d2)) { info->status = O_NONFINITE; i++; break; }
        if (fixed_iters <= 0 && nr <= tol) { info->status = O_CONVERGED; i++; break; }
        if (rho_new == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        beta = (alpha / omega) * (rho_new / rho);
        double den = r0w_new + beta * r0s - beta * omega * r0z;
        if (den == 0.0) { info->status = O_BREAKDOWN; i++; break; }
        alpha = rho_new / den;
        rho = rho_new;
    }
    if (fixed_iters > 0 && info->status == O_NOT_CONVERGED && i == limit) info->status = O_CONVERGED;
out:
    info->iters = i;
    finish(&A, b, x, tmp, nr, info, &cnt);
    free(mem);
    return info->status;
}
