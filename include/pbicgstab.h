/*
 * pbicgstab.h -- C ABI of the GB300 pipelined BiCGStab library.
 *
 * Solves A x = b for a real unsymmetric sparse A (CSR or 5/7-point stencil) in
 * FP64 on one NVIDIA GB300 GPU with
 *   - pipelined BiCGStab (p-BiCGStab), Cools & Vanroose, arXiv:1612.01395,
 *     Algorithm 9 (Section 3.3), with the residual replacement of Section 4.2;
 *   - standard BiCGStab, Algorithm 7 (Section 3.1), for comparison.
 *
 * Conventions
 *   - Pointers named d_* are device pointers (CUDA global memory of the device
 *     that was current at create); h_* are host pointers. Vectors are dense
 *     FP64 arrays of length n, indices int32, CSR rows sorted or not.
 *   - The caller owns every buffer: the matrix, the workspace, b, x and the
 *     optional history. The library never allocates or frees device memory;
 *     all scratch lives in the caller's workspace (size from
 *     pbicgstab_workspace_bytes). Buffers must stay valid while a handle that
 *     refers to them is in use.
 *   - Work is enqueued on the stream given at create. A solve returns after its
 *     result summary (pbcg_info) is on the host: one stream synchronisation per
 *     solve and none per iteration. Two solves on the same handle must not run
 *     concurrently (they share the workspace).
 *   - No call throws; each returns a pbcg_status. pbicgstab_last_error() gives
 *     a message for the last failing call of the calling thread.
 *   - Results are deterministic: dot products are reduced in a fixed order, so
 *     the same inputs on the same GPU give bitwise identical outputs.
 */
#ifndef PBICGSTAB_H
#define PBICGSTAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pbicgstab_s *pbicgstab_t;

typedef enum {
    PBCG_OK = 0,            /* converged (or ran the requested fixed_iters) */
    PBCG_NOT_CONVERGED = 1, /* maxit reached before the tolerance */
    PBCG_BREAKDOWN = 2,     /* zero denominator of alpha, (y,y) = 0 with q != 0,
                               omega = 0, or (r0, r_{i+1}) = 0; x is the last
                               full iterate */
    PBCG_NONFINITE = 3,     /* a reduced scalar is Inf/NaN; x is the last full iterate */
    PBCG_ERR_ARG = 4,       /* invalid argument (message in pbicgstab_last_error) */
    PBCG_ERR_CUDA = 5,      /* a CUDA runtime call failed */
    PBCG_ERR_OOM = 6,       /* workspace too small */
    PBCG_ERR_TIMEOUT = 7    /* a device-side grid synchronisation exceeded its time
                               limit; results are invalid, the context stays usable */
} pbcg_status;

/* Preconditioners (right preconditioning, Section 3.6): none, or Jacobi
 * M = diag(A), applied elementwise inside the sweeps of Algorithms 10 and 11. */
typedef enum { PBCG_PREC_NONE = 0, PBCG_PREC_JACOBI = 1 } pbcg_prec;

/* One stencil coefficient as a function of the grid node (i, j, k):
 *   c(i,j,k) = (data  ? data [i*stride[0]  + j*stride[1]  + k*stride[2]]  : value)
 *            + (data2 ? data2[i*stride2[0] + j*stride2[1] + k*stride2[2]] : nothing)
 * data/data2 are device pointers. A stride of 0 makes the coefficient constant
 * along that axis, so constants, 1-D/2-D tables and full 3-D fields all fit.
 * Strides must be >= 0; create rejects a table whose largest index over the
 * grid is >= its len. */
typedef struct {
    double value;
    const double *data;
    int64_t stride[3];
    int64_t len;          /* elements readable at data (every index used must be < len) */
    const double *data2;
    int64_t stride2[3];
    int64_t len2;         /* elements readable at data2 */
} pbcg_coef;

/* Direction indices of pbcg_stencil.coef. */
enum { PBCG_C = 0, PBCG_W = 1, PBCG_E = 2, PBCG_S = 3, PBCG_N = 4, PBCG_B = 5, PBCG_T = 6 };

/* A 5-point (nz == 1) or 7-point stencil on an nx x ny x nz grid, rows ordered
 * lexicographically with x fastest: row = i + nx*(j + ny*k). Row `row` of A has
 * coef[C] on the diagonal and coef[W]/[E] at columns row -/+ 1, coef[S]/[N] at
 * row -/+ nx, coef[B]/[T] at row -/+ nx*ny, each evaluated at the row's node;
 * neighbours outside the grid are dropped (Dirichlet elimination). A row is
 * summed in the order B, S, W, C, E, N, T (ascending column), which makes the
 * stencil and the equivalent sorted CSR give identical products. */
typedef struct {
    int32_t nx, ny, nz;
    pbcg_coef coef[7];
} pbcg_stencil;

/* Per-solve options; pass NULL for the defaults shown. */
typedef struct {
    int32_t max_replacements; /* cap on residual replacements, -1 = unlimited (default -1) */
    int32_t fixed_iters;      /* > 0: run exactly this many iterations and ignore rtol
                                 (breakdown still stops); for step-by-step comparison (default 0) */
    double *d_history;        /* NULL, or device buffer of (fixed_iters>0 ? fixed_iters : maxit)+1
                                 doubles: ||r_i||_2 of the recursive residual, i = 0..iters;
                                 entries past iters are untouched (default NULL) */
    int32_t plain_variant;    /* bicgstab_solve only: 0 = automatic, 3 = three grid-wide
                                 synchronisations per iteration with neighbour values of p and
                                 q formed on the fly, 5 = five synchronisations and fewer FP64
                                 operations (default 0) */
    int32_t grid;             /* 0 = automatic; > 0 forces the number of thread blocks
                                 (clamped to what can be co-resident) (default 0) */
    double *d_inner_history;  /* pbicgstab_solve_mixed only: NULL, or device buffer of
                                 (fixed_iters>0 ? fixed_iters : inner_maxit)+1 doubles that
                                 receives ||r_i||_2 of the recursive residual of the FIRST
                                 refinement step's inner solve, i = 0..its iterations (entry 0
                                 is the norm of the FP32 right-hand side) (default NULL) */
    int32_t cluster;          /* pbicgstab_solve / bicgstab_solve on an unpreconditioned handle:
                                 0 = automatic (systems of up to 24576 stored entries -- stencil:
                                 points x unknowns -- are solved by one thread-block cluster,
                                 larger ones by a cooperative grid); -1 = always the
                                 cooperative grid; 2, 4, 8 or 16 = one cluster of that many CTAs
                                 (default 0; ignored when grid > 0). A PBCG_PREC_JACOBI handle
                                 always takes the grid, and a positive value, or a size the
                                 device cannot make resident, returns PBCG_ERR_ARG */
    int32_t stall_steps;      /* pbicgstab_solve_mixed only: stop (PBCG_NOT_CONVERGED) after this
                                 many refinement steps in a row that fail to bring the FP64
                                 residual below the best one so far; 0 = the default, 6 (converging
                                 refinements with capped inner solves were measured to have up
                                 to 4 such steps in a row) */
} pbcg_opts;

/* Result summary, written to host memory by every solve. */
typedef struct {
    int32_t iters;            /* iterations performed; a final half step counts as one */
    int32_t status;           /* pbcg_status of the solve */
    int32_t half_step;        /* 1 if it stopped at x_i + alpha_i p_i because ||q_i|| <= tol */
    int32_t n_replacements;   /* residual replacement steps performed */
    double nr0;               /* ||r_0||_2 = ||b - A x_0||_2 */
    double rel_res_recursive; /* ||r_iters||_2 / ||r_0||_2 (recursive residual) */
    double rel_res_true;      /* ||b - A x||_2 / ||r_0||_2, computed after the loop */
    int32_t grid;             /* thread blocks used */
    int32_t block;            /* threads per block */
    int32_t grid_syncs;       /* device-wide synchronisations performed */
    int32_t spmvs;            /* sparse matrix-vector products performed */
    float kernel_ms;          /* duration of the solver kernel, CUDA events on the handle's stream */
    int32_t cluster;          /* > 0: the solve ran on one thread-block cluster of this many CTAs
                                 (grid == cluster); 0: on a cooperative grid */
} pbcg_info;

/* Bytes of device workspace a handle for n unknowns needs (256-byte aligned
 * start required). Covers 12 FP64 vectors of length n and a control block. */
size_t pbicgstab_workspace_bytes(int32_t n);

/* Workspace of a handle created with PBCG_PREC_JACOBI: 6 more FP64 vectors
 * (M^{-1} and the preconditioned vectors r^, s^, z^, q^, w^ of Algorithm 11). */
size_t pbicgstab_workspace_bytes_prec(int32_t n);

/* Create a handle for a CSR matrix (Section 3: A general sparse, unsymmetric).
 *   n, nnz         size; 0 <= n, 0 <= nnz < 2^31
 *   d_rowptr[n+1]  row offsets (d_rowptr[0] == 0, non-decreasing, d_rowptr[n] == nnz)
 *   d_col[nnz]     column indices in [0, n)
 *   d_val[nnz]     values
 *   prec           PBCG_PREC_NONE, or PBCG_PREC_JACOBI (M^{-1} = 1/diag(A) computed here;
 *                  a zero or missing diagonal entry returns PBCG_ERR_ARG)
 *   d_workspace    caller-owned, >= pbicgstab_workspace_bytes(n) bytes (PBCG_PREC_JACOBI:
 *                  pbicgstab_workspace_bytes_prec(n)), 256-byte aligned
 *   stream         a cudaStream_t (NULL = legacy default stream)
 * The structure is validated on the device (one synchronisation); an invalid
 * matrix returns PBCG_ERR_ARG and no handle. */
pbcg_status pbicgstab_create_csr(int32_t n, int32_t nnz, const int32_t *d_rowptr, const int32_t *d_col,
                                 const double *d_val, pbcg_prec prec, void *d_workspace, size_t ws_bytes,
                                 void *stream, pbicgstab_t *out);

/* Create a handle for a stencil operator (Section 5, PTP1/PTP2 are such
 * stencils). desc is copied; its coefficient tables must stay valid. */
pbcg_status pbicgstab_create_stencil(const pbcg_stencil *desc, pbcg_prec prec, void *d_workspace,
                                     size_t ws_bytes, void *stream, pbicgstab_t *out);

/* Pipelined BiCGStab, Algorithm 9 (Algorithm 11 on a PBCG_PREC_JACOBI handle),
 * with residual replacement (Section 4.2; preconditioned: r, r^, w, s, s^, z).
 *   d_b[n]           right-hand side
 *   d_x[n]           in: x_0; out: the last iterate
 *   rtol             stop when ||r_i||_2 <= rtol * ||r_0||_2 on the recursive residual
 *   maxit            iteration cap (>= 0)
 *   replace_period   k > 0: replace r, w, s, z by their true values every k
 *                    iterations (r := b - A x and w := A r before the second
 *                    reduction of iteration i-1, s := A p and z := A s after p_i
 *                    in iteration i, for i mod k == 0); 0 disables
 *   opts             NULL or options
 *   info             host pointer, filled on return (also on failure when possible)
 * Returns info->status, or an error code. */
pbcg_status pbicgstab_solve(pbicgstab_t h, const double *d_b, double *d_x, double rtol, int32_t maxit,
                            int32_t replace_period, const pbcg_opts *opts, pbcg_info *info);

/* Standard BiCGStab, Algorithm 7 (Algorithm 10 on a PBCG_PREC_JACOBI handle,
 * always in the five-exchange form), on the same handle and workspace.
 * Arguments as pbicgstab_solve without replacement. */
pbcg_status bicgstab_solve(pbicgstab_t h, const double *d_b, double *d_x, double rtol, int32_t maxit,
                           const pbcg_opts *opts, pbcg_info *info);

/* pbicgstab_solve on HOST buffers: copies h_b and h_x (x_0) to the workspace,
 * solves, and copies the iterate back into h_x; all on the handle's stream.
 * Page-locked host buffers give the fastest copies. method: 0 = pipelined
 * (Algorithm 9), 1 = standard (Algorithm 7, replace_period ignored). */
pbcg_status pbicgstab_solve_host(pbicgstab_t h, int32_t method, const double *h_b, double *h_x, double rtol,
                                 int32_t maxit, int32_t replace_period, const pbcg_opts *opts, pbcg_info *info);

/* y = A x with the handle's operator (the SpMV building block, Section 1).
 * Asynchronous on the handle's stream; d_x and d_y must not overlap. Each
 * row is one chain of FP64 fused multiply-adds, acc = fma(a, x[col], acc)
 * from acc = 0, over the row's entries in storage order (CSR) or in the
 * order B, S, W, C, E, N, T (stencil); the solvers form their products the
 * same way. */
pbcg_status pbicgstab_spmv(pbicgstab_t h, const double *d_x, double *d_y);

/* Number of unknowns of the handle. */
int32_t pbicgstab_size(pbicgstab_t h);

/* Result summary of pbicgstab_solve_mixed. */
typedef struct {
    int32_t outer;            /* refinement steps performed (inner solves) */
    int32_t inner_iters;      /* inner iterations summed over all steps */
    int32_t status;           /* PBCG_OK once ||b - A x|| <= rtol ||b - A x0|| in FP64 */
    int32_t grid;             /* thread blocks used */
    double nr0;               /* ||b - A x0||_2 */
    double rel_res_true;      /* ||b - A x||_2 / ||b - A x0||_2 at exit, in FP64 */
    int32_t grid_syncs;       /* device-wide synchronisations performed */
    int32_t spmvs;            /* sparse matrix-vector products (FP64 and low precision) */
    float kernel_ms;          /* duration of the solve kernel, CUDA events on the handle's stream */
    int32_t restored;         /* 1 if the solve stopped unconverged and x was reset to the best
                                 iterate (the one with the smallest FP64 residual) */
} pbcg_mixed_info;

/* Low-precision value types for pbicgstab_solve_mixed. */
enum { PBCG_VALUES_F32 = 0, PBCG_VALUES_BF16 = 1 };

/* Mixed-precision solve (an extension of the paper's method, which states no
 * precision): FP64 iterative refinement around pipelined BiCGStab
 * (Algorithm 9) run on FP32 vectors. Each step computes r = b - A x with the
 * handle's FP64 operator, solves A d = r with the FP32 pipelined iteration
 * to ||r_inner|| <= inner_rtol ||r|| (at most inner_maxit iterations) on a
 * low-precision copy of A, and sets x := x + d in FP64. Dot products that set
 * alpha, beta and omega are summed per thread in compensated FP32 (algorithm
 * Dot2: as accurate as twice FP32 precision) and across threads in FP64; the
 * scalars are FP64.
 * Stops when the FP64 residual satisfies ||b - A x|| <= rtol ||b - A x0||
 * (PBCG_OK); after max_outer steps (PBCG_NOT_CONVERGED); or when
 * opts->stall_steps (default 6) steps in a row fail to bring the FP64
 * residual below the best one so far -- refinement does not contract, e.g.
 * when cond(A) times the rounding of the low-precision values exceeds 1
 * (PBCG_NOT_CONVERGED). A solve that stops unconverged returns
 * the best iterate (info->restored = 1 when that is not the last one) and
 * info->rel_res_true is that iterate's residual.
 *   h            a CSR or stencil handle
 *   d_val_lowp   CSR handle: nnz values of the same CSR structure as float
 *                (PBCG_VALUES_F32) or bfloat16 (PBCG_VALUES_BF16),
 *                caller-owned. Stencil handle: NULL with PBCG_VALUES_F32; the
 *                library rounds the coefficient tables to FP32 into the
 *                workspace each call (PBCG_ERR_ARG if they need more than the
 *                10 * round32(n) floats the inner vectors and the copy of the
 *                best iterate leave free, or for other arguments)
 *   opts         NULL or options; d_history (max_outer + 1 doubles) receives
 *                the FP64 residual norm before each step; grid as for solve;
 *                fixed_iters > 0 makes every inner solve run exactly that many
 *                iterations (inner_rtol ignored; for step-by-step comparison);
 *                d_inner_history receives the first inner solve's residual norms
 * Uses the handle's workspace (no extra memory). */
pbcg_status pbicgstab_solve_mixed(pbicgstab_t h, const void *d_val_lowp, int32_t lowp_type, const double *d_b,
                                  double *d_x, double rtol, int32_t max_outer, double inner_rtol,
                                  int32_t inner_maxit, const pbcg_opts *opts, pbcg_mixed_info *info);

/* Batched solves: nsys independent CSR systems concatenated. System s owns
 * rows [row_offset[s], row_offset[s+1]) of the concatenation; d_rowptr holds
 * offsets into the shared d_col / d_val arrays (total nnz < 2^31); column
 * indices are local to their system (0 <= col < n_s). */
typedef struct {
    int32_t nsys;
    int32_t nnz;                   /* total stored entries (length of d_col and d_val) */
    const int64_t *d_row_offset;   /* [nsys + 1], d_row_offset[0] == 0 */
    const int32_t *d_rowptr;       /* [total rows + 1] */
    const int32_t *d_col;
    const double *d_val;
} pbcg_batch;

/* Per-system result of a batched solve (written to device memory). */
typedef struct {
    int32_t iters;
    int32_t status;           /* pbcg_status; PBCG_ERR_ARG for an invalid system structure */
    int32_t half_step;
    int32_t n_replacements;
    double rel_res_recursive;
    double rel_res_true;
} pbcg_batch_result;

/* Launch shape of a batched solve. A large system is solved by all CTAs of a
 * thread-block cluster (rows split between them, reductions through the
 * cluster's distributed shared memory); a small one by a single CTA.
 * Zero fields take the defaults. */
typedef struct {
    int32_t cluster_size;       /* CTAs per cluster: 1 (no clusters), 2, 4, 8 or 16; 0 = 8 */
    int32_t fixed_iters;        /* > 0: every system runs exactly this many iterations and
                                   ignores rtol (breakdown still stops); for step-by-step
                                   comparison (default 0) */
    int64_t cluster_min_rows;   /* systems with at least this many rows use a whole cluster; 0 = 512 */
    double *d_history;          /* NULL, or device buffer of nsys * history_stride doubles:
                                   ||r_i||_2 of system s's recursive residual at
                                   d_history[s * history_stride + i], i = 0..its iterations;
                                   entries past them are untouched (default NULL) */
    int64_t history_stride;     /* >= (fixed_iters > 0 ? fixed_iters : maxit) + 1 when
                                   d_history is set (PBCG_ERR_ARG otherwise) */
} pbcg_batch_opts;

/* Workspace of a batched solve: 10 FP64 vectors over all rows + a counter. */
size_t pbicgstab_batched_workspace_bytes(int64_t total_rows);

/* Solve every system of the batch with pipelined BiCGStab (Algorithm 9 with
 * residual replacement every replace_period iterations, 0 = off), each to
 * ||r|| <= rtol ||r_0|| of its own, in one launch (an extension of the
 * paper's method to many small systems; no counterpart in the paper).
 * Systems converge independently: a system with at least
 * opts->cluster_min_rows rows is solved by the CTAs of one thread-block
 * cluster together, a smaller one by one CTA with block-level reductions;
 * clusters take systems in index order from a counter (order them largest
 * first). opts may be NULL (defaults); an unsupported cluster size returns
 * PBCG_ERR_ARG, and a cluster shape the GPU cannot make resident returns
 * PBCG_ERR_CUDA. Fully asynchronous on `stream`: no host
 * synchronisation and no allocation, so a call can be captured into a CUDA
 * graph and replayed. d_b, d_x (in: x0, out: x) span all rows; d_results
 * receives nsys pbcg_batch_result in device memory; the workspace must stay
 * untouched until the work completes. Column indices are checked on the
 * device per system (an invalid system gets PBCG_ERR_ARG and is skipped).
 * Host-side argument errors return PBCG_ERR_ARG immediately. */
pbcg_status pbicgstab_solve_batched(const pbcg_batch *batch, int64_t total_rows, const double *d_b, double *d_x,
                                    double rtol, int32_t maxit, int32_t replace_period, const pbcg_batch_opts *opts,
                                    void *d_workspace, size_t ws_bytes, pbcg_batch_result *d_results, void *stream);

/* Launch-shape autotuner for pbicgstab_solve_batched (no counterpart in the
 * paper): solves the batch once per candidate shape (cluster size 1, 2, 4, 8
 * or 16; cluster_min_rows 512, 4096 or 16384), each from x0 = 0 and timed
 * with CUDA events on `stream`, after one warm-up solve; then solves once
 * more with the fastest shape, so that on return d_x and d_results hold that
 * solve. *best receives the shape and *best_ms (if not NULL) its time. Other
 * arguments as pbicgstab_solve_batched; d_x is overwritten. Shapes the GPU
 * cannot make resident are skipped. Blocks the calling thread. */
pbcg_status pbicgstab_batched_autotune(const pbcg_batch *batch, int64_t total_rows, const double *d_b, double *d_x,
                                       double rtol, int32_t maxit, int32_t replace_period, void *d_workspace,
                                       size_t ws_bytes, pbcg_batch_result *d_results, void *stream,
                                       pbcg_batch_opts *best, float *best_ms);

/* Adjoint solves (an extension: reverse-mode gradients through a solve; the
 * paper has no counterpart). For x = A^{-1} b and a loss L(x), lambda solves
 * A^T lambda = dL/dx; then dL/db = lambda and dL/da_ij = -lambda_i x_j. */

/* Work buffer bytes of pbicgstab_csr_transpose. */
size_t pbicgstab_transpose_work_bytes(int32_t n);

/* A^T of an n x n CSR matrix into caller-owned arrays d_trowptr[n+1],
 * d_tcol[nnz], d_tval[nnz]; rows of A^T sorted by column (deterministic).
 * The input structure is validated on the device (one synchronisation);
 * invalid input returns PBCG_ERR_ARG. Otherwise asynchronous on `stream`. */
pbcg_status pbicgstab_csr_transpose(int32_t n, int32_t nnz, const int32_t *d_rowptr, const int32_t *d_col,
                                    const double *d_val, int32_t *d_trowptr, int32_t *d_tcol, double *d_tval,
                                    void *d_work, size_t work_bytes, void *stream);

/* d_grad[k] = -d_lambda[i] * d_x[d_col[k]] for every stored entry k of row i
 * (dL/da_ij). Asynchronous on `stream`. */
pbcg_status pbicgstab_csr_value_grad(int32_t n, const int32_t *d_rowptr, const int32_t *d_col,
                                     const double *d_lambda, const double *d_x, double *d_grad, void *stream);

/* Diagnostic of failure detection (no counterpart in the paper): runs, on
 * h's stream and workspace, a two-block grid synchronisation that one block
 * never joins, with each wait bounded by limit_ms (1..4000). The wait must end
 * at its limit; *status receives the status the device recorded
 * (PBCG_ERR_TIMEOUT when the bound works; PBCG_OK would mean the wait was not
 * bounded). Returns PBCG_ERR_ARG / PBCG_ERR_CUDA for bad arguments or a failed
 * launch, else PBCG_OK. The handle stays usable. Blocks the calling thread
 * until the probe ends. */
pbcg_status pbicgstab_probe_sync_timeout(pbicgstab_t h, int32_t limit_ms, int32_t *status);

/* Bounds-checked builds (the library compiled with -DPBCG_CHECK; a debugging
 * aid with no counterpart in the paper): the kernels check every index they
 * form from data or geometry -- CSR entry positions taken from the row
 * pointers (against nnz), gathered CSR columns, stencil neighbours and
 * stencil coefficient-table positions (against the table length reached over
 * the grid), and the gathered columns of the adjoint transpose and value
 * gradient; an out-of-range one is replaced by 0 so that no access leaves its
 * buffer, and the source line of the first is recorded on the current device.
 * Synchronises the device, returns that line (0: none since the last call) and
 * clears it; -2 if a CUDA call fails. The default build has no checks and
 * returns -1. */
int32_t pbicgstab_check_faults(void);

/* Largest system pbicgstab_solve_csr_noalloc accepts. */
#define PBCG_NOALLOC_MAX_N 32768

/* pbicgstab_solve for a CSR matrix without allocating anything and without a
 * handle or workspace. The paper has no counterpart: this serves callers that
 * may not allocate device memory or cannot provide a workspace -- e.g. code
 * inside an application that owns all device memory and forbids allocation
 * after start-up (cudaMalloc synchronises the device and can fail under
 * pressure), real-time loops, or plug-ins that only get input and output
 * pointers. Its scratch is a fixed array in the library's device memory sized
 * for PBCG_NOALLOC_MAX_N unknowns (about 3.4 MB), which every GPU that loads
 * the library keeps until the process exits.
 *   Arguments as pbicgstab_create_csr + pbicgstab_solve (CSR validated on the
 *   device each call; info->kernel_ms is 0). n > PBCG_NOALLOC_MAX_N returns
 *   PBCG_ERR_ARG.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture. The address is kept for the life of the process: after a
 *   cudaDeviceReset of that device the kept address is stale, so do not call
 *   this entry point on that device again.
 *   All calls on a device share the one array, and each call resets the parts
 *   that must start from a known state. Calls whose work overlaps on the GPU
 *   (other streams, other host threads) race on it; serialise them.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
pbcg_status pbicgstab_solve_csr_noalloc(int32_t n, int32_t nnz, const int32_t *d_rowptr, const int32_t *d_col,
                                        const double *d_val, const double *d_b, double *d_x, double rtol,
                                        int32_t maxit, int32_t replace_period, const pbcg_opts *opts, void *stream,
                                        pbcg_info *info);

/* Release the handle (host memory only; the caller's buffers are untouched).
 * Synchronises the handle's stream first. NULL is ignored. */
void pbicgstab_destroy(pbicgstab_t h);

/* Message of the last failing call on this thread ("" if none). */
const char *pbicgstab_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PBICGSTAB_H */
