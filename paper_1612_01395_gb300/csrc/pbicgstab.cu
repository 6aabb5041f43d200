// C ABI of the library (declared in include/pbicgstab.h): argument checks,
// workspace layout, launch-shape choice and the cooperative launches.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "pbicgstab.h"
#include "adjoint.cuh"
#include "solvers.cuh"

namespace {

// A named range on the host timeline of profilers that read NVTX (header-only
// NVTX3: without an attached tool each call is a no-op). A solve is one
// kernel, so ranges mark library calls, not solver phases.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

thread_local char g_err[512] = "";

pbcg_status fail(pbcg_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define PBCG_CUDA(call)                                                                                  \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return fail(PBCG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kVectors = 12;   // r r0 p s z q y w t v + host staging b, x
constexpr int kPrecVectors = 6;   // preconditioned handles: M^{-1}, r^ s^ z^ q^ w^

size_t vec_stride(int32_t n) { return ((size_t)(n > 0 ? n : 1) + 31) / 32 * 32; }   // doubles

pbcg::CsrOpChunked chunked(const pbcg::CsrOpScalar &a) { return pbcg::CsrOpChunked{a.n, a.rowptr, a.col, a.val, a.nnz}; }

}  // namespace

struct pbicgstab_s {
    int kind;   // 0 = CSR, 1 = stencil
    pbcg::CsrOpScalar csr;   // CSR arrays
    bool csr_chunked;        // CSR: solver and SpMV use pbcg::CsrOpChunked (long rows)
    pbcg::StencilOp st;
    int n;
    char *ws;
    cudaStream_t stream;
    int device, num_sms;
    int occ_pipe, occ_plain;   // co-resident blocks per SM of each solver kernel
    pbcg::Vectors V;
    double *b_stage, *x_stage;
    pbcg::Control *ctl;
    double *partials;
    cudaEvent_t ev0, ev1;   // bracket the solver kernel
    int prec;               // pbcg_prec of the handle
    int occ_pipe_prec, occ_plain_prec;
    double *minv, *rh, *sh, *zh, *qh, *wh;   // Jacobi: M^{-1} and the hat vectors
    long long st_len[7][2];  // stencil: table elements the grid reaches (0: no table)
    long long nnz;           // stored entries (stencil: 7 per row), for the launch shape
    int cluster_max;         // largest resident cluster of the cluster solver (16 or 8; 0: none)
};

extern "C" {

size_t pbicgstab_workspace_bytes(int32_t n) {
    if (n < 0) return 0;
    return pbcg::kControlBytes + pbcg::kPartialBytes + (size_t)kVectors * vec_stride(n) * sizeof(double);
}

size_t pbicgstab_workspace_bytes_prec(int32_t n) {
    if (n < 0) return 0;
    return pbicgstab_workspace_bytes(n) + (size_t)kPrecVectors * vec_stride(n) * sizeof(double);
}

const char *pbicgstab_last_error(void) { return g_err; }

int32_t pbicgstab_size(pbicgstab_t h) { return h ? h->n : -1; }

}  // extern "C"

namespace {

template <class Op>
pbcg_status occupancy(int *pipe, int *plain) {
    PBCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(pipe, pbcg::pbicgstab_kernel<Op, false>, pbcg::kTPB, 0));
    PBCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(plain, pbcg::bicgstab_kernel<Op, false>, pbcg::kTPB, 0));
    if (*pipe < 1 || *plain < 1) return fail(PBCG_ERR_CUDA, "solver kernel cannot be resident on an SM");
    return PBCG_OK;
}

template <class Op>
pbcg_status occupancy_prec(int *pipe, int *plain) {
    PBCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(pipe, pbcg::pbicgstab_kernel<Op, true>, pbcg::kTPB, 0));
    PBCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(plain, pbcg::bicgstab_kernel<Op, true>, pbcg::kTPB, 0));
    if (*pipe < 1 || *plain < 1) return fail(PBCG_ERR_CUDA, "solver kernel cannot be resident on an SM");
    return PBCG_OK;
}

pbcg_status common_init(pbicgstab_s *h, int32_t n, pbcg_prec prec, void *d_ws, size_t ws_bytes, void *stream,
                        bool events = true) {
    if (prec != PBCG_PREC_NONE && prec != PBCG_PREC_JACOBI)
        return fail(PBCG_ERR_ARG, "unknown preconditioner %d", (int)prec);
    if (!d_ws) return fail(PBCG_ERR_ARG, "workspace is NULL");
    if (((uintptr_t)d_ws) % kAlign) return fail(PBCG_ERR_ARG, "workspace must be 256-byte aligned");
    const size_t need = prec == PBCG_PREC_JACOBI ? pbicgstab_workspace_bytes_prec(n) : pbicgstab_workspace_bytes(n);
    h->prec = (int)prec;
    if (ws_bytes < need) return fail(PBCG_ERR_OOM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    h->n = n;
    h->ws = (char *)d_ws;
    h->stream = (cudaStream_t)stream;
    PBCG_CUDA(cudaGetDevice(&h->device));
    PBCG_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    int coop = 0;
    PBCG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    if (!coop) return fail(PBCG_ERR_CUDA, "device does not support cooperative launches");
    if (events) {
        PBCG_CUDA(cudaEventCreate(&h->ev0));
        PBCG_CUDA(cudaEventCreate(&h->ev1));
    }
    h->ctl = (pbcg::Control *)h->ws;
    h->partials = (double *)(h->ws + pbcg::kControlBytes);
    double *v0 = (double *)(h->ws + pbcg::kControlBytes + pbcg::kPartialBytes);
    const size_t s = vec_stride(n);
    double **slots[kVectors] = {&h->V.r, &h->V.r0, &h->V.p, &h->V.s, &h->V.z, &h->V.q,
                                &h->V.y, &h->V.w, &h->V.t, &h->V.v, &h->b_stage, &h->x_stage};
    for (int k = 0; k < kVectors; ++k) *slots[k] = v0 + (size_t)k * s;
    if (prec == PBCG_PREC_JACOBI) {
        double **pslots[kPrecVectors] = {&h->minv, &h->rh, &h->sh, &h->zh, &h->qh, &h->wh};
        for (int k = 0; k < kPrecVectors; ++k) *pslots[k] = v0 + (size_t)(kVectors + k) * s;
    }
    return PBCG_OK;
}

// M^{-1} = 1 / diag(A) into the workspace; a zero diagonal is an argument error.
template <class Launch>
pbcg_status setup_jacobi(pbicgstab_s *h, Launch launch) {
    int *flag = &h->ctl->abort;
    PBCG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), h->stream));
    int blocks = (h->n + 255) / 256;
    if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
    if (blocks < 1) blocks = 1;
    launch(blocks, flag);
    PBCG_CUDA(cudaGetLastError());
    int bad = 0;
    PBCG_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PBCG_CUDA(cudaStreamSynchronize(h->stream));
    if (bad) return fail(PBCG_ERR_ARG, "Jacobi preconditioner: a diagonal entry is zero or missing");
    return PBCG_OK;
}

// Largest table index a strided coefficient reaches over the grid.
long long max_index(const int64_t st[3], int nx, int ny, int nz) {
    return st[0] * (long long)(nx - 1) + st[1] * (long long)(ny - 1) + st[2] * (long long)(nz - 1);
}

int pick_grid(const pbicgstab_s *h, int occ, int req) {
    int max_grid = occ * h->num_sms;
    if (max_grid > pbcg::kMaxGrid) max_grid = pbcg::kMaxGrid;
    if (req > 0) return req < max_grid ? req : max_grid;
    // The time of an iteration is the sweep (rows per thread, one after the
    // other) plus the grid-wide exchanges, whose cost grows with the number of
    // blocks. Block counts by work, measured on GB300 for both methods (60
    // iterations; the optimum was flat within a few per cent around these).
    // Work w = rows x max(1, entries per row / 7): for 5- and 7-point stencils
    // 128 blocks up to w = 80k, then 2, 3, 4, 5 blocks per SM up to 180k,
    // 400k, 1.2M, 3M and all co-resident blocks beyond; never fewer than one
    // row per thread up to that count. Rows of ~21 random entries preferred
    // one row per thread up to 256 blocks, which the work scaling gives.
    const long long n = h->n;
    const double per_row = n > 0 ? (double)h->nnz / (double)n : 0.0;
    const double w = (double)n * (per_row > 7.0 ? per_row / 7.0 : 1.0);
    long long want;
    if (w <= 80000.0) {
        want = 128;
    } else {
        const int per_sm = w <= 180000.0 ? 2 : w <= 400000.0 ? 3 : w <= 1200000.0 ? 4 : w <= 3000000.0 ? 5 : occ;
        want = (long long)per_sm * h->num_sms;
    }
    const long long one_row = (n + pbcg::kTPB - 1) / pbcg::kTPB;
    if (want > one_row) want = one_row;
    if (want < 1) want = 1;
    return (int)(want < max_grid ? want : max_grid);
}

template <class Op>
pbcg_status launch_solver(pbicgstab_s *h, const Op &op, bool pipelined, const pbcg::SolveArgs &args, int grid) {
    void *params[2] = {(void *)&op, (void *)&args};
    const void *fn = pipelined ? (args.minv ? (const void *)pbcg::pbicgstab_kernel<Op, true>
                                            : (const void *)pbcg::pbicgstab_kernel<Op, false>)
                               : (args.minv ? (const void *)pbcg::bicgstab_kernel<Op, true>
                                            : (const void *)pbcg::bicgstab_kernel<Op, false>);
    PBCG_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(pbcg::kTPB), params, 0, h->stream));
    return PBCG_OK;
}

// Systems with up to this many stored entries (stencil: points x unknowns)
// are solved by one thread-block cluster by default (pbcg_opts.cluster = 0).
// Measured per iteration (100 fixed iterations, 16-CTA cluster against the
// cooperative grid): 2-D 64^2 (20k entries) 11.3 against 12.4 us (both
// methods faster, BiCGStab 12.4 against 15.2 us), 32^2 8.1 against 11.0 us;
// but 3-D 16^3 (27k entries) in stencil form 13.7 against 13.1 us, and every
// larger system slower on the cluster (its 16 SMs of FP64 throughput: 19.6
// against 12.7 us at 8100 unknowns). The cluster's floor is the FP64 latency
// of the reductions and the scalar updates, not the barrier.
constexpr long long kClusterMaxEntries = 24576;

// Largest cluster (16, else 8) of cluster_solve_kernel<Op> that the device can
// make resident; 0 if none.
template <class Op, bool P>
int cluster_capacity(int want) {
    const void *fn = (const void *)pbcg::cluster_solve_kernel<Op, P>;
    if (want > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)want;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)want);
    cfg.blockDim = dim3(pbcg::kTPB);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return clusters >= 1 ? want : 0;
}

template <class Op>
int cluster_max_for() {
    int c = cluster_capacity<Op, true>(16);
    if (c && !cluster_capacity<Op, false>(16)) c = 0;
    if (!c) c = cluster_capacity<Op, true>(8) && cluster_capacity<Op, false>(8) ? 8 : 0;
    return c;
}

template <class Op>
pbcg_status launch_cluster(pbicgstab_s *h, const Op &op, bool pipelined, const pbcg::SolveArgs &args, int size) {
    if (size > 8) {
        if (pipelined)
            PBCG_CUDA(cudaFuncSetAttribute((const void *)pbcg::cluster_solve_kernel<Op, true>,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        else
            PBCG_CUDA(cudaFuncSetAttribute((const void *)pbcg::cluster_solve_kernel<Op, false>,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)size);
    cfg.blockDim = dim3(pbcg::kTPB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (pipelined)
        PBCG_CUDA(cudaLaunchKernelEx(&cfg, pbcg::cluster_solve_kernel<Op, true>, op, args));
    else
        PBCG_CUDA(cudaLaunchKernelEx(&cfg, pbcg::cluster_solve_kernel<Op, false>, op, args));
    return PBCG_OK;
}

pbcg_status run_solve(pbicgstab_s *h, bool pipelined, const double *d_b, double *d_x, double rtol, int32_t maxit,
                      int32_t replace_period, const pbcg_opts *opts, pbcg_info *info) {
    if (!h) return fail(PBCG_ERR_ARG, "handle is NULL");
    if (info) memset(info, 0, sizeof(*info));
    if (h->n > 0 && (!d_b || !d_x)) return fail(PBCG_ERR_ARG, "b or x is NULL");
    if (!(rtol >= 0.0)) return fail(PBCG_ERR_ARG, "rtol must be >= 0");
    if (maxit < 0) return fail(PBCG_ERR_ARG, "maxit must be >= 0");
    if (replace_period < 0) return fail(PBCG_ERR_ARG, "replace_period must be >= 0");
    pbcg_opts o{-1, 0, nullptr, 0, 0, nullptr, 0, 0};
    if (opts) o = *opts;
    if (o.fixed_iters < 0) return fail(PBCG_ERR_ARG, "fixed_iters must be >= 0");
    if (o.plain_variant != 0 && o.plain_variant != 3 && o.plain_variant != 5)
        return fail(PBCG_ERR_ARG, "plain_variant must be 0, 3 or 5");
    if (o.grid < 0) return fail(PBCG_ERR_ARG, "grid must be >= 0");
    if (o.cluster != 0 && o.cluster != -1 && o.cluster != 2 && o.cluster != 4 && o.cluster != 8 && o.cluster != 16)
        return fail(PBCG_ERR_ARG, "cluster must be 0, -1, 2, 4, 8 or 16 (got %d)", o.cluster);

    pbcg::SolveArgs a;
    a.n = h->n;
    a.b = d_b;
    a.x = d_x;
    a.V = h->V;
    a.ctl = h->ctl;
    a.partials = h->partials;
    a.hist = o.d_history;
    a.rtol = rtol;
    a.fixed = o.fixed_iters > 0 ? 1 : 0;
    a.limit = o.fixed_iters > 0 ? o.fixed_iters : maxit;
    a.replace_period = pipelined ? replace_period : 0;
    a.max_repl = o.max_replacements;
    // Variant 3 saves two grid synchronisations per iteration at the price of
    // 18 more FP64 operations per row. Measured per iteration on 3-D
    // convection-diffusion: variant 3 is faster up to 110k unknowns (33.0 vs
    // 34.1 us), variant 5 from 176k (42.5 vs 43.1 us; 65 vs 74 us at 512k).
    a.variant = o.plain_variant ? o.plain_variant : (h->n < 150000 ? 3 : 5);
    a.minv = h->prec == PBCG_PREC_JACOBI ? h->minv : nullptr;
    a.rh = h->rh;
    a.sh = h->sh;
    a.zh = h->zh;
    a.qh = h->qh;
    a.wh = h->wh;

    const int occ = h->prec == PBCG_PREC_JACOBI ? (pipelined ? h->occ_pipe_prec : h->occ_plain_prec)
                                                : (pipelined ? h->occ_pipe : h->occ_plain);
    // one thread-block cluster for small unpreconditioned systems, else a cooperative grid
    int csize = 0;
    if (h->prec != PBCG_PREC_JACOBI && o.grid == 0 && h->cluster_max > 0) {
        if (o.cluster > 0) {
            if (o.cluster > h->cluster_max)
                return fail(PBCG_ERR_ARG, "clusters of %d CTAs cannot be resident on this device", o.cluster);
            csize = o.cluster;
        } else if (o.cluster == 0 && h->nnz <= kClusterMaxEntries) {
            csize = h->cluster_max;
        }
        while (csize > 2 && (long long)csize * pbcg::kTPB > 2ll * h->n) csize /= 2;   // about 2 rows per thread or more
    } else if (o.cluster > 0 && o.grid == 0) {
        return fail(PBCG_ERR_ARG, "cluster solves need an unpreconditioned handle on a device with clusters");
    }
    const int grid = csize ? csize : pick_grid(h, occ, o.grid);
    PBCG_CUDA(cudaMemsetAsync(h->ctl, 0, sizeof(pbcg::Control), h->stream));
    if (h->ev0) PBCG_CUDA(cudaEventRecord(h->ev0, h->stream));
    if (h->n > 0) {
        pbcg_status st;
        if (csize)
            st = h->kind == 1 ? launch_cluster(h, h->st, pipelined, a, csize)
                 : h->csr_chunked ? launch_cluster(h, chunked(h->csr), pipelined, a, csize)
                                  : launch_cluster(h, h->csr, pipelined, a, csize);
        else
            st = h->kind == 1 ? launch_solver(h, h->st, pipelined, a, grid)
                 : h->csr_chunked ? launch_solver(h, chunked(h->csr), pipelined, a, grid)
                                  : launch_solver(h, h->csr, pipelined, a, grid);
        if (st != PBCG_OK) return st;
    }
    if (h->ev1) PBCG_CUDA(cudaEventRecord(h->ev1, h->stream));
    pbcg::Control c;
    PBCG_CUDA(cudaMemcpyAsync(&c, h->ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    PBCG_CUDA(cudaStreamSynchronize(h->stream));
    pbcg_status st;
    if (h->n == 0) {
        c.status = PBCG_OK;
        c.iters = 0;
    }
    if (c.abort != 0) {
        st = fail((pbcg_status)c.abort, "solver aborted: a grid-wide synchronisation timed out");
        c.status = c.abort;
    } else {
        st = (pbcg_status)c.status;
    }
    if (info) {
        info->iters = c.iters;
        info->status = c.status;
        info->half_step = c.half_step;
        info->n_replacements = c.n_repl;
        info->nr0 = c.nr0;
        info->rel_res_recursive = c.rel_rec;
        info->rel_res_true = c.rel_true;
        info->grid = h->n > 0 ? grid : 0;
        info->block = pbcg::kTPB;
        info->cluster = h->n > 0 ? csize : 0;
        info->grid_syncs = c.grid_syncs;
        info->spmvs = c.spmvs;
        float ms = 0.0f;
        if (h->ev0 && cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) info->kernel_ms = ms;
    }
    return st;
}

// CSR structure check on the device; the flag lives in the control block.
pbcg_status check_csr(pbicgstab_s *h, int32_t n, int32_t nnz, const int32_t *d_rowptr, const int32_t *d_col) {
    int *flag = &h->ctl->abort;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) {
        int blocks = (int)(((long long)(nnz > n ? nnz : n) + 1 + 255) / 256);
        if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
        if (blocks < 1) blocks = 1;
        pbcg::csr_check_kernel<<<blocks, 256, 0, h->stream>>>(n, nnz, d_rowptr, d_col, flag);
        e = cudaGetLastError();
    }
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(PBCG_ERR_CUDA, "CSR check: %s", cudaGetErrorString(e));
    if (bad) return fail(PBCG_ERR_ARG, "invalid CSR structure (check code %d)", bad);
    return PBCG_OK;
}

}  // namespace

extern "C" {

pbcg_status pbicgstab_create_csr(int32_t n, int32_t nnz, const int32_t *d_rowptr, const int32_t *d_col,
                                 const double *d_val, pbcg_prec prec, void *d_workspace, size_t ws_bytes,
                                 void *stream, pbicgstab_t *out) {
    if (!out) return fail(PBCG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || nnz < 0) return fail(PBCG_ERR_ARG, "n and nnz must be >= 0");
    if (!d_rowptr || (nnz > 0 && (!d_col || !d_val))) return fail(PBCG_ERR_ARG, "CSR array is NULL");
    pbicgstab_s *h = new (std::nothrow) pbicgstab_s();
    if (!h) return fail(PBCG_ERR_OOM, "host allocation failed");
    pbcg_status st = common_init(h, n, prec, d_workspace, ws_bytes, stream);
    if (st == PBCG_OK) {
        h->kind = 0;
        h->csr = pbcg::CsrOpScalar{n, d_rowptr, d_col, d_val, nnz};
        h->nnz = nnz;
        h->csr_chunked = (long long)nnz > pbcg::kChunkedMinAvgRow * (long long)n;
        if (h->csr_chunked) {
            st = occupancy<pbcg::CsrOpChunked>(&h->occ_pipe, &h->occ_plain);
            h->cluster_max = cluster_max_for<pbcg::CsrOpChunked>();
            if (st == PBCG_OK) st = occupancy_prec<pbcg::CsrOpChunked>(&h->occ_pipe_prec, &h->occ_plain_prec);
        } else {
            st = occupancy<pbcg::CsrOpScalar>(&h->occ_pipe, &h->occ_plain);
            h->cluster_max = cluster_max_for<pbcg::CsrOpScalar>();
            if (st == PBCG_OK) st = occupancy_prec<pbcg::CsrOpScalar>(&h->occ_pipe_prec, &h->occ_plain_prec);
        }
    }
    if (st == PBCG_OK) st = check_csr(h, n, nnz, d_rowptr, d_col);
    if (st == PBCG_OK && prec == PBCG_PREC_JACOBI && n > 0)
        st = setup_jacobi(h, [&](int blocks, int *flag) {
            pbcg::jacobi_csr_kernel<<<blocks, 256, 0, h->stream>>>(n, d_rowptr, d_col, d_val, h->minv, flag);
        });
    if (st != PBCG_OK) {
        pbicgstab_destroy(h);
        return st;
    }
    *out = h;
    return PBCG_OK;
}

pbcg_status pbicgstab_create_stencil(const pbcg_stencil *desc, pbcg_prec prec, void *d_workspace, size_t ws_bytes,
                                     void *stream, pbicgstab_t *out) {
    if (!out) return fail(PBCG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(PBCG_ERR_ARG, "stencil descriptor is NULL");
    const int nx = desc->nx, ny = desc->ny, nz = desc->nz;
    if (nx < 1 || ny < 1 || nz < 1) return fail(PBCG_ERR_ARG, "grid dimensions must be >= 1");
    const long long nn = (long long)nx * ny * nz;
    if (nn >= (1ll << 31)) return fail(PBCG_ERR_ARG, "grid has more than 2^31-1 nodes");
    for (int d = 0; d < 7; ++d) {
        const pbcg_coef &c = desc->coef[d];
        for (int k = 0; k < 3; ++k)
            if (c.stride[k] < 0 || c.stride2[k] < 0) return fail(PBCG_ERR_ARG, "coefficient %d: negative stride", d);
        if (c.data && max_index(c.stride, nx, ny, nz) >= c.len)
            return fail(PBCG_ERR_ARG, "coefficient %d: table too short (len %lld)", d, (long long)c.len);
        if (c.data2 && max_index(c.stride2, nx, ny, nz) >= c.len2)
            return fail(PBCG_ERR_ARG, "coefficient %d: second table too short (len %lld)", d, (long long)c.len2);
        if ((c.data && max_index(c.stride, nx, ny, nz) >= (1ll << 31) - 1) ||
            (c.data2 && max_index(c.stride2, nx, ny, nz) >= (1ll << 31) - 1))
            return fail(PBCG_ERR_ARG, "coefficient %d: table index exceeds 2^31-2", d);
    }
    pbicgstab_s *h = new (std::nothrow) pbicgstab_s();
    if (!h) return fail(PBCG_ERR_OOM, "host allocation failed");
    pbcg_status st = common_init(h, (int32_t)nn, prec, d_workspace, ws_bytes, stream);
    if (st == PBCG_OK) {
        h->kind = 1;
        h->nnz = (nz == 1 ? 5 : 7) * nn;
        pbcg::StencilOp &o = h->st;
        o.n = (int)nn;
        o.nx = nx;
        o.ny = ny;
        o.nz = nz;
        o.nxy = nx * ny;
        o.dx.init((uint32_t)nx);
        o.dy.init((uint32_t)ny);
        for (int d = 0; d < 7; ++d) {
            const pbcg_coef &c = desc->coef[d];
            pbcg::StCoef q;
            q.t1 = c.data;
            q.t2 = c.data2;
            q.a1 = c.data ? (int)c.stride[0] : 0;
            q.b1 = c.data ? (int)c.stride[1] : 0;
            q.c1 = c.data ? (int)c.stride[2] : 0;
            q.a2 = c.data2 ? (int)c.stride2[0] : 0;
            q.b2 = c.data2 ? (int)c.stride2[1] : 0;
            q.c2 = c.data2 ? (int)c.stride2[2] : 0;
            q.n2 = c.data2 ? 1 : 0;
            q.value = c.value;
            q.len1 = c.data ? (int)(max_index(c.stride, nx, ny, nz) + 1) : 0;
            q.len2 = c.data2 ? (int)(max_index(c.stride2, nx, ny, nz) + 1) : 0;
            o.c[d] = q;
            h->st_len[d][0] = c.data ? max_index(c.stride, nx, ny, nz) + 1 : 0;
            h->st_len[d][1] = c.data2 ? max_index(c.stride2, nx, ny, nz) + 1 : 0;
        }
        st = occupancy<pbcg::StencilOp>(&h->occ_pipe, &h->occ_plain);
        h->cluster_max = cluster_max_for<pbcg::StencilOp>();
        if (st == PBCG_OK) st = occupancy_prec<pbcg::StencilOp>(&h->occ_pipe_prec, &h->occ_plain_prec);
    }
    if (st == PBCG_OK && prec == PBCG_PREC_JACOBI)
        st = setup_jacobi(h, [&](int blocks, int *flag) {
            pbcg::jacobi_stencil_kernel<<<blocks, 256, 0, h->stream>>>(h->st, h->minv, flag);
        });
    if (st != PBCG_OK) {
        pbicgstab_destroy(h);
        return st;
    }
    *out = h;
    return PBCG_OK;
}

pbcg_status pbicgstab_solve(pbicgstab_t h, const double *d_b, double *d_x, double rtol, int32_t maxit,
                            int32_t replace_period, const pbcg_opts *opts, pbcg_info *info) {
    TraceRange tr("pbicgstab_solve");
    return run_solve(h, true, d_b, d_x, rtol, maxit, replace_period, opts, info);
}

pbcg_status bicgstab_solve(pbicgstab_t h, const double *d_b, double *d_x, double rtol, int32_t maxit,
                           const pbcg_opts *opts, pbcg_info *info) {
    TraceRange tr("bicgstab_solve");
    return run_solve(h, false, d_b, d_x, rtol, maxit, 0, opts, info);
}

pbcg_status pbicgstab_solve_host(pbicgstab_t h, int32_t method, const double *h_b, double *h_x, double rtol,
                                 int32_t maxit, int32_t replace_period, const pbcg_opts *opts, pbcg_info *info) {
    if (!h) return fail(PBCG_ERR_ARG, "handle is NULL");
    if (method != 0 && method != 1) return fail(PBCG_ERR_ARG, "method must be 0 (pipelined) or 1 (standard)");
    if (h->n > 0 && (!h_b || !h_x)) return fail(PBCG_ERR_ARG, "b or x is NULL");
    const size_t bytes = (size_t)h->n * sizeof(double);
    if (bytes) {
        PBCG_CUDA(cudaMemcpyAsync(h->b_stage, h_b, bytes, cudaMemcpyHostToDevice, h->stream));
        PBCG_CUDA(cudaMemcpyAsync(h->x_stage, h_x, bytes, cudaMemcpyHostToDevice, h->stream));
    }
    pbcg_status st = run_solve(h, method == 0, h->b_stage, h->x_stage, rtol, maxit, replace_period, opts, info);
    if (st == PBCG_ERR_ARG || st == PBCG_ERR_CUDA || st == PBCG_ERR_OOM) return st;
    if (bytes) {
        PBCG_CUDA(cudaMemcpyAsync(h_x, h->x_stage, bytes, cudaMemcpyDeviceToHost, h->stream));
        PBCG_CUDA(cudaStreamSynchronize(h->stream));
    }
    return st;
}

pbcg_status pbicgstab_spmv(pbicgstab_t h, const double *d_x, double *d_y) {
    if (!h) return fail(PBCG_ERR_ARG, "handle is NULL");
    if (h->n == 0) return PBCG_OK;
    if (!d_x || !d_y) return fail(PBCG_ERR_ARG, "x or y is NULL");
    if ((d_x < d_y + h->n) && (d_y < d_x + h->n)) return fail(PBCG_ERR_ARG, "x and y overlap");
    int blocks = (h->n + pbcg::kTPB - 1) / pbcg::kTPB;
    if (blocks > 16 * h->num_sms) blocks = 16 * h->num_sms;
    if (h->kind == 0 && h->csr_chunked)
        pbcg::spmv_kernel<<<blocks, pbcg::kTPB, 0, h->stream>>>(chunked(h->csr), d_x, d_y);
    else if (h->kind == 0)
        pbcg::spmv_kernel<<<blocks, pbcg::kTPB, 0, h->stream>>>(h->csr, d_x, d_y);
    else
        pbcg::spmv_kernel<<<blocks, pbcg::kTPB, 0, h->stream>>>(h->st, d_x, d_y);
    PBCG_CUDA(cudaGetLastError());
    return PBCG_OK;
}

void pbicgstab_destroy(pbicgstab_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Mixed precision (FP64 refinement around FP32 pipelined BiCGStab).
// ---------------------------------------------------------------------------
namespace {

template <class Op64, class Op32>
pbcg_status launch_mixed(pbicgstab_s *h, const Op64 &a64, const Op32 &a32, const pbcg::MixedArgs &m, int req_grid,
                         int *grid_out) {
    // stencil inner sweeps stage their streamed vectors in dynamic shared memory
    const size_t smem = pbcg::HasRow2<Op32>::value ? pbcg::kStageSmemBytes : 0;
    int occ = 0;
    PBCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pbcg::mixed_kernel<Op64, Op32>, pbcg::kTPB, smem));
    if (occ < 1) return fail(PBCG_ERR_CUDA, "mixed-precision kernel cannot be resident on an SM");
    const int grid = pick_grid(h, occ, req_grid);
    *grid_out = grid;
    PBCG_CUDA(cudaMemsetAsync(h->ctl, 0, sizeof(pbcg::Control), h->stream));
    if (h->ev0) PBCG_CUDA(cudaEventRecord(h->ev0, h->stream));
    void *params[3] = {(void *)&a64, (void *)&a32, (void *)&m};
    PBCG_CUDA(cudaLaunchCooperativeKernel((const void *)pbcg::mixed_kernel<Op64, Op32>, dim3(grid),
                                          dim3(pbcg::kTPB), params, smem, h->stream));
    if (h->ev1) PBCG_CUDA(cudaEventRecord(h->ev1, h->stream));
    return PBCG_OK;
}

}  // namespace

extern "C" pbcg_status pbicgstab_solve_mixed(pbicgstab_t h, const void *d_val_lowp, int32_t lowp_type,
                                             const double *d_b, double *d_x, double rtol, int32_t max_outer,
                                             double inner_rtol, int32_t inner_maxit, const pbcg_opts *opts,
                                             pbcg_mixed_info *info) {
    TraceRange tr("pbicgstab_solve_mixed");
    if (info) memset(info, 0, sizeof(*info));
    if (!h) return fail(PBCG_ERR_ARG, "handle is NULL");
    if (lowp_type != PBCG_VALUES_F32 && lowp_type != PBCG_VALUES_BF16)
        return fail(PBCG_ERR_ARG, "lowp_type must be PBCG_VALUES_F32 or PBCG_VALUES_BF16");
    if (h->kind == 1 && (lowp_type != PBCG_VALUES_F32 || d_val_lowp))
        return fail(PBCG_ERR_ARG, "stencil handles take d_val_lowp = NULL and PBCG_VALUES_F32");
    if (h->n > 0 && (!d_b || !d_x)) return fail(PBCG_ERR_ARG, "b or x is NULL");
    if (h->kind == 0 && h->n > 0 && !d_val_lowp) return fail(PBCG_ERR_ARG, "low-precision values are NULL");
    if (!(rtol >= 0.0) || !(inner_rtol >= 0.0)) return fail(PBCG_ERR_ARG, "tolerances must be >= 0");
    if (max_outer < 0 || inner_maxit < 1) return fail(PBCG_ERR_ARG, "max_outer >= 0 and inner_maxit >= 1 required");
    pbcg_opts o{-1, 0, nullptr, 0, 0, nullptr, 0, 0};
    if (opts) o = *opts;
    if (o.grid < 0) return fail(PBCG_ERR_ARG, "grid must be >= 0");
    if (o.fixed_iters < 0) return fail(PBCG_ERR_ARG, "fixed_iters must be >= 0");
    if (o.stall_steps < 0) return fail(PBCG_ERR_ARG, "stall_steps must be >= 0");
    if (h->n == 0) {
        if (info) info->status = PBCG_OK;
        return PBCG_OK;
    }
    // 12 float vectors carved from the FP64 vector area of the workspace (12 s
    // doubles = 24 s floats), then an FP64 copy of the best iterate (2 s floats)
    float *f0 = (float *)h->V.r;
    const size_t s = vec_stride(h->n);
    pbcg::MixedArgs m;
    m.n = h->n;
    m.b = d_b;
    m.x = d_x;
    float **slots[10] = {&m.V.r, &m.V.r0, &m.V.p, &m.V.s, &m.V.z, &m.V.q, &m.V.y, &m.V.w, &m.V.t, &m.V.v};
    for (int k = 0; k < 10; ++k) *slots[k] = f0 + (size_t)k * s;
    m.d = f0 + 10 * s;
    m.rhs = f0 + 11 * s;
    m.xbest = (double *)(f0 + 12 * s);
    m.ctl = h->ctl;
    m.partials = h->partials;
    m.hist = o.d_history;
    m.inner_hist = o.d_inner_history;
    m.rtol = rtol;
    m.max_outer = max_outer;
    m.inner_rtol = inner_rtol;
    m.inner_maxit = inner_maxit;
    m.inner_fixed = o.fixed_iters;
    m.stall_steps = o.stall_steps > 0 ? o.stall_steps : pbcg::kMixedStallSteps;
    int grid = 0;
    pbcg_status st;
    if (h->kind == 1) {
        // The coefficient tables rounded to FP32, in the part of the FP64
        // vector area the 12 float vectors and the best iterate leave free
        // (10 * s floats).
        pbcg::StencilOpT<float> a32;
        const pbcg::StencilOp &a64 = h->st;
        a32.n = a64.n;
        a32.nx = a64.nx;
        a32.ny = a64.ny;
        a32.nz = a64.nz;
        a32.nxy = a64.nxy;
        a32.dx = a64.dx;
        a32.dy = a64.dy;
        float *tab = f0 + 14 * s;
        const size_t cap = 10 * s;
        size_t used = 0;
        for (int d = 0; d < 7; ++d) {
            const pbcg::StCoef &q = a64.c[d];
            pbcg::StCoefT<float> &q32 = a32.c[d];
            q32.a1 = q.a1;
            q32.b1 = q.b1;
            q32.c1 = q.c1;
            q32.a2 = q.a2;
            q32.b2 = q.b2;
            q32.c2 = q.c2;
            q32.n2 = q.n2;
            q32.value = (float)q.value;
            q32.len1 = q.len1;
            q32.len2 = q.len2;
            const double *src[2] = {q.t1, q.t2};
            const float **dst[2] = {&q32.t1, &q32.t2};
            for (int t = 0; t < 2; ++t) {
                *dst[t] = nullptr;
                if (!src[t]) continue;
                const size_t len = (size_t)h->st_len[d][t];
                const size_t padded = (len + 31) / 32 * 32;
                if (used + padded > cap)
                    return fail(PBCG_ERR_ARG, "stencil coefficient tables too large for the mixed-precision "
                                              "workspace (%zu floats free)", cap);
                float *out = tab + used;
                const int blocks = (int)((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096);
                pbcg::to_float_kernel<<<blocks > 0 ? blocks : 1, 256, 0, h->stream>>>(src[t], out, (long long)len);
                PBCG_CUDA(cudaGetLastError());
                *dst[t] = out;
                used += padded;
            }
        }
        st = launch_mixed(h, a64, a32, m, o.grid, &grid);
    } else if (lowp_type == PBCG_VALUES_F32) {
        const pbcg::CsrOpT<float> a32{h->n, h->csr.rowptr, h->csr.col, (const float *)d_val_lowp, h->csr.nnz};
        st = launch_mixed(h, h->csr, a32, m, o.grid, &grid);
    } else {
        const pbcg::CsrOpT<__nv_bfloat16> a16{h->n, h->csr.rowptr, h->csr.col, (const __nv_bfloat16 *)d_val_lowp,
                                                h->csr.nnz};
        st = launch_mixed(h, h->csr, a16, m, o.grid, &grid);
    }
    if (st != PBCG_OK) return st;
    pbcg::Control c;
    PBCG_CUDA(cudaMemcpyAsync(&c, h->ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    PBCG_CUDA(cudaStreamSynchronize(h->stream));
    if (c.abort != 0) {
        st = fail((pbcg_status)c.abort, "solver aborted: a grid-wide synchronisation timed out");
        c.status = c.abort;
    } else {
        st = (pbcg_status)c.status;
    }
    if (info) {
        info->outer = c.iters;
        info->inner_iters = c.inner_iters;
        info->status = c.status;
        info->grid = grid;
        info->nr0 = c.nr0;
        info->rel_res_true = c.rel_true;
        info->grid_syncs = c.grid_syncs;
        info->spmvs = c.spmvs;
        info->restored = c.half_step;
        float ms = 0.0f;
        if (h->ev0 && cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) info->kernel_ms = ms;
    }
    return st;
}

// ---------------------------------------------------------------------------
// Bounds-checked builds.
// ---------------------------------------------------------------------------
extern "C" int32_t pbicgstab_check_faults(void) {
#ifdef PBCG_CHECK
    int line = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -2;
    if (cudaMemcpyFromSymbol(&line, pbcg::g_check_fault, sizeof(int)) != cudaSuccess) return -2;
    const int zero = 0;
    if (cudaMemcpyToSymbol(pbcg::g_check_fault, &zero, sizeof(int)) != cudaSuccess) return -2;
    return line;
#else
    return -1;
#endif
}

// ---------------------------------------------------------------------------
// Diagnostic of the bounded grid-wide wait.
// ---------------------------------------------------------------------------
extern "C" pbcg_status pbicgstab_probe_sync_timeout(pbicgstab_t h, int32_t limit_ms, int32_t *status) {
    if (!h || !status) return fail(PBCG_ERR_ARG, "handle or status is NULL");
    if (limit_ms < 1 || limit_ms > 4000) return fail(PBCG_ERR_ARG, "limit_ms must be in [1, 4000]");
    *status = PBCG_OK;
    PBCG_CUDA(cudaMemsetAsync(h->ctl, 0, sizeof(pbcg::Control), h->stream));
    pbcg::Control *ctl = h->ctl;
    double *slots = h->partials;
    uint64_t limit_ns = (uint64_t)limit_ms * 1000000ull;
    void *args[] = {&ctl, &slots, &limit_ns};
    PBCG_CUDA(cudaLaunchCooperativeKernel((const void *)pbcg::sync_timeout_probe_kernel, dim3(2), dim3(pbcg::kTPB),
                                          args, 0, h->stream));
    pbcg::Control c;
    PBCG_CUDA(cudaMemcpyAsync(&c, h->ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    PBCG_CUDA(cudaStreamSynchronize(h->stream));
    *status = c.status;
    return PBCG_OK;
}

// ---------------------------------------------------------------------------
// Batched solves.
// ---------------------------------------------------------------------------
extern "C" size_t pbicgstab_batched_workspace_bytes(int64_t total_rows) {
    if (total_rows < 0) return 0;
    const size_t s = ((size_t)(total_rows > 0 ? total_rows : 1) + 31) / 32 * 32;
    return 256 + 10 * s * sizeof(double);
}

extern "C" pbcg_status pbicgstab_solve_batched(const pbcg_batch *batch, int64_t total_rows, const double *d_b,
                                               double *d_x, double rtol, int32_t maxit, int32_t replace_period,
                                               const pbcg_batch_opts *opts, void *d_workspace, size_t ws_bytes,
                                               pbcg_batch_result *d_results, void *stream) {
    TraceRange tr("pbicgstab_solve_batched");
    if (!batch) return fail(PBCG_ERR_ARG, "batch is NULL");
    if (batch->nsys < 0 || batch->nnz < 0 || total_rows < 0) return fail(PBCG_ERR_ARG, "negative size");
    if (batch->nsys == 0) return PBCG_OK;
    if (!batch->d_row_offset || !batch->d_rowptr || !d_results) return fail(PBCG_ERR_ARG, "batch array is NULL");
    if (batch->nnz > 0 && (!batch->d_col || !batch->d_val)) return fail(PBCG_ERR_ARG, "batch array is NULL");
    if (total_rows > 0 && (!d_b || !d_x)) return fail(PBCG_ERR_ARG, "b or x is NULL");
    if (!(rtol >= 0.0) || maxit < 0 || replace_period < 0) return fail(PBCG_ERR_ARG, "invalid tolerance or counts");
    if (!d_workspace || ((uintptr_t)d_workspace) % kAlign) return fail(PBCG_ERR_ARG, "workspace NULL or unaligned");
    if (ws_bytes < pbicgstab_batched_workspace_bytes(total_rows))
        return fail(PBCG_ERR_OOM, "workspace has %zu bytes, needs %zu", ws_bytes,
                    pbicgstab_batched_workspace_bytes(total_rows));
    int csize = opts && opts->cluster_size ? opts->cluster_size : 8;
    const long long cmin = opts && opts->cluster_min_rows ? opts->cluster_min_rows : 512;
    if (csize != 1 && csize != 2 && csize != 4 && csize != 8 && csize != 16)
        return fail(PBCG_ERR_ARG, "cluster_size must be 1, 2, 4, 8 or 16 (got %d)", csize);
    if (cmin < 0) return fail(PBCG_ERR_ARG, "cluster_min_rows must be >= 0");
    const int fixed = opts ? opts->fixed_iters : 0;
    double *hist = opts ? opts->d_history : nullptr;
    const long long hstride = opts ? opts->history_stride : 0;
    if (fixed < 0) return fail(PBCG_ERR_ARG, "fixed_iters must be >= 0");
    if (hist && hstride < (long long)(fixed > 0 ? fixed : maxit) + 1)
        return fail(PBCG_ERR_ARG, "history_stride must be >= (fixed_iters > 0 ? fixed_iters : maxit) + 1");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PBCG_CUDA(cudaGetDevice(&dev));
    PBCG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    pbcg::BatchArgs B;
    B.nsys = batch->nsys;
    B.nnz = batch->nnz;
    B.total_rows = total_rows;
    B.row_offset = (const long long *)batch->d_row_offset;
    B.rowptr = batch->d_rowptr;
    B.col = batch->d_col;
    B.val = batch->d_val;
    B.b = d_b;
    B.x = d_x;
    B.next = (unsigned *)d_workspace;
    double *v0 = (double *)((char *)d_workspace + 256);
    const size_t s = ((size_t)(total_rows > 0 ? total_rows : 1) + 31) / 32 * 32;
    double **slots[10] = {&B.V.r, &B.V.r0, &B.V.p, &B.V.s, &B.V.z, &B.V.q, &B.V.y, &B.V.w, &B.V.t, &B.V.v};
    for (int k = 0; k < 10; ++k) *slots[k] = v0 + (size_t)k * s;
    B.out = d_results;
    B.rtol = rtol;
    B.maxit = maxit;
    B.replace_period = replace_period;
    B.cluster_min_rows = cmin;
    B.fixed = fixed;
    B.hist = hist;
    B.hist_stride = hstride;

    // One resident wave of clusters; clusters take systems until none is left.
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(pbcg::kTPB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    int grid = 0;
    if (csize > 1) {
        if (csize > 8)
            PBCG_CUDA(cudaFuncSetAttribute(pbcg::batched_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3((unsigned)(csize * sms));
        int clusters = 0;
        PBCG_CUDA(cudaOccupancyMaxActiveClusters(&clusters, pbcg::batched_kernel, &cfg));
        if (clusters < 1) return fail(PBCG_ERR_CUDA, "clusters of %d CTAs cannot be resident", csize);
        grid = clusters * csize;
    } else {
        int occ = 0;
        PBCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pbcg::batched_kernel, pbcg::kTPB, 0));
        if (occ < 1) return fail(PBCG_ERR_CUDA, "batched kernel cannot be resident on an SM");
        grid = occ * sms;
        if (grid > batch->nsys) grid = batch->nsys;
        cfg.attrs = nullptr;
        cfg.numAttrs = 0;
    }
    cfg.gridDim = dim3((unsigned)grid);
    PBCG_CUDA(cudaMemsetAsync(B.next, 0, sizeof(unsigned), st));
    PBCG_CUDA(cudaLaunchKernelEx(&cfg, pbcg::batched_kernel, B));
    return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_batched_autotune(const pbcg_batch *batch, int64_t total_rows, const double *d_b,
                                                  double *d_x, double rtol, int32_t maxit, int32_t replace_period,
                                                  void *d_workspace, size_t ws_bytes, pbcg_batch_result *d_results,
                                                  void *stream, pbcg_batch_opts *best, float *best_ms) {
    TraceRange tr("pbicgstab_batched_autotune");
    if (!best) return fail(PBCG_ERR_ARG, "best is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    static const pbcg_batch_opts kCandidates[] = {
        {1, 0, 1}, {2, 0, 512}, {4, 0, 512}, {8, 0, 512}, {16, 0, 512},
        {4, 0, 4096}, {8, 0, 4096}, {16, 0, 4096}, {16, 0, 16384},
    };
    constexpr int kCount = (int)(sizeof(kCandidates) / sizeof(kCandidates[0]));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PBCG_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(PBCG_ERR_CUDA, "cudaEventCreate failed");
    }
    pbcg_status status = PBCG_OK;
    float best_t = 0.0f;
    int best_i = -1;
    // a warm-up solve, then one timed solve per shape, each from x0 = 0
    for (int c = -1; c < kCount && status == PBCG_OK; ++c) {
        const pbcg_batch_opts &o = kCandidates[c < 0 ? 3 : c];
        if (total_rows > 0 && cudaMemsetAsync(d_x, 0, (size_t)total_rows * sizeof(double), st) != cudaSuccess) {
            status = fail(PBCG_ERR_CUDA, "cudaMemsetAsync failed");
            break;
        }
        if (cudaEventRecord(e0, st) != cudaSuccess) { status = fail(PBCG_ERR_CUDA, "event record failed"); break; }
        const pbcg_status r = pbicgstab_solve_batched(batch, total_rows, d_b, d_x, rtol, maxit, replace_period, &o,
                                                      d_workspace, ws_bytes, d_results, stream);
        if (r == PBCG_ERR_CUDA && c >= 0) continue;   // a cluster shape the GPU cannot make resident
        if (r != PBCG_OK) { status = r; break; }
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            status = fail(PBCG_ERR_CUDA, "event synchronisation failed");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (c >= 0 && (best_i < 0 || ms < best_t)) {
            best_t = ms;
            best_i = c;
        }
    }
    // the best shape runs last, so d_x and d_results hold its solves
    if (status == PBCG_OK && best_i >= 0) {
        if (total_rows > 0 && cudaMemsetAsync(d_x, 0, (size_t)total_rows * sizeof(double), st) != cudaSuccess)
            status = fail(PBCG_ERR_CUDA, "cudaMemsetAsync failed");
        if (status == PBCG_OK)
            status = pbicgstab_solve_batched(batch, total_rows, d_b, d_x, rtol, maxit, replace_period,
                                             &kCandidates[best_i], d_workspace, ws_bytes, d_results, stream);
        if (status == PBCG_OK && cudaStreamSynchronize(st) != cudaSuccess)
            status = fail(PBCG_ERR_CUDA, "cudaStreamSynchronize failed");
    } else if (status == PBCG_OK) {
        status = fail(PBCG_ERR_CUDA, "no cluster shape could be launched");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != PBCG_OK) return status;
    *best = kCandidates[best_i];
    if (best_ms) *best_ms = best_t;
    return PBCG_OK;
}

// ---------------------------------------------------------------------------
// Adjoint building blocks: transpose and value gradient.
// ---------------------------------------------------------------------------
extern "C" size_t pbicgstab_transpose_work_bytes(int32_t n) {
    if (n < 0) return 0;
    const size_t b = (size_t)(n + 1) * sizeof(int);
    return b < 256 ? 256 : b;   // also holds the structure-check flag
}

extern "C" pbcg_status pbicgstab_csr_transpose(int32_t n, int32_t nnz, const int32_t *d_rowptr,
                                               const int32_t *d_col, const double *d_val, int32_t *d_trowptr,
                                               int32_t *d_tcol, double *d_tval, void *d_work, size_t work_bytes,
                                               void *stream) {
    if (n < 0 || nnz < 0) return fail(PBCG_ERR_ARG, "n and nnz must be >= 0");
    if (!d_rowptr || !d_trowptr || (nnz > 0 && (!d_col || !d_val || !d_tcol || !d_tval)))
        return fail(PBCG_ERR_ARG, "CSR array is NULL");
    if (!d_work || work_bytes < pbicgstab_transpose_work_bytes(n)) return fail(PBCG_ERR_OOM, "work buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PBCG_CUDA(cudaGetDevice(&dev));
    PBCG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // validate the input structure first (columns index rows of A^T)
    pbicgstab_s h{};
    h.num_sms = sms;
    h.stream = st;
    h.ctl = (pbcg::Control *)d_work;   // the check flag lives in the work buffer's first word
    pbcg_status s0 = check_csr(&h, n, nnz, d_rowptr, d_col);
    if (s0 != PBCG_OK) return s0;
    int *cursor = (int *)d_work;
    const int blocks = 4 * sms;
    PBCG_CUDA(cudaMemsetAsync(d_trowptr, 0, (size_t)(n + 1) * sizeof(int), st));
    if (nnz > 0) pbcg::transpose_count_kernel<<<blocks, 256, 0, st>>>(nnz, d_col, d_trowptr);
    pbcg::scan_kernel<<<1, 1024, 0, st>>>(n + 1, d_trowptr);
    PBCG_CUDA(cudaMemsetAsync(cursor, 0, (size_t)(n + 1) * sizeof(int), st));
    if (n > 0) {
        pbcg::transpose_scatter_kernel<<<blocks, 256, 0, st>>>(n, d_rowptr, d_col, d_val, d_trowptr, cursor, d_tcol,
                                                               d_tval);
        pbcg::sort_rows_kernel<<<blocks, 256, 0, st>>>(n, d_trowptr, d_tcol, d_tval);
    }
    PBCG_CUDA(cudaGetLastError());
    return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_csr_value_grad(int32_t n, const int32_t *d_rowptr, const int32_t *d_col,
                                                const double *d_lambda, const double *d_x, double *d_grad,
                                                void *stream) {
    if (n < 0) return fail(PBCG_ERR_ARG, "n must be >= 0");
    if (n == 0) return PBCG_OK;
    if (!d_rowptr || !d_col || !d_lambda || !d_x || !d_grad) return fail(PBCG_ERR_ARG, "array is NULL");
    int dev = 0, sms = 0;
    PBCG_CUDA(cudaGetDevice(&dev));
    PBCG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    pbcg::value_grad_kernel<<<4 * sms, 256, 0, (cudaStream_t)stream>>>(n, d_rowptr, d_col, d_lambda, d_x, d_grad);
    PBCG_CUDA(cudaGetLastError());
    return PBCG_OK;
}

// ---------------------------------------------------------------------------
// Solve without any device allocation, for callers that may not allocate.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running inside a host application that owns all device memory and forbids
// allocation after start-up (allocation synchronises the device and can fail
// under memory pressure at a point the application cannot handle), real-time
// loops that must not block on the allocator, and plug-ins that only receive
// input and output pointers. For them the workspace of one solve lives in a
// fixed array in this library's device memory, sized for at most
// PBCG_NOALLOC_MAX_N unknowns; every GPU that loads the library keeps that
// array (about 3.4 MB) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = pbcg::kControlBytes + pbcg::kPartialBytes +
                                 (size_t)kVectors * (((size_t)PBCG_NOALLOC_MAX_N + 31) / 32 * 32) * sizeof(double);

// The shared scratch. Host code must not use this name as an address: it is a
// host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch on the current device; looked up once per
// device, with that device current.
pbcg_status noalloc_scratch(void **out) {
    int dev = 0;
    PBCG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(PBCG_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(PBCG_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PBCG_OK;
}

}  // namespace

extern "C" pbcg_status pbicgstab_solve_csr_noalloc(int32_t n, int32_t nnz, const int32_t *d_rowptr,
                                                   const int32_t *d_col, const double *d_val, const double *d_b,
                                                   double *d_x, double rtol, int32_t maxit, int32_t replace_period,
                                                   const pbcg_opts *opts, void *stream, pbcg_info *info) {
    if (info) memset(info, 0, sizeof(*info));
    if (n < 0 || nnz < 0) return fail(PBCG_ERR_ARG, "n and nnz must be >= 0");
    if (n > PBCG_NOALLOC_MAX_N)
        return fail(PBCG_ERR_ARG, "n = %d exceeds the no-allocation limit of %d unknowns", n, PBCG_NOALLOC_MAX_N);
    if (!d_rowptr || (nnz > 0 && (!d_col || !d_val))) return fail(PBCG_ERR_ARG, "CSR array is NULL");
    void *ws = nullptr;
    pbcg_status st = noalloc_scratch(&ws);
    if (st != PBCG_OK) return st;
    pbicgstab_s h{};   // on the stack; no events (creating them is not needed here)
    st = common_init(&h, n, PBCG_PREC_NONE, ws, kNoAllocBytes, stream, false);
    if (st == PBCG_OK) {
        h.kind = 0;
        h.csr = pbcg::CsrOpScalar{n, d_rowptr, d_col, d_val, nnz};
        h.nnz = nnz;
        h.csr_chunked = (long long)nnz > pbcg::kChunkedMinAvgRow * (long long)n;
        st = h.csr_chunked ? occupancy<pbcg::CsrOpChunked>(&h.occ_pipe, &h.occ_plain)
                           : occupancy<pbcg::CsrOpScalar>(&h.occ_pipe, &h.occ_plain);
        h.cluster_max = h.csr_chunked ? cluster_max_for<pbcg::CsrOpChunked>() : cluster_max_for<pbcg::CsrOpScalar>();
    }
    if (st == PBCG_OK) st = check_csr(&h, n, nnz, d_rowptr, d_col);
    if (st != PBCG_OK) return st;
    // run_solve clears the control block before the launch
    return run_solve(&h, true, d_b, d_x, rtol, maxit, replace_period, opts, info);
}
