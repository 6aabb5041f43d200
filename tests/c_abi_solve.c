/* The library used from C alone, through include/pbicgstab.h: a 2-D
 * convection-diffusion system (5-point upwind, velocity (10, 10), m x m grid,
 * Dirichlet boundary, scaled by h^2) in CSR form is copied to the device,
 * solved with pipelined BiCGStab and with standard BiCGStab, and the true
 * residual ||b - A x|| / ||b|| of each result is recomputed on the host.
 * Prints one JSON line; exits non-zero on any failure. Test code: the tests
 * compile and run it on a GPU. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "pbicgstab.h"

#define CHECK(call)                                                              \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));  \
            return 2;                                                            \
        }                                                                        \
    } while (0)

static double true_rel(int n, const int *rp, const int *ci, const double *v, const double *b, const double *x) {
    double rr = 0.0, bb = 0.0;
    for (int i = 0; i < n; ++i) {
        double ax = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) ax += v[k] * x[ci[k]];
        const double r = b[i] - ax;
        rr += r * r;
        bb += b[i] * b[i];
    }
    return sqrt(rr) / sqrt(bb);
}

int main(int argc, char **argv) {
    const int m = argc > 1 ? atoi(argv[1]) : 64;
    const int n = m * m;
    const double h = 1.0 / (m + 1), cx = 10.0, cy = 10.0;
    int *rp = malloc((n + 1) * sizeof(int)), *ci = malloc(5 * n * sizeof(int));
    double *v = malloc(5 * n * sizeof(double)), *b = malloc(n * sizeof(double)), *x = malloc(n * sizeof(double));
    if (!rp || !ci || !v || !b || !x) return 2;
    int nnz = 0;
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            const int r = j * m + i;
            rp[r] = nnz;
            /* columns in ascending order: south, west, centre, east, north */
            if (j > 0) { ci[nnz] = r - m; v[nnz++] = -1.0 - h * cy; }
            if (i > 0) { ci[nnz] = r - 1; v[nnz++] = -1.0 - h * cx; }
            ci[nnz] = r; v[nnz++] = 4.0 + h * (cx + cy);
            if (i < m - 1) { ci[nnz] = r + 1; v[nnz++] = -1.0; }
            if (j < m - 1) { ci[nnz] = r + m; v[nnz++] = -1.0; }
        }
    rp[n] = nnz;
    unsigned long long z = 12345u;   /* b from a simple LCG; any right-hand side will do */
    for (int i = 0; i < n; ++i) {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        b[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    }

    int *d_rp, *d_ci;
    double *d_v, *d_b, *d_x;
    void *d_ws;
    const size_t ws = pbicgstab_workspace_bytes(n);
    CHECK(cudaMalloc((void **)&d_rp, (n + 1) * sizeof(int)));
    CHECK(cudaMalloc((void **)&d_ci, nnz * sizeof(int)));
    CHECK(cudaMalloc((void **)&d_v, nnz * sizeof(double)));
    CHECK(cudaMalloc((void **)&d_b, n * sizeof(double)));
    CHECK(cudaMalloc((void **)&d_x, n * sizeof(double)));
    CHECK(cudaMalloc(&d_ws, ws));
    CHECK(cudaMemcpy(d_rp, rp, (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(d_ci, ci, nnz * sizeof(int), cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(d_v, v, nnz * sizeof(double), cudaMemcpyHostToDevice));
    CHECK(cudaMemcpy(d_b, b, n * sizeof(double), cudaMemcpyHostToDevice));

    pbicgstab_t hdl = NULL;
    pbcg_status st = pbicgstab_create_csr(n, nnz, d_rp, d_ci, d_v, PBCG_PREC_NONE, d_ws, ws, NULL, &hdl);
    if (st != PBCG_OK) {
        fprintf(stderr, "create: %s\n", pbicgstab_last_error());
        return 3;
    }
    double rel[2];
    int iters[2], status[2];
    for (int method = 0; method < 2; ++method) {
        pbcg_info info;
        CHECK(cudaMemset(d_x, 0, n * sizeof(double)));
        st = method == 0 ? pbicgstab_solve(hdl, d_b, d_x, 1e-10, 5000, 20, NULL, &info)
                         : bicgstab_solve(hdl, d_b, d_x, 1e-10, 5000, NULL, &info);
        CHECK(cudaMemcpy(x, d_x, n * sizeof(double), cudaMemcpyDeviceToHost));
        rel[method] = true_rel(n, rp, ci, v, b, x);
        iters[method] = info.iters;
        status[method] = (int)st;
    }
    pbicgstab_destroy(hdl);
    cudaFree(d_rp);
    cudaFree(d_ci);
    cudaFree(d_v);
    cudaFree(d_b);
    cudaFree(d_x);
    cudaFree(d_ws);
    printf("{\"n\": %d, \"nnz\": %d, \"pbicgstab\": {\"status\": %d, \"iters\": %d, \"true_rel\": %.3e}, "
           "\"bicgstab\": {\"status\": %d, \"iters\": %d, \"true_rel\": %.3e}}\n",
           n, nnz, status[0], iters[0], rel[0], status[1], iters[1], rel[1]);
    free(rp);
    free(ci);
    free(v);
    free(b);
    free(x);
    return (status[0] == PBCG_OK && status[1] == PBCG_OK && rel[0] < 1e-9 && rel[1] < 1e-9) ? 0 : 1;
}
