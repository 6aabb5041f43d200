// Building blocks of the adjoint (reverse-mode) solve: the transpose of a CSR
// matrix and the gradient with respect to its stored values.
//
// For x = A^{-1} b and a loss L(x), the adjoint lambda = A^{-T} dL/dx gives
// dL/db = lambda and dL/da_ij = -lambda_i x_j for every stored entry (i, j).
// The transpose is built deterministically: entries are scattered with atomic
// cursors and each row of A^T is then sorted by column, so the row order (and
// hence every SpMV with A^T) does not depend on scheduling.
#pragma once

#include "device_common.cuh"

namespace pbcg {

// counts[c + 1] += 1 for every stored column c (counts zeroed by the caller)
__global__ void transpose_count_kernel(int nnz, const int *col, int *counts) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
        atomicAdd(&counts[col[k] + 1], 1);
}

// In-place inclusive prefix sum of a[0..m), one block: each thread sums a
// contiguous chunk, the chunk totals are scanned in shared memory, then each
// chunk is rewritten with its offset. Turns counts into row pointers.
__global__ void scan_kernel(int m, int *a) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const long long chunk = ((long long)m + T - 1) / T;
    const long long b = t * chunk, e = b + chunk < m ? b + chunk : m;
    long long s = 0;
    for (long long i = b; i < e; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long run = 0;
        for (int i = 0; i < T; ++i) {
            const long long v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = part[t];
    for (long long i = b; i < e; ++i) {
        run += a[i];
        a[i] = (int)run;
    }
}

// Scatter entry (i, c, v) of A to row c of A^T at the next free slot.
__global__ void transpose_scatter_kernel(int n, const int *rowptr, const int *col, const double *val,
                                         const int *trow, int *cursor, int *tcol, double *tval) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int c = PBCG_SAFE(col[k], n);
            const int pos = trow[c] + atomicAdd(&cursor[c], 1);
            tcol[pos] = i;
            tval[pos] = val[k];
        }
    }
}

// Sort every row of A^T by column (insertion sort; rows are short).
__global__ void sort_rows_kernel(int n, const int *rowptr, int *col, double *val) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = rowptr[i], e = rowptr[i + 1];
        for (int k = b + 1; k < e; ++k) {
            const int c = col[k];
            const double v = val[k];
            int j = k - 1;
            while (j >= b && col[j] > c) {
                col[j + 1] = col[j];
                val[j + 1] = val[j];
                --j;
            }
            col[j + 1] = c;
            val[j + 1] = v;
        }
    }
}

// g[k] = -lambda[i] * x[col[k]] for every stored entry k of row i.
__global__ void value_grad_kernel(int n, const int *rowptr, const int *col, const double *lambda, const double *x,
                                  double *g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double li = lambda[i];
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) g[k] = -li * x[PBCG_SAFE(col[k], n)];
    }
}

}  // namespace pbcg
