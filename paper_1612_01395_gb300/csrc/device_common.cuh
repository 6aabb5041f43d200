// Device-side building blocks shared by the solver kernels: constants, the
// workspace control block, fast integer division, fixed-order reductions and
// the bounded grid-wide synchronisation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pbicgstab.h"

namespace pbcg {

constexpr int kTPB = 128;          // threads per block of every kernel here
constexpr int kMaxGrid = 2048;     // upper bound on thread blocks (sizes the partial-sum slots)
constexpr int kMaxDots = 8;        // dot products carried by one reduction
constexpr uint64_t kSyncTimeoutNs = 4000000000ull;   // 4 s per grid-wide wait

// Control block at the start of the workspace; zeroed before every solve.
struct Control {
    unsigned int arrivals;   // grid-sync arrivals, monotonic within one launch
    int abort;               // nonzero: pbcg_status that stopped the launch
    int pad0[14];
    // result, written by block 0 at the end of a solve
    int iters, status, half_step, n_repl, grid_syncs, spmvs, pad1[2];
    double nr0, rel_rec, rel_true, pad2;
};
static_assert(sizeof(Control) <= 256, "control block must fit 256 bytes");
constexpr size_t kControlBytes = 256;
constexpr size_t kPartialBytes = 2ull * kMaxGrid * kMaxDots * sizeof(double);

// n / d for 0 <= n < 2^31 and 1 <= d < 2^31 by one multiply-high: the
// round-up method of Granlund & Montgomery, "Division by invariant integers
// using multiplication" (PLDI 1994): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(m, n) + n) >> l.
struct FastDiv {
    uint32_t d, m, l;
    __host__ void init(uint32_t dd) {
        d = dd;
        l = 0;
        while ((1ull << l) < dd) ++l;
        m = (uint32_t)(((((1ull << l) - dd)) << 32) / dd + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(m, n) + n) >> l; }
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Butterfly sum over a warp. Every lane ends with the same bits: at each level
// a lane adds its partner's value to its own, and addition is commutative.
template <int K>
__device__ __forceinline__ void warp_sum(double (&v)[K]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
}

// Fixed-order block sum; every thread receives the result. sm: [kMaxDots][32].
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (*sm)[32]) {
    constexpr int kWarps = kTPB / 32;
    warp_sum<K>(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sm[k][wid] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = lane < kWarps ? sm[k][lane] : 0.0;
    warp_sum<K>(v);   // each warp reduces the same kWarps values
    __syncthreads();
}

// Grid-wide synchronisation of a cooperative launch, optionally carrying a
// fixed-order sum of K doubles. Arrivals are counted on one word; every wait is
// bounded by kSyncTimeoutNs and by the abort flag, so a launch can only end.
struct GridSync {
    Control *ctl;
    double *partials;   // [2][kMaxGrid][kMaxDots]
    unsigned epoch;     // synchronisations passed by this block
    int count;          // synchronisations performed (for diagnostics)
};

__device__ __forceinline__ bool grid_wait(GridSync &g, int *sflag) {
    __syncthreads();   // every thread's stores of this phase precede the fence below
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&g.ctl->arrivals, 1u);
        const unsigned target = (g.epoch + 1u) * gridDim.x;
        const uint64_t t0 = globaltimer_ns();
        int ok = 1;
        while (ld_acquire_u32(&g.ctl->arrivals) < target) {
            if (ld_relaxed_s32(&g.ctl->abort) != 0) { ok = 0; break; }
            if (globaltimer_ns() - t0 > kSyncTimeoutNs) {
                atomicCAS(&g.ctl->abort, 0, (int)PBCG_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        *sflag = ok;
    }
    __syncthreads();
    const bool ok = *sflag != 0;
    g.epoch++;
    g.count++;
    return ok;
}

// Barrier without data.
__device__ __forceinline__ bool grid_sync(GridSync &g, int *sflag) { return grid_wait(g, sflag); }

// Barrier that also returns, in every thread of every block, the same
// fixed-order sum over the grid of the K per-thread values v.
template <int K>
__device__ __forceinline__ bool grid_sum(GridSync &g, double (&v)[K], double (*sm)[32], int *sflag) {
    block_sum<K>(v, sm);
    const unsigned slot = g.epoch & 1u;
    double *base = g.partials + (size_t)slot * kMaxGrid * kMaxDots;
    if (threadIdx.x == 0) {
        double *mine = base + (size_t)blockIdx.x * kMaxDots;
#pragma unroll
        for (int k = 0; k < K; ++k) mine[k] = v[k];
    }
    if (!grid_wait(g, sflag)) return false;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kTPB) {
        const double *src = base + (size_t)b * kMaxDots;
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += __ldcg(src + k);
    }
    block_sum<K>(acc, sm);
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = acc[k];
    return true;
}

}  // namespace pbcg
