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

// Bounds-checked build (-DPBCG_CHECK): PBCG_SAFE(i, n) yields i when 0 <= i < n,
// else records the source line in g_check_fault (the first such access only)
// and yields 0, so the access stays in bounds and the solve carries on; the
// host reads the record with pbicgstab_check_faults. It guards the indices
// that the operators form from data or geometry (gathered columns, stencil
// neighbours, row pointers). The default build compiles it to plain i.
#ifdef PBCG_CHECK
__device__ int g_check_fault;
__device__ __forceinline__ long long checked_index(long long i, long long n, int line) {
    if (i >= 0 && i < n) return i;
    atomicCAS(&g_check_fault, 0, line);
    return 0;
}
#define PBCG_SAFE(i, n) ((int)::pbcg::checked_index((long long)(i), (long long)(n), __LINE__))
#else
#define PBCG_SAFE(i, n) (i)
#endif

// Control block at the start of the workspace; zeroed before every solve.
struct Control {
    unsigned int arrivals;   // grid-sync arrivals, monotonic within one launch
    int abort;               // nonzero: pbcg_status that stopped the launch
    unsigned int ready;      // large grids: 1 + the last exchange whose totals are published
    int pad0[13];
    // result, written by block 0 at the end of a solve
    int iters, status, half_step, n_repl, grid_syncs, spmvs, inner_iters, pad1;
    double nr0, rel_rec, rel_true, pad2;
};
static_assert(sizeof(Control) <= 256, "control block must fit 256 bytes");
constexpr size_t kControlBytes = 256;
// 3 rotating buffers of one 8-double slot per block, then 3 rotating 8-double
// totals; rounded up to 256 bytes so the vectors after it stay 256-byte aligned
constexpr size_t kPartialBytes = ((3ull * kMaxGrid + 3) * 8 * sizeof(double) + 255) / 256 * 256;

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

constexpr unsigned kFull = 0xffffffffu;

// Sum of each of K values over the 32 lanes of a warp, returned to every lane.
// FP64 adds are the scarce resource on this GPU (one warp-wide DADD occupies a
// sub-partition's FP64 pipe for ~64 cycles), so the first log2(P) levels use
// recursive halving (P = K rounded up to a power of two): at each level a lane
// keeps half of its values and adds its partner's copy of them, costing P/2
// additions instead of P; the remaining levels are a butterfly on one value.
// K = 5 takes 9 additions instead of 25. After the halving, value index k
// lives in the lanes whose bits 4, 3, 2 (most significant first) spell k.
// Deterministic: in the butterfly both partners add the same two numbers (in
// either order, hence to the same bits), so all lanes holding index k agree.
template <int K>
__device__ __forceinline__ void warp_allsum(double (&v)[K]) {
    constexpr int P = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : 8;
    constexpr int M = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : 3;
    static_assert(K <= 8, "at most 8 values");
    const int lane = threadIdx.x & 31;
    double w[P];
#pragma unroll
    for (int k = 0; k < P; ++k) w[k] = k < K ? v[k] : 0.0;
#pragma unroll
    for (int lvl = 0; lvl < M; ++lvl) {
        const int o = 16 >> lvl;
        const int half = P >> (lvl + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double send = upper ? w[k] : w[k + half];
            const double keep = upper ? w[k + half] : w[k];
            w[k] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> M; o > 0; o >>= 1) w[0] += __shfl_xor_sync(kFull, w[0], o);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int src = 0;
#pragma unroll
        for (int b = 0; b < M; ++b)
            if (k & (1 << (M - 1 - b))) src |= 16 >> b;
        v[k] = __shfl_sync(kFull, w[0], src);
    }
}

// Fixed-order block sum; every thread receives the K results. sm: [kMaxDots][32].
// Warps reduce independently, then lane k of every warp adds value k of the
// warps in warp order and shuffles it to the other lanes.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (*sm)[32]) {
    constexpr int kWarps = kTPB / 32;
    warp_allsum<K>(v);
    if (kWarps == 1) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sm[k][wid] = v[k];
    }
    __syncthreads();
    double t = 0.0;
    if (lane < K) {
        t = sm[lane][0];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) t += sm[lane][w];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = __shfl_sync(kFull, t, k);
    __syncthreads();
}

// Grid-wide exchange of a cooperative launch. Each block owns one 64-byte
// slot (8 doubles) in each of 3 rotating buffers; exchange number e uses
// buffer e % 3. Thread 0 of a block stores its K block sums in its slot,
// fences (gpu scope: every store of the phase, made visible to thread 0 by
// __syncthreads, is ordered before the arrival) and adds 1 to the arrival
// counter. Then, by grid size:
//  * small grids: thread 0 spins on the counter until all blocks of exchange
//    e arrived, and every block adds all slots in the same fixed order;
//  * large grids (at least kLastReduceGrid blocks): the block whose arrival
//    completes the count adds all slots (same fixed order), publishes the K
//    totals and raises `ready`; the others spin on `ready` and read the
//    totals. Every block adding every slot costs each SM (blocks per SM x
//    blocks x K) FP64 additions per exchange -- about 12 us of its FP64 pipe
//    at 1216 blocks -- against one extra flag hop.
// One poller per block on one word: polling all slots from every thread
// congests the L2 and was measured slower. The rotation keeps a slot or a
// total from being rewritten while a slow block may still read it (exchange
// e+3 is written only after all blocks arrived at e+2, i.e. after all finished
// reading exchange e). Results are bitwise identical in every block and do
// not depend on arrival order. Every wait is bounded (limit_ns,
// kSyncTimeoutNs by default) and watches the abort flag.
constexpr int kSlotDoubles = 8;
constexpr int kLastReduceGrid = 512;

struct GridSync {
    Control *ctl;
    double *slots;      // [3][gridDim.x][kSlotDoubles], then [3][kSlotDoubles] totals
    unsigned epoch;     // exchanges done by this block
    int count;          // exchanges performed (for diagnostics)
    uint64_t limit_ns = kSyncTimeoutNs;   // bound on each wait
};

__device__ __forceinline__ double *slot_ptr(const GridSync &g, unsigned buf, int block) {
    return g.slots + ((size_t)buf * gridDim.x + block) * kSlotDoubles;
}
__device__ __forceinline__ double *totals_ptr(const GridSync &g, unsigned buf) {
    return g.slots + ((size_t)3 * gridDim.x + buf) * kSlotDoubles;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The block that records per-solve results (the residual history) under each
// synchronisation policy: block 0 of a grid; the block itself when a block
// solves alone; CTA rank 0 of a cluster (is_leader overloads below).
__device__ __forceinline__ bool is_leader(const GridSync &) { return blockIdx.x == 0; }

// Thread 0: spin until *word >= target, bounded; false on abort or timeout.
__device__ __forceinline__ bool wait_at_least(GridSync &g, const unsigned *word, unsigned target) {
    const uint64_t t0 = globaltimer_ns();
    while (ld_acquire_u32(word) < target) {
        if (ld_relaxed_s32(&g.ctl->abort) != 0) return false;
        if (globaltimer_ns() - t0 > g.limit_ns) {
            atomicCAS(&g.ctl->abort, 0, (int)PBCG_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// *sflag (shared, set to 1 once at kernel start) only ever goes from 1 to 0:
// thread 0 clears it when a wait is abandoned, and every thread returns its
// value after the barrier that follows. Never resetting it keeps a slow thread
// from reading a later exchange's value.

// Barrier without data.
__device__ __forceinline__ bool grid_sync(GridSync &g, double (*)[32], int *sflag) {
    __syncthreads();   // every thread's stores of this phase precede thread 0's fence
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&g.ctl->arrivals, 1u);
        if (!wait_at_least(g, &g.ctl->arrivals, (g.epoch + 1u) * gridDim.x)) *sflag = 0;
        __threadfence();
    }
    __syncthreads();
    g.epoch++;
    g.count++;
    return *sflag != 0;
}

// Fixed-order sum over all slots of buffer buf, returned in every thread.
template <int K>
__device__ __forceinline__ void sum_slots(const GridSync &g, unsigned buf, double (&v)[K], double (*sm)[32]) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kTPB) {
        const double *src = slot_ptr(g, buf, b);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __ldcg(src + k);
    }
    block_sum<K>(v, sm);
}

// Barrier that also returns, in every thread of every block, the same
// fixed-order sum over the grid of the K per-thread values v.
template <int K>
__device__ __forceinline__ bool grid_sum(GridSync &g, double (&v)[K], double (*sm)[32], int *sflag) {
    static_assert(K <= kSlotDoubles, "at most 8 values per exchange");
    __shared__ int last;
    block_sum<K>(v, sm);   // ends with __syncthreads
    const unsigned buf = g.epoch % 3u;
    const unsigned target = (g.epoch + 1u) * gridDim.x;
    const bool by_last = gridDim.x >= (unsigned)kLastReduceGrid;
    if (threadIdx.x == 0) {
        double *out = slot_ptr(g, buf, blockIdx.x);
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = v[k];
        __threadfence();
        const unsigned before = atomicAdd(&g.ctl->arrivals, 1u);
        last = before == target - 1u;
        if (!by_last) {
            if (!wait_at_least(g, &g.ctl->arrivals, target)) *sflag = 0;
        }
        __threadfence();
    }
    __syncthreads();
    if (!by_last) {
        sum_slots<K>(g, buf, v, sm);
    } else if (last) {
        sum_slots<K>(g, buf, v, sm);   // every slot is visible: all blocks fenced before arriving
        if (threadIdx.x == 0) {
            double *tot = totals_ptr(g, buf);
#pragma unroll
            for (int k = 0; k < K; ++k) tot[k] = v[k];
            __threadfence();
            st_release_u32(&g.ctl->ready, g.epoch + 1u);
        }
    } else {
        if (threadIdx.x == 0) {
            if (!wait_at_least(g, &g.ctl->ready, g.epoch + 1u)) *sflag = 0;
            __threadfence();
        }
        __syncthreads();
        const double *tot = totals_ptr(g, buf);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = __ldcg(tot + k);
    }
    g.epoch++;
    g.count++;
    __syncthreads();   // `last` is rewritten by the next exchange
    return *sflag != 0;
}

// Synchronisation policy of a solve owned by one thread block (batched
// solves): the "grid" is the block, a barrier is __syncthreads and a reduction
// is the block sum. Same interface as GridSync, so the solver loops are shared.
struct BlockSync {
    int count;
};

__device__ __forceinline__ bool is_leader(const BlockSync &) { return true; }

__device__ __forceinline__ bool grid_sync(BlockSync &g, double (*)[32], int *) {
    __syncthreads();
    g.count++;
    return true;
}

template <int K>
__device__ __forceinline__ bool grid_sum(BlockSync &g, double (&v)[K], double (*sm)[32], int *) {
    block_sum<K>(v, sm);   // its __syncthreads also orders the block's stores of the phase
    g.count++;
    return true;
}

// ---------------------------------------------------------------------------
// 1-D bulk copies from global into shared memory (the TMA unit's untiled
// copy, cp.async.bulk), completed on a shared-memory mbarrier. One thread
// posts the expected byte count and issues the copies; every thread waits on
// the barrier's phase. Addresses and sizes must be multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make barrier initialisations visible to the asynchronous (copy) proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Order this thread's earlier generic-proxy global accesses before later
// bulk copies (async proxy) of the same memory.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Wait until the barrier's phase of the given parity has completed. Bounded:
// after kSyncTimeoutNs the launch is flagged PBCG_ERR_TIMEOUT and false is
// returned (a copy can only stay incomplete if its byte count disagreed with
// the posted one).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, Control *ctl) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > kSyncTimeoutNs) {
            atomicCAS(&ctl->abort, 0, (int)PBCG_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Thread-block clusters (batched solves of large systems). The CTAs of a
// cluster are co-scheduled by the hardware, so a wait on the hardware cluster
// barrier always completes once every CTA reaches it; each CTA can address
// the shared memory of the others (distributed shared memory).
// ---------------------------------------------------------------------------
constexpr int kMaxCluster = 16;

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_ctas() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives and waits. Release on
// arrival and acquire on the wait (cluster scope) order each CTA's earlier
// stores -- global and shared -- before the other CTAs' later loads.
// (The non-.aligned forms: no requirement that a warp arrives converged.)
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Address of *p (a __shared__ object of this CTA) in the shared memory of CTA `rank`.
__device__ __forceinline__ uint32_t cluster_map(const void *p, unsigned rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(rank));
    return out;
}
__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ double ld_cluster_f64(uint32_t addr) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster_s32(uint32_t addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Synchronisation policy of a solve shared by the `size` CTAs of a cluster:
// a barrier is the cluster barrier; a reduction pushes each CTA's K block sums
// into slot [rank] of EVERY CTA's slot array (distributed shared memory,
// posted stores), crosses the barrier, and then each warp of each CTA adds the
// `size` slots of its own shared memory with the same fixed-order warp
// reduction -- the same additions in the same order everywhere, so all CTAs
// (and all warps) hold identical scalars, with no remote loads on the
// critical path and no block barrier after the sum. Slot arrays alternate
// between two buffers: buffer e % 2 is rewritten by exchange e + 2, which a
// CTA starts only after the barrier of exchange e + 1, which every thread of
// every CTA reaches only after it has read exchange e. Same interface as
// GridSync and BlockSync.
struct ClusterSync {
    double (*slots)[kMaxCluster][kSlotDoubles];   // this CTA's shared [2][kMaxCluster][kSlotDoubles]
    unsigned rank, size;
    unsigned epoch;     // reductions done
    int count;
};

__device__ __forceinline__ bool is_leader(const ClusterSync &g) { return g.rank == 0; }

__device__ __forceinline__ bool grid_sync(ClusterSync &g, double (*)[32], int *) {
    cluster_barrier();
    g.count++;
    return true;
}

template <int K>
__device__ __forceinline__ bool grid_sum(ClusterSync &g, double (&v)[K], double (*sm)[32], int *) {
    block_sum<K>(v, sm);   // ends with __syncthreads; every thread holds the block sums
    const unsigned buf = g.epoch & 1u;
    const unsigned t = threadIdx.x;
    if (t < g.size * K) {
        const unsigned dst = t / K, k = t - dst * K;
        double mine = v[0];
#pragma unroll
        for (int q = 1; q < K; ++q)
            if ((int)k == q) mine = v[q];
        st_cluster_f64(cluster_map(&g.slots[buf][g.rank][k], dst), mine);
    }
    cluster_barrier();
    // every warp: lane l holds slot l, then a fixed-order warp sum
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = lane < (int)g.size ? g.slots[buf][lane][k] : 0.0;
    warp_allsum<K>(v);
    g.epoch++;
    g.count++;
    return true;
}

}  // namespace pbcg
