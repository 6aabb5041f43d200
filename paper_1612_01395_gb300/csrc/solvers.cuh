// Persistent cooperative solver kernels: one launch runs a whole solve.
//
// Rows are split into gridDim.x contiguous ranges, one per thread block, and a
// thread owns the rows lo + threadIdx.x + m * kTPB of its block's range in
// every phase. A phase is one sweep over the rows that fuses an SpMV, the
// AXPY recurrences that consume it and the partial dot products of a
// reduction; phases are separated by grid_sum / grid_sync. Every block then
// holds the same reduced scalars (alpha, beta, omega, rho), so the scalars
// never leave the GPU and the host is not involved between iterations.
//
// Pipelined BiCGStab (Algorithm 9) takes 2 grid-wide synchronisations per
// iteration: on one GPU the SpMV of each phase needs its input vector complete
// across the grid, and that same synchronisation completes the reduction whose
// scalar the phase consumes -- the two reductions of Algorithm 9 ride on the
// two synchronisations its SpMVs need anyway. Standard BiCGStab (Algorithm 7)
// needs 3 (variant 3: neighbour values of p and q are formed on the fly inside
// the SpMV) or 5 (variant 5: p and q are written first, fewer FP64 operations).
#pragma once

#include "operators.cuh"

namespace pbcg {

template <typename T>
struct VectorsT {
    T *r, *r0, *p, *s, *z, *q, *y, *w, *t, *v;
};
using Vectors = VectorsT<double>;

template <typename T>
struct SolveArgsT {
    int n;
    const T *b;
    T *x;
    VectorsT<T> V;
    Control *ctl;
    double *partials;
    double *hist;       // nullable
    double rtol;
    int limit;          // iterations allowed (maxit or fixed_iters)
    int fixed;          // 1: ignore rtol
    int replace_period;
    int max_repl;       // < 0: unlimited
    int variant;        // Algorithm 7 only: 3 or 5
    // preconditioned solves (Algorithms 10 and 11): M^{-1} u = minv .* u and the
    // hat vectors r^, s^, z^, q^, w^ (null when unpreconditioned)
    const T *minv;
    T *rh, *sh, *zh, *qh, *wh;
};
using SolveArgs = SolveArgsT<double>;

// Resident blocks per SM the solver kernels are compiled for (register cap
// 65536 / (kTPB * kMinBlocks) = 64 at 8): the large-n sweeps are limited by
// the FP64 pipe, which needs many warps in flight to cover memory latency. At
// 256^3 the stencil kernels take 1.25 (p-BiCGStab) and 1.27 ms (BiCGStab) per
// iteration with 6 blocks per SM and 1.14 and 1.08 ms with 8. With 9 (56
// registers), p-BiCGStab slows to 1.20 ms while BiCGStab, whose sweeps hold
// fewer values, speeds up to 1.05 ms; 10 is slower for both. Each method's
// stencil kernel takes its own best.
template <class Op>
struct Tune {
    static constexpr int kMinBlocks = 8;
};
template <class Op>
struct TunePlain {
    static constexpr int kMinBlocks = Tune<Op>::kMinBlocks;
};
template <>
struct TunePlain<StencilOp> {
    static constexpr int kMinBlocks = 9;
};

struct Outcome {
    int iters, status, half, nrr;
    double nr0, nr;   // nr: squared norm of the last recursive residual (or of q after a half step)
};

template <int K>
__device__ __forceinline__ bool all_finite(const double (&v)[K]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < K; ++i) ok = ok && isfinite(v[i]);
    return ok;
}

#define PBCG_ROWS(i) for (int i = lo + (int)threadIdx.x; i < hi; i += kTPB)

// Stopping tests compare squared norms first, so that the square root (about
// ten FP64 instructions, ~700 cycles per warp on this GPU) stays off the
// critical path: sqrt(a) <= tol implies a <= 2 tol^2, and the exact test
// sqrt(a) <= tol is then evaluated only in that rare case.
__device__ __forceinline__ bool norm_below(double sq, double tol, double tol2) {
    return (sq <= 2.0 * tol2 || !(tol2 >= 2.2250738585072014e-308)) && sqrt(sq) <= tol;
}

// The divisions of an iteration's scalar updates are evaluated once per block,
// by one warp each, and shared through shared memory. An FP64 warp
// instruction occupies its sub-partition's FP64 pipe for 64 cycles whether
// one warp or all four compute the same scalar, so with several resident
// blocks per SM the redundant copies queued on the same pipes, on the
// critical path between two sweeps. The warp is rotated by the block index,
// (blockIdx.x + k) mod 4, so the resident blocks spread their divisions over
// the four sub-partitions. Every thread receives the same bits as before.
// sq: a row of 32 shared doubles; slots 0-1 beta, 2-3 den and alpha, 4 omega.
__device__ __forceinline__ int scalar_warp(int k) { return (int)((blockIdx.x + (unsigned)k) % (kTPB / 32)); }

// a / b on one warp, returned to every thread (the slot is rewritten only
// after later barriers).
__device__ __forceinline__ double div_shared(double a, double b, int warp, double *slot) {
    if ((int)(threadIdx.x >> 5) == warp) {
        const double q = __ddiv_rn(a, b);
        if ((threadIdx.x & 31) == 0) *slot = q;
    }
    __syncthreads();
    return *slot;
}

// Denominator of eq. (3), r0w + beta r0s - beta omega r0z, and alpha_{i+1} =
// rho_n / den (only when den != 0) on one warp; both returned to every thread.
__device__ __forceinline__ void alpha_shared(double rho_n, double r0w, double r0s, double r0z, double beta,
                                             double omega, double *sq, double &den, double &alpha) {
    if ((int)(threadIdx.x >> 5) == scalar_warp(2)) {
        const double d = __dsub_rn(__dadd_rn(r0w, __dmul_rn(beta, r0s)), __dmul_rn(__dmul_rn(beta, omega), r0z));
        const double al = d == 0.0 ? 0.0 : __ddiv_rn(rho_n, d);
        if ((threadIdx.x & 31) == 0) {
            sq[2] = d;
            sq[3] = al;
        }
    }
    __syncthreads();
    den = sq[2];
    alpha = sq[3];
}

// beta = (alpha / omega) (rho_n / rho): the two divisions are independent, so
// two warps evaluate one each (every warp has its own FP64 pipe) and share
// them through shared memory.
__device__ __forceinline__ double beta_of(double alpha, double omega, double rho_n, double rho, double *sq) {
    const int wid = threadIdx.x >> 5;
    if (wid == scalar_warp(0)) sq[0] = __ddiv_rn(alpha, omega);
    if (wid == scalar_warp(1)) sq[1] = __ddiv_rn(rho_n, rho);
    __syncthreads();
    const double b = __dmul_rn(sq[0], sq[1]);
    __syncthreads();
    return b;
}

// Final true residual ||b - A x|| and the result record (block 0). The
// history holds squared norms during the loop; they become norms here.
template <class Op, class Sync>
__device__ __forceinline__ void finish(const Op &A, const SolveArgs &a, Sync &g, double (*sm)[32], int *sflag,
                                       int lo, int hi, const Outcome &o, int spmvs) {
    double d[1] = {0.0};
    PBCG_ROWS(i) {
        const double res = a.b[i] - A.row(i, VecLoad{a.x});
        d[0] = fma(res, res, d[0]);
    }
    if (!grid_sum<1>(g, d, sm, sflag)) return;
    if (blockIdx.x == 0) {
        if (a.hist)
            for (int i = 1 + (int)threadIdx.x; i <= o.iters; i += kTPB) a.hist[i] = sqrt(a.hist[i]);
        if (threadIdx.x == 0) {
            Control *c = a.ctl;
            const double nt = sqrt(d[0]);
            const double nr = o.iters > 0 ? sqrt(o.nr) : o.nr0;
            c->iters = o.iters;
            c->status = o.status;
            c->half_step = o.half;
            c->n_repl = o.nrr;
            c->grid_syncs = g.count;
            c->spmvs = spmvs + 1;
            c->nr0 = o.nr0;
            c->rel_rec = o.nr0 > 0.0 ? nr / o.nr0 : 0.0;
            c->rel_true = o.nr0 > 0.0 ? nt / o.nr0 : nt;
        }
    }
}

// Per-thread accumulation of a dot product over the rows of a sweep. FP64
// vectors: an FMA into a double. FP32 vectors (the inner solves of the
// mixed-precision refinement, CSR and stencil form): compensated FP32
// accumulation, algorithm Dot2 of Ogita, Rump & Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005): each product is split exactly into
// its rounded value and rounding error (TwoProduct by FMA), the running sum is
// updated by the error-free TwoSum and all errors are summed apart; the result
// is as accurate as if accumulated in twice the working precision and is
// converted to double once per thread and sweep, and the threads' values are
// summed in FP64. On this GPU an FP32 operation costs 1/64 of an FP64 one, so
// the inner solves keep FP64-grade dot products (the ones that set alpha,
// beta and omega) without any FP64 instruction per row. Explicit _rn
// intrinsics keep the compiler from fusing the steps of the error-free
// transformations.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);   // a b - p, exactly
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));   // s + p - t, exactly
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <class Op, typename T>
struct DotAccFor {
    using type = DotAcc<T>;
};

template <class Acc, int K>
__device__ __forceinline__ void dot_values(const Acc (&acc)[K], double (&d)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = acc[k].value();
}

// G adjacent elements p[i..i+cnt) of a vector (cnt <= G; the rest read as 0)
// and their store. G = 2 uses one 64-bit access when both are present: i is
// even and the vectors are 8-byte aligned (the FP32 inner sweeps).
template <int G, typename T>
__device__ __forceinline__ void load_group(const T *p, int i, int cnt, T (&out)[G]) {
    if constexpr (G == 2 && sizeof(T) == 4) {
        if (cnt == 2) {
            const float2 q = *reinterpret_cast<const float2 *>(p + i);
            out[0] = q.x;
            out[1] = q.y;
            return;
        }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) out[u] = u < cnt ? p[i + u] : T(0);
}
// load_group for a fused sweep: through L2 only (ld.global.cg) for operators
// whose sweeps leave L1 to their SpMV's row streams.
template <class Op, int G, typename T>
__device__ __forceinline__ void load_sweep(const T *p, int i, int cnt, T (&out)[G]) {
    if constexpr (SweepLoadsL2<Op>::value) {
#pragma unroll
        for (int u = 0; u < G; ++u) out[u] = u < cnt ? __ldcg(p + i + u) : T(0);
    } else {
        load_group(p, i, cnt, out);
    }
}
template <int G, typename T>
__device__ __forceinline__ void store_group(T *p, int i, int cnt, const T (&in)[G]) {
    if constexpr (G == 2 && sizeof(T) == 4) {
        if (cnt == 2) {
            *reinterpret_cast<float2 *>(p + i) = make_float2(in[0], in[1]);
            return;
        }
    }
#pragma unroll
    for (int u = 0; u < G; ++u)
        if (u < cnt) p[i + u] = in[u];
}

// ===========================================================================
// Staged FP32 stencil sweeps (the inner solves of the mixed-precision
// refinement). These sweeps move 96 bytes per unknown and iteration and were
// bound by load latency with every thread issuing its own vector loads. Here
// the vectors a phase streams (read once, by the rows' own block) arrive in
// shared memory by 1-D bulk copies: a block walks its rows in tiles of
// kStageRows, thread 0 keeps kStages - 1 tiles in flight ahead of the one it
// computes, and the threads read their rows from shared memory. Each buffer
// has a "full" mbarrier (the copies' bytes arrived) and an "empty" one (all
// threads have read it): thread 0 refills a buffer only after every thread
// released it, so warps are not held together tile by tile and may run up to
// kStages - 1 tiles apart. The SpMV input (neighbours in other tiles and
// blocks) and the stores stay ordinary global accesses. Block row ranges
// start on multiples of 4 rows, so every copy starts on a 16-byte boundary;
// the last tile's copy is rounded up to 16 bytes, inside the vectors' padding.
// ===========================================================================
// (The same staging of the FP64 stencil sweeps of Algorithm 9 gave bitwise
// identical results but was 2.7 % slower at 256^3, 1178 against 1148 us per
// iteration: those sweeps are bound by the FP64 pipe, and staging only adds
// instructions. They keep their direct loads.)
constexpr int kStageTileBytes = 1024;   // per vector and tile: 256 FP32 rows (a pair per thread) or 128 FP64 rows
constexpr int kStages = 3;              // buffers: 2 tiles in flight ahead
constexpr int kStageVecs = 6;           // streamed vectors per phase
constexpr int kStageRows = kStageTileBytes / (int)sizeof(float);   // FP32 rows per tile
constexpr size_t kStageSmemBytes = (size_t)kStages * kStageVecs * kStageTileBytes;

struct Stager {
    char *buf;         // shared [kStages][kStageVecs][kStageTileBytes]
    uint64_t *full;    // shared [kStages]: copies of the buffer's tile arrived (count 1 + bytes)
    uint64_t *empty;   // shared [kStages]: every thread finished reading the buffer (count kTPB)
    unsigned seq;      // tiles begun by this block so far (every thread holds the same value)
    Control *ctl;
};

// thread 0: post and issue the copies of tile `seq` (rows [row0, row0 + rows)),
// the byte count rounded up to 16.
template <typename T, int NV>
__device__ __forceinline__ void stage_issue(const Stager &S, unsigned seq, const T *const *src, int row0, int rows) {
    const unsigned b = seq % kStages;
    const unsigned bytes = ((unsigned)rows * (unsigned)sizeof(T) + 15u) & ~15u;
    mbar_arrive_expect_tx(&S.full[b], bytes * NV);
#pragma unroll
    for (int k = 0; k < NV; ++k)
        bulk_g2s(S.buf + ((size_t)b * kStageVecs + k) * kStageTileBytes, src[k] + row0, bytes, &S.full[b]);
}

// Run body(tile buffer, first row of the tile) over the block's rows [lo, hi)
// with the NV (<= kStageVecs) vectors `src` staged, in tiles of
// kStageTileBytes / sizeof(T) rows. Every staged vector must be a workspace
// vector (16-byte aligned, padded past n). Returns false if a wait timed out.
template <typename T, int NV, class Body>
__device__ __forceinline__ bool staged_sweep(Stager &S, const T *const *src, int lo, int hi, Body body) {
    static_assert(NV <= kStageVecs, "at most kStageVecs staged vectors");
    constexpr int R = kStageTileBytes / (int)sizeof(T);
    const int ntiles = hi > lo ? (hi - lo + R - 1) / R : 0;
    // every thread: earlier generic writes of these rows (this block's, made
    // visible by the preceding barriers) before the copies read them; after
    // this barrier every thread has also released every buffer
    fence_proxy_async_global();
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 0; t < kStages - 1 && t < ntiles; ++t) {
            const int r0 = lo + t * R;
            stage_issue<T, NV>(S, S.seq + t, src, r0, hi - r0 < R ? hi - r0 : R);
        }
    for (int t = 0; t < ntiles; ++t) {
        const unsigned seq = S.seq + (unsigned)t;
        const int ahead = t + kStages - 1;
        if (threadIdx.x == 0 && ahead < ntiles) {
            // the buffer of tile seq + kStages - 1 last held tile seq - 1: wait until all threads released it
            if (seq >= 1 && !mbar_wait(&S.empty[(seq - 1) % kStages], ((seq - 1) / kStages) & 1u, S.ctl)) return false;
            const int r0 = lo + ahead * R;
            stage_issue<T, NV>(S, seq + kStages - 1, src, r0, hi - r0 < R ? hi - r0 : R);
        }
        if (!mbar_wait(&S.full[seq % kStages], (seq / kStages) & 1u, S.ctl)) return false;
        body(reinterpret_cast<const T *>(S.buf + (size_t)(seq % kStages) * kStageVecs * kStageTileBytes), lo + t * R);
        mbar_arrive(&S.empty[seq % kStages]);   // this thread is done with the buffer
    }
    S.seq += (unsigned)ntiles;
    return true;
}

// Elements j, j+1 of a staged vector (j even: one 64-bit shared load).
__device__ __forceinline__ void staged_pair(const float *tb, int k, int j, float (&out)[2]) {
    const float2 v = *reinterpret_cast<const float2 *>(tb + k * kStageRows + j);
    out[0] = v.x;
    out[1] = v.y;
}

// ===========================================================================
// Algorithm 9 (pipelined BiCGStab) with the residual replacement of
// Section 4.2 (r := b - A x, w := A r before the second reduction of iteration
// i-1; s := A p, z := A s after p_i; for i mod k == 0).
// ===========================================================================
// T is the vector and sweep arithmetic type: double for the FP64 solver,
// float for the inner solves of the mixed-precision refinement. Dot products
// are summed per thread in T (DotAccFor) and across threads in double, and
// alpha, beta, omega, rho are doubles; a sweep uses them rounded to T.
template <class Op, typename T, class Sync = GridSync>
__device__ __forceinline__ bool pipelined_loop(const Op &A, const SolveArgsT<T> &a, Sync &g, double (*sm)[32],
                                               int *sflag, int lo, int hi, Outcome &o, int &spmvs,
                                               Stager *stg = nullptr) {
    const VectorsT<T> &V = a.V;
    T *x = a.x;
    const bool fixed = a.fixed != 0;
    // Rows per thread and step of the two main sweeps: kGroup adjacent rows,
    // loaded before any is stored (the stores of one row may alias the loads
    // of the next as far as the compiler knows). FP64 sweeps are bound by the
    // FP64 pipe and take one row. The FP32 inner sweeps are bound by load
    // latency and take two adjacent rows with 64-bit vector accesses, which
    // halves their load and store instructions; their callers give every
    // block an even first row.
    constexpr int kGroup = sizeof(T) == 4 ? 2 : 1;
    using Acc = typename DotAccFor<Op, T>::type;

    // r_0 := b - A x_0; shadow r0 := r_0; p, s, z, v := 0 (they are multiplied by beta_{-1} = 0)
    double d0[1];
    {
        Acc acc[1];
        PBCG_ROWS(i) {
            const T ri = a.b[i] - A.row(i, VecLoadT<T>{x});
            V.r[i] = ri;
            V.r0[i] = ri;
            V.p[i] = T(0);
            V.s[i] = T(0);
            V.z[i] = T(0);
            V.v[i] = T(0);
            acc[0].add(ri, ri);
        }
        dot_values(acc, d0);
    }
    ++spmvs;
    if (!grid_sum<1>(g, d0, sm, sflag)) return false;
    double rho = d0[0];                 // (r0, r_0)
    o.nr0 = sqrt(rho);
    o.nr = o.nr0;
    if (threadIdx.x == 0 && a.hist && is_leader(g)) a.hist[0] = o.nr0;
    const double tol = __dmul_rn(a.rtol, o.nr0), tol2 = __dmul_rn(tol, tol);
    if (o.nr0 == 0.0) { o.status = PBCG_OK; return true; }

    // w_0 := A r_0; alpha_0 := (r0, r0) / (r0, w0)
    {
        Acc acc[1];
        PBCG_ROWS(i) {
            const T wi = A.row(i, VecLoadT<T>{V.r});
            V.w[i] = wi;
            acc[0].add(V.r0[i], wi);
        }
        dot_values(acc, d0);
    }
    ++spmvs;
    if (!grid_sum<1>(g, d0, sm, sflag)) return false;
    if (!isfinite(d0[0])) { o.status = PBCG_NONFINITE; return true; }
    if (d0[0] == 0.0) { o.status = PBCG_BREAKDOWN; return true; }
    double alpha = __ddiv_rn(rho, d0[0]), beta = 0.0, omega = 0.0;

    bool replaced_rw = false;   // r_i, w_i were replaced at the end of iteration i-1
    int it = 0;
    while (it < a.limit) {
        // ---- phase A: t_i = A w_i; p_i, s_i, z_i, q_i, y_i; first reduction
        Acc a1[5];   // (q,y) (y,y) (q,q) (r0,s) (r0,z)
        const T al = (T)alpha, be = (T)beta, om = (T)omega;
        bool swept = false;   // the staged sweep did phase A
        if constexpr (kGroup == 2 && HasRow2<Op>::value) {
            if (!replaced_rw && stg) {
                // staged: r s z p v r0 through shared memory, w (SpMV) from global
                const float *src[kStageVecs] = {V.r, V.s, V.z, V.p, V.v, V.r0};
                const bool ok = staged_sweep<float, kStageVecs>(*stg, src, lo, hi, [&](const float *tb, int row0) {
                    const int j = 2 * (int)threadIdx.x;
                    const int i0 = row0 + j;
                    if (i0 >= hi) return;
                    const int cnt = hi - i0 < 2 ? hi - i0 : 2;
                    T ti[2] = {}, ri[2], wi[2], si[2], zi[2], pi[2], vi[2], r0i[2];
                    if (cnt == 2 && A.pairs_on_lines()) {
                        A.row2(i0, V.w, ti);
                    } else {
#pragma unroll
                        for (int u = 0; u < 2; ++u)
                            if (u < cnt) ti[u] = A.row(i0 + u, VecLoadT<T>{V.w});
                    }
                    load_group(V.w, i0, cnt, wi);
                    staged_pair(tb, 0, j, ri);
                    staged_pair(tb, 1, j, si);
                    staged_pair(tb, 2, j, zi);
                    staged_pair(tb, 3, j, pi);
                    staged_pair(tb, 4, j, vi);
                    staged_pair(tb, 5, j, r0i);
                    T pn[2], sn[2], zn[2], qn[2], yn[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        pn[u] = fmaT(be, fmaT(-om, si[u], pi[u]), ri[u]);   // p_i
                        sn[u] = fmaT(be, fmaT(-om, zi[u], si[u]), wi[u]);   // s_i, eq. (1)
                        zn[u] = fmaT(be, fmaT(-om, vi[u], zi[u]), ti[u]);   // z_i, eq. (6)
                        qn[u] = fmaT(-al, sn[u], ri[u]);                    // q_i
                        yn[u] = fmaT(-al, zn[u], wi[u]);                    // y_i, eq. (4)
                        if (u < cnt) {
                            a1[0].add(qn[u], yn[u]);
                            a1[1].add(yn[u], yn[u]);
                            a1[2].add(qn[u], qn[u]);
                            a1[3].add(r0i[u], sn[u]);
                            a1[4].add(r0i[u], zn[u]);
                        }
                    }
                    store_group(V.t, i0, cnt, ti);
                    store_group(V.p, i0, cnt, pn);
                    store_group(V.s, i0, cnt, sn);
                    store_group(V.z, i0, cnt, zn);
                    store_group(V.q, i0, cnt, qn);
                    store_group(V.y, i0, cnt, yn);
                });
                if (!ok) return false;
                ++spmvs;
                swept = true;
            }
        }
        if (swept) {
        } else if (!replaced_rw) {
            for (int i0 = lo + kGroup * (int)threadIdx.x; i0 < hi; i0 += kGroup * kTPB) {
                const int cnt = kGroup == 1 ? 1 : (hi - i0 < kGroup ? hi - i0 : kGroup);
                T ti[kGroup] = {}, ri[kGroup], wi[kGroup], si[kGroup], zi[kGroup], pi[kGroup], vi[kGroup], r0i[kGroup];
                if constexpr (kGroup == 2 && HasRow2<Op>::value) {
                    if (cnt == 2 && A.pairs_on_lines()) {
                        A.row2(i0, V.w, ti);
                    } else {
#pragma unroll
                        for (int u = 0; u < kGroup; ++u)
                            if (u < cnt) ti[u] = A.row(i0 + u, VecLoadT<T>{V.w});
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < kGroup; ++u)
                        if (u < cnt) ti[u] = A.row(i0 + u, VecLoadT<T>{V.w});
                }
                load_sweep<Op>(V.r, i0, cnt, ri);
                load_sweep<Op>(V.w, i0, cnt, wi);
                load_sweep<Op>(V.s, i0, cnt, si);
                load_sweep<Op>(V.z, i0, cnt, zi);
                load_sweep<Op>(V.p, i0, cnt, pi);
                load_sweep<Op>(V.v, i0, cnt, vi);
                load_sweep<Op>(V.r0, i0, cnt, r0i);
                T pn[kGroup], sn[kGroup], zn[kGroup], qn[kGroup], yn[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    pn[u] = fmaT(be, fmaT(-om, si[u], pi[u]), ri[u]);   // p_i
                    sn[u] = fmaT(be, fmaT(-om, zi[u], si[u]), wi[u]);   // s_i, eq. (1)
                    zn[u] = fmaT(be, fmaT(-om, vi[u], zi[u]), ti[u]);   // z_i, eq. (6)
                    qn[u] = fmaT(-al, sn[u], ri[u]);                    // q_i
                    yn[u] = fmaT(-al, zn[u], wi[u]);                    // y_i, eq. (4)
                    if (u < cnt) {
                        a1[0].add(qn[u], yn[u]);
                        a1[1].add(yn[u], yn[u]);
                        a1[2].add(qn[u], qn[u]);
                        a1[3].add(r0i[u], sn[u]);
                        a1[4].add(r0i[u], zn[u]);
                    }
                }
                store_group(V.t, i0, cnt, ti);
                store_group(V.p, i0, cnt, pn);
                store_group(V.s, i0, cnt, sn);
                store_group(V.z, i0, cnt, zn);
                store_group(V.q, i0, cnt, qn);
                store_group(V.y, i0, cnt, yn);
            }
            ++spmvs;
        } else {
            // replacement, second part: t_i = A w_i (w_i replaced), p_i; then s_i := A p_i; z_i := A s_i
            PBCG_ROWS(i) {
                V.t[i] = A.row(i, VecLoadT<T>{V.w});
                V.p[i] = fmaT(be, fmaT(-om, V.s[i], V.p[i]), V.r[i]);
            }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) { V.s[i] = A.row(i, VecLoadT<T>{V.p}); }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const T zn = A.row(i, VecLoadT<T>{V.s});
                const T sn = V.s[i], ri = V.r[i], wi = V.w[i];
                const T qi = fmaT(-al, sn, ri);
                const T yi = fmaT(-al, zn, wi);
                V.z[i] = zn;
                V.q[i] = qi;
                V.y[i] = yi;
                const T r0i = V.r0[i];
                a1[0].add(qi, yi);
                a1[1].add(yi, yi);
                a1[2].add(qi, qi);
                a1[3].add(r0i, sn);
                a1[4].add(r0i, zn);
            }
            spmvs += 3;
        }
        double d1[5];
        dot_values(a1, d1);
        if (!grid_sum<5>(g, d1, sm, sflag)) return false;
        const double qy = d1[0], yy = d1[1], qq = d1[2], r0s = d1[3], r0z = d1[4];
        if (!all_finite(d1)) { o.status = PBCG_NONFINITE; break; }
        const bool small_q = !fixed && norm_below(qq, tol, tol2);
        if (small_q || yy == 0.0) {
            if (!small_q && qq != 0.0) { o.status = PBCG_BREAKDOWN; break; }
            PBCG_ROWS(i) { x[i] = fmaT(al, V.p[i], x[i]); }   // half step x_i + alpha_i p_i
            if (!grid_sync(g, sm, sflag)) return false;
            ++it;
            o.nr = qq;
            o.half = 1;
            o.status = PBCG_OK;
            if (threadIdx.x == 0 && a.hist && is_leader(g)) a.hist[it] = qq;
            break;
        }
        omega = div_shared(qy, yy, scalar_warp(3), &sm[kMaxDots - 1][4]);
        if (omega == 0.0) { o.status = PBCG_BREAKDOWN; break; }

        // ---- phase B: v_i = A z_i; x_{i+1}, r_{i+1}, w_{i+1}; second reduction
        const bool replace_now = a.replace_period > 0 && (it + 1) % a.replace_period == 0 &&
                                 (a.max_repl < 0 || o.nrr < a.max_repl);
        Acc a2[3];   // (r0,r) (r0,w) (r,r)
        const T om2 = (T)omega;
        bool swept_b = false;   // the staged sweep did phase B
        if constexpr (kGroup == 2 && HasRow2<Op>::value) {
            if (!replace_now && stg) {
                // staged: q y x p t r0 through shared memory, z (SpMV) from global
                const float *src[kStageVecs] = {V.q, V.y, x, V.p, V.t, V.r0};
                const bool ok = staged_sweep<float, kStageVecs>(*stg, src, lo, hi, [&](const float *tb, int row0) {
                    const int j = 2 * (int)threadIdx.x;
                    const int i0 = row0 + j;
                    if (i0 >= hi) return;
                    const int cnt = hi - i0 < 2 ? hi - i0 : 2;
                    T vi[2] = {}, qi[2], yi[2], xi[2], pi[2], ti[2], r0i[2];
                    if (cnt == 2 && A.pairs_on_lines()) {
                        A.row2(i0, V.z, vi);
                    } else {
#pragma unroll
                        for (int u = 0; u < 2; ++u)
                            if (u < cnt) vi[u] = A.row(i0 + u, VecLoadT<T>{V.z});
                    }
                    staged_pair(tb, 0, j, qi);
                    staged_pair(tb, 1, j, yi);
                    staged_pair(tb, 2, j, xi);
                    staged_pair(tb, 3, j, pi);
                    staged_pair(tb, 4, j, ti);
                    staged_pair(tb, 5, j, r0i);
                    T xn[2], rn[2], wn[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        xn[u] = fmaT(om2, qi[u], fmaT(al, pi[u], xi[u]));
                        rn[u] = fmaT(-om2, yi[u], qi[u]);                     // eq. (7)
                        wn[u] = fmaT(-om2, fmaT(-al, vi[u], ti[u]), yi[u]);   // eq. (8)
                        if (u < cnt) {
                            a2[0].add(r0i[u], rn[u]);
                            a2[1].add(r0i[u], wn[u]);
                            a2[2].add(rn[u], rn[u]);
                        }
                    }
                    store_group(x, i0, cnt, xn);
                    store_group(V.v, i0, cnt, vi);
                    store_group(V.r, i0, cnt, rn);
                    store_group(V.w, i0, cnt, wn);
                });
                if (!ok) return false;
                ++spmvs;
                swept_b = true;
            }
        }
        if (swept_b) {
        } else if (!replace_now) {
            for (int i0 = lo + kGroup * (int)threadIdx.x; i0 < hi; i0 += kGroup * kTPB) {
                const int cnt = kGroup == 1 ? 1 : (hi - i0 < kGroup ? hi - i0 : kGroup);
                T vi[kGroup] = {}, qi[kGroup], yi[kGroup], xi[kGroup], pi[kGroup], ti[kGroup], r0i[kGroup];
                if constexpr (kGroup == 2 && HasRow2<Op>::value) {
                    if (cnt == 2 && A.pairs_on_lines()) {
                        A.row2(i0, V.z, vi);
                    } else {
#pragma unroll
                        for (int u = 0; u < kGroup; ++u)
                            if (u < cnt) vi[u] = A.row(i0 + u, VecLoadT<T>{V.z});
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < kGroup; ++u)
                        if (u < cnt) vi[u] = A.row(i0 + u, VecLoadT<T>{V.z});
                }
                load_sweep<Op>(V.q, i0, cnt, qi);
                load_sweep<Op>(V.y, i0, cnt, yi);
                load_sweep<Op>(x, i0, cnt, xi);
                load_sweep<Op>(V.p, i0, cnt, pi);
                load_sweep<Op>(V.t, i0, cnt, ti);
                load_sweep<Op>(V.r0, i0, cnt, r0i);
                T xn[kGroup], rn[kGroup], wn[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    xn[u] = fmaT(om2, qi[u], fmaT(al, pi[u], xi[u]));
                    rn[u] = fmaT(-om2, yi[u], qi[u]);                     // eq. (7)
                    wn[u] = fmaT(-om2, fmaT(-al, vi[u], ti[u]), yi[u]);   // eq. (8)
                    if (u < cnt) {
                        a2[0].add(r0i[u], rn[u]);
                        a2[1].add(r0i[u], wn[u]);
                        a2[2].add(rn[u], rn[u]);
                    }
                }
                store_group(x, i0, cnt, xn);
                store_group(V.v, i0, cnt, vi);
                store_group(V.r, i0, cnt, rn);
                store_group(V.w, i0, cnt, wn);
            }
            ++spmvs;
        } else {
            // replacement, first part: x_{i+1}; r_{i+1} := b - A x_{i+1}; w_{i+1} := A r_{i+1}
            PBCG_ROWS(i) { x[i] = fmaT(om2, V.q[i], fmaT(al, V.p[i], x[i])); }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) { V.r[i] = a.b[i] - A.row(i, VecLoadT<T>{x}); }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const T wn = A.row(i, VecLoadT<T>{V.r});
                const T ri = V.r[i], r0i = V.r0[i];
                V.w[i] = wn;
                a2[0].add(r0i, ri);
                a2[1].add(r0i, wn);
                a2[2].add(ri, ri);
            }
            spmvs += 2;
            o.nrr++;
        }
        double d2[3];
        dot_values(a2, d2);
        replaced_rw = replace_now;
        if (!grid_sum<3>(g, d2, sm, sflag)) return false;
        ++it;
        const double rho_n = d2[0], r0w = d2[1];
        o.nr = d2[2];
        if (threadIdx.x == 0 && a.hist && is_leader(g)) a.hist[it] = d2[2];
        if (!all_finite(d2)) { o.status = PBCG_NONFINITE; break; }
        if (!fixed && norm_below(d2[2], tol, tol2)) { o.status = PBCG_OK; break; }
        if (rho_n == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        // beta_i = (alpha_i / omega_i) (r0, r_{i+1}) / (r0, r_i); alpha_{i+1} by eq. (3)
        beta = beta_of(alpha, omega, rho_n, rho, sm[kMaxDots - 1]);
        double den;
        alpha_shared(rho_n, r0w, r0s, r0z, beta, omega, sm[kMaxDots - 1], den, alpha);
        if (den == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        rho = rho_n;
    }
    o.iters = it;
    if (it == a.limit && o.status == PBCG_NOT_CONVERGED && fixed) o.status = PBCG_OK;
    return true;
}

// ===========================================================================
// Algorithm 11 (preconditioned pipelined BiCGStab) with a diagonal M^{-1},
// applied elementwise inside the sweeps, so an iteration still takes two
// grid-wide exchanges. The hat vectors of Algorithm 11 are M^{-1} times their
// plain counterparts (r^ = M^{-1} r, s^ = M^{-1} s, q^ = M^{-1} q, z^, w^);
// the algorithm carries r^, s^, q^ as recurrences because applying a general
// M^{-1} costs a solve. With a diagonal M^{-1} it costs one product, so this
// loop forms r^, s^, q^ where they are used (m_i r_i, m_i s_i, m_i q_i) and
// stores only the hat vectors an SpMV reads: z^ (v = A z^) and w^ (t = A w^),
// plus p^ (V.p). That removes the r^, s^, q^ recurrences and their 48 bytes
// per unknown and iteration of traffic; in exact arithmetic the iterates are
// Algorithm 11's. Residual replacement (Section 4.2): r := b - A x and
// w := A r^ before the second reduction of iteration i-1; s := A p^ and
// z := A s^ after p^_i; r^ and s^ are then stored as SpMV inputs (rh, sh).
// ===========================================================================
template <class Op>
__device__ __forceinline__ bool pipelined_prec_loop(const Op &A, const SolveArgs &a, GridSync &g, double (*sm)[32],
                                                    int *sflag, int lo, int hi, Outcome &o, int &spmvs) {
    const Vectors &V = a.V;
    double *x = a.x;
    const double *mi = a.minv;
    double *rh = a.rh, *sh = a.sh, *zh = a.zh, *wh = a.wh;
    const bool fixed = a.fixed != 0;

    // r_0 := b - A x_0; r0 := r_0; r^_0 := M^{-1} r_0 (an SpMV input); p^, s, z, v := 0
    double d0[1] = {0.0};
    PBCG_ROWS(i) {
        const double ri = a.b[i] - A.row(i, VecLoad{x});
        V.r[i] = ri;
        V.r0[i] = ri;
        rh[i] = mi[i] * ri;
        V.p[i] = 0.0;
        V.s[i] = 0.0;
        V.z[i] = 0.0;
        V.v[i] = 0.0;
        d0[0] = fma(ri, ri, d0[0]);
    }
    ++spmvs;
    if (!grid_sum<1>(g, d0, sm, sflag)) return false;
    double rho = d0[0];
    o.nr0 = sqrt(rho);
    o.nr = o.nr0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[0] = o.nr0;
    const double tol = __dmul_rn(a.rtol, o.nr0), tol2 = __dmul_rn(tol, tol);
    if (o.nr0 == 0.0) { o.status = PBCG_OK; return true; }

    // w_0 := A r^_0; w^_0 := M^{-1} w_0; alpha_0 := (r0, r0) / (r0, w0)
    d0[0] = 0.0;
    PBCG_ROWS(i) {
        const double wi = A.row(i, VecLoad{rh});
        V.w[i] = wi;
        wh[i] = mi[i] * wi;
        d0[0] = fma(V.r0[i], wi, d0[0]);
    }
    ++spmvs;
    if (!grid_sum<1>(g, d0, sm, sflag)) return false;
    if (!isfinite(d0[0])) { o.status = PBCG_NONFINITE; return true; }
    if (d0[0] == 0.0) { o.status = PBCG_BREAKDOWN; return true; }
    double alpha = __ddiv_rn(rho, d0[0]), beta = 0.0, omega = 0.0;

    bool replaced = false;
    int it = 0;
    while (it < a.limit) {
        // ---- phase A: t = A w^; p^, s, z, z^, q, y; first reduction
        double d1[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // (q,y) (y,y) (q,q) (r0,s) (r0,z)
        if (!replaced) {
            PBCG_ROWS(i) {
                const double ti = A.row(i, VecLoad{wh});
                const double m = mi[i], ri = V.r[i], si = V.s[i], zi = V.z[i], wi = V.w[i];
                const double ph = fma(beta, fma(-omega, m * si, V.p[i]), m * ri);   // p^_i = r^_i + beta (p^ - omega s^)
                const double sn = fma(beta, fma(-omega, zi, si), wi);               // s_i
                const double zn = fma(beta, fma(-omega, V.v[i], zi), ti);           // z_i
                const double qi = fma(-alpha, sn, ri);                              // q_i
                const double yi = fma(-alpha, zn, wi);                              // y_i
                V.t[i] = ti;
                V.p[i] = ph;
                V.s[i] = sn;
                V.z[i] = zn;
                zh[i] = m * zn;                                                     // z^_i
                V.q[i] = qi;
                V.y[i] = yi;
                const double r0i = V.r0[i];
                d1[0] = fma(qi, yi, d1[0]);
                d1[1] = fma(yi, yi, d1[1]);
                d1[2] = fma(qi, qi, d1[2]);
                d1[3] = fma(r0i, sn, d1[3]);
                d1[4] = fma(r0i, zn, d1[4]);
            }
            ++spmvs;
        } else {
            // replacement, second part: t = A w^ (w^ replaced), p^; then s := A p^, s^ := M^{-1} s, z := A s^
            PBCG_ROWS(i) {
                const double m = mi[i];
                V.t[i] = A.row(i, VecLoad{wh});
                V.p[i] = fma(beta, fma(-omega, m * V.s[i], V.p[i]), m * V.r[i]);   // r^ = M^{-1} r replaced
            }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const double sn = A.row(i, VecLoad{V.p});
                V.s[i] = sn;
                sh[i] = mi[i] * sn;
            }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const double zn = A.row(i, VecLoad{sh});
                const double sn = V.s[i];
                const double qi = fma(-alpha, sn, V.r[i]);
                const double yi = fma(-alpha, zn, V.w[i]);
                V.z[i] = zn;
                zh[i] = mi[i] * zn;
                V.q[i] = qi;
                V.y[i] = yi;
                const double r0i = V.r0[i];
                d1[0] = fma(qi, yi, d1[0]);
                d1[1] = fma(yi, yi, d1[1]);
                d1[2] = fma(qi, qi, d1[2]);
                d1[3] = fma(r0i, sn, d1[3]);
                d1[4] = fma(r0i, zn, d1[4]);
            }
            spmvs += 3;
        }
        if (!grid_sum<5>(g, d1, sm, sflag)) return false;
        const double qy = d1[0], yy = d1[1], qq = d1[2], r0s = d1[3], r0z = d1[4];
        if (!all_finite(d1)) { o.status = PBCG_NONFINITE; break; }
        const bool small_q = !fixed && norm_below(qq, tol, tol2);
        if (small_q || yy == 0.0) {
            if (!small_q && qq != 0.0) { o.status = PBCG_BREAKDOWN; break; }
            PBCG_ROWS(i) { x[i] = fma(alpha, V.p[i], x[i]); }   // half step x_i + alpha_i p^_i
            if (!grid_sync(g, sm, sflag)) return false;
            ++it;
            o.nr = qq;
            o.half = 1;
            o.status = PBCG_OK;
            if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[it] = qq;
            break;
        }
        omega = div_shared(qy, yy, scalar_warp(3), &sm[kMaxDots - 1][4]);
        if (omega == 0.0) { o.status = PBCG_BREAKDOWN; break; }

        // ---- phase B: v = A z^; x, r, w, w^; second reduction
        const bool replace_now = a.replace_period > 0 && (it + 1) % a.replace_period == 0 &&
                                 (a.max_repl < 0 || o.nrr < a.max_repl);
        double d2[3] = {0.0, 0.0, 0.0};   // (r0,r) (r0,w) (r,r)
        if (!replace_now) {
            PBCG_ROWS(i) {
                const double vi = A.row(i, VecLoad{zh});
                const double m = mi[i], qi = V.q[i], yi = V.y[i];
                x[i] = fma(omega, m * qi, fma(alpha, V.p[i], x[i]));   // x + alpha p^ + omega q^
                const double rn = fma(-omega, yi, qi);
                const double wn = fma(-omega, fma(-alpha, vi, V.t[i]), yi);
                V.v[i] = vi;
                V.r[i] = rn;
                V.w[i] = wn;
                wh[i] = m * wn;                                         // w^_{i+1}
                const double r0i = V.r0[i];
                d2[0] = fma(r0i, rn, d2[0]);
                d2[1] = fma(r0i, wn, d2[1]);
                d2[2] = fma(rn, rn, d2[2]);
            }
            ++spmvs;
        } else {
            PBCG_ROWS(i) { x[i] = fma(omega, mi[i] * V.q[i], fma(alpha, V.p[i], x[i])); }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const double rn = a.b[i] - A.row(i, VecLoad{x});
                V.r[i] = rn;
                rh[i] = mi[i] * rn;
            }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const double wn = A.row(i, VecLoad{rh});
                const double rn = V.r[i], r0i = V.r0[i];
                V.w[i] = wn;
                wh[i] = mi[i] * wn;
                d2[0] = fma(r0i, rn, d2[0]);
                d2[1] = fma(r0i, wn, d2[1]);
                d2[2] = fma(rn, rn, d2[2]);
            }
            spmvs += 2;
            o.nrr++;
        }
        replaced = replace_now;
        if (!grid_sum<3>(g, d2, sm, sflag)) return false;
        ++it;
        const double rho_n = d2[0], r0w = d2[1];
        o.nr = d2[2];
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[it] = d2[2];
        if (!all_finite(d2)) { o.status = PBCG_NONFINITE; break; }
        if (!fixed && norm_below(d2[2], tol, tol2)) { o.status = PBCG_OK; break; }
        if (rho_n == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        beta = beta_of(alpha, omega, rho_n, rho, sm[kMaxDots - 1]);
        double den;
        alpha_shared(rho_n, r0w, r0s, r0z, beta, omega, sm[kMaxDots - 1], den, alpha);
        if (den == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        rho = rho_n;
    }
    o.iters = it;
    if (it == a.limit && o.status == PBCG_NOT_CONVERGED && fixed) o.status = PBCG_OK;
    return true;
}

template <class Op, bool Prec>
__global__ void __launch_bounds__(kTPB, Tune<Op>::kMinBlocks) pbicgstab_kernel(const Op A, const SolveArgs a) {
    __shared__ double sm[kMaxDots][32];
    __shared__ int sflag;
    if (threadIdx.x == 0) sflag = 1;   // read only after the first exchange's barrier
    GridSync g{a.ctl, a.partials, 0u, 0};   // partials: the exchange slots
    const int lo = (int)((long long)blockIdx.x * a.n / gridDim.x);
    const int hi = (int)((long long)(blockIdx.x + 1) * a.n / gridDim.x);
    Outcome o{0, PBCG_NOT_CONVERGED, 0, 0, 0.0, 0.0};
    int spmvs = 0;
    bool ok;
    if constexpr (Prec)
        ok = pipelined_prec_loop(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    else
        ok = pipelined_loop<Op, double>(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    if (!ok) return;
    finish(A, a, g, sm, &sflag, lo, hi, o, spmvs);
}

// ===========================================================================
// Algorithm 7 (standard BiCGStab). p and s use two buffers each in variant 3:
// the phase that forms p_i for its SpMV reads p_{i-1}, s_{i-1} of neighbours
// while writing p_i, s_i, so the old and new values must not share storage.
// ===========================================================================
template <class Op, class Sync = GridSync>
__device__ __forceinline__ bool standard_loop(const Op &A, const SolveArgs &a, Sync &g, double (*sm)[32],
                                              int *sflag, int lo, int hi, Outcome &o, int &spmvs) {
    const Vectors &V = a.V;
    double *x = a.x;
    const bool fixed = a.fixed != 0;
    const bool v3 = a.variant == 3;
    // buffers: variant 3 ping-pongs p between V.p / V.z and s between V.s / V.w
    double *pA = V.p, *pB = V.z, *sA = V.s, *sB = V.w;

    // r_0 := b - A x_0; shadow r0 := r_0; p_0 := r_0 (as r + 0 (0 - 0 s))
    double d0[1] = {0.0};
    PBCG_ROWS(i) {
        const double ri = a.b[i] - A.row(i, VecLoad{x});
        V.r[i] = ri;
        V.r0[i] = ri;
        pA[i] = 0.0;
        sA[i] = 0.0;
        d0[0] = fma(ri, ri, d0[0]);
    }
    ++spmvs;
    if (!grid_sum<1>(g, d0, sm, sflag)) return false;
    double rho = d0[0];
    o.nr0 = sqrt(rho);
    o.nr = o.nr0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[0] = o.nr0;
    const double tol = __dmul_rn(a.rtol, o.nr0), tol2 = __dmul_rn(tol, tol);
    if (o.nr0 == 0.0) { o.status = PBCG_OK; return true; }
    double beta = 0.0, omega = 0.0;

    int it = 0;
    while (it < a.limit) {
        // ---- s_i = A p_i, alpha_i = (r0, r_i) / (r0, s_i)
        double d1[1] = {0.0};
        if (v3) {
            const PLoad pl{V.r, pA, sA, beta, omega};
            PBCG_ROWS(i) {
                const double si = A.row(i, pl);
                pB[i] = pl(i);
                sB[i] = si;
                d1[0] = fma(V.r0[i], si, d1[0]);
            }
        } else {
            PBCG_ROWS(i) { pA[i] = fma(beta, fma(-omega, sA[i], pA[i]), V.r[i]); }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const double si = A.row(i, VecLoad{pA});
                sA[i] = si;
                d1[0] = fma(V.r0[i], si, d1[0]);
            }
        }
        ++spmvs;
        double *pc = v3 ? pB : pA, *sc = v3 ? sB : sA;   // p_i, s_i
        if (!grid_sum<1>(g, d1, sm, sflag)) return false;
        if (!isfinite(d1[0])) { o.status = PBCG_NONFINITE; break; }
        if (d1[0] == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        const double alpha = div_shared(rho, d1[0], scalar_warp(2), &sm[kMaxDots - 1][3]);

        // ---- q_i = r_i - alpha s_i; y_i = A q_i; omega_i
        double d2[3] = {0.0, 0.0, 0.0};   // (q,y) (y,y) (q,q)
        if (v3) {
            const QLoad ql{V.r, sc, alpha};
            PBCG_ROWS(i) {
                const double yi = A.row(i, ql);
                const double qi = ql(i);
                V.q[i] = qi;
                V.y[i] = yi;
                d2[0] = fma(qi, yi, d2[0]);
                d2[1] = fma(yi, yi, d2[1]);
                d2[2] = fma(qi, qi, d2[2]);
            }
        } else {
            PBCG_ROWS(i) { V.q[i] = fma(-alpha, sc[i], V.r[i]); }
            if (!grid_sync(g, sm, sflag)) return false;
            PBCG_ROWS(i) {
                const double yi = A.row(i, VecLoad{V.q});
                const double qi = V.q[i];
                V.y[i] = yi;
                d2[0] = fma(qi, yi, d2[0]);
                d2[1] = fma(yi, yi, d2[1]);
                d2[2] = fma(qi, qi, d2[2]);
            }
        }
        ++spmvs;
        if (!grid_sum<3>(g, d2, sm, sflag)) return false;
        const double qy = d2[0], yy = d2[1], qq = d2[2];
        if (!all_finite(d2)) { o.status = PBCG_NONFINITE; break; }
        const bool small_q = !fixed && norm_below(qq, tol, tol2);
        if (small_q || yy == 0.0) {
            if (!small_q && qq != 0.0) { o.status = PBCG_BREAKDOWN; break; }
            PBCG_ROWS(i) { x[i] = fma(alpha, pc[i], x[i]); }
            if (!grid_sync(g, sm, sflag)) return false;
            ++it;
            o.nr = qq;
            o.half = 1;
            o.status = PBCG_OK;
            if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[it] = qq;
            break;
        }
        omega = div_shared(qy, yy, scalar_warp(3), &sm[kMaxDots - 1][4]);
        if (omega == 0.0) { o.status = PBCG_BREAKDOWN; break; }

        // ---- x_{i+1}, r_{i+1}; beta_i
        double d3[2] = {0.0, 0.0};   // (r0,r) (r,r)
        PBCG_ROWS(i) {
            const double qi = V.q[i];
            x[i] = fma(omega, qi, fma(alpha, pc[i], x[i]));
            const double rn = fma(-omega, V.y[i], qi);
            V.r[i] = rn;
            d3[0] = fma(V.r0[i], rn, d3[0]);
            d3[1] = fma(rn, rn, d3[1]);
        }
        if (!grid_sum<2>(g, d3, sm, sflag)) return false;
        ++it;
        const double rho_n = d3[0];
        o.nr = d3[1];
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[it] = d3[1];
        if (!all_finite(d3)) { o.status = PBCG_NONFINITE; break; }
        if (!fixed && norm_below(d3[1], tol, tol2)) { o.status = PBCG_OK; break; }
        if (rho_n == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        beta = beta_of(alpha, omega, rho_n, rho, sm[kMaxDots - 1]);
        rho = rho_n;
        if (v3) {
            double *tp = pA; pA = pB; pB = tp;
            double *ts = sA; sA = sB; sB = ts;
        }
    }
    o.iters = it;
    if (it == a.limit && o.status == PBCG_NOT_CONVERGED && fixed) o.status = PBCG_OK;
    return true;
}

// ===========================================================================
// Algorithm 10 (preconditioned BiCGStab) with a diagonal M^{-1}: the
// five-exchange form of the standard loop with p^ = M^{-1} p and
// q^ = M^{-1} q written next to p and q. Buffers: V.z holds p^, a.qh holds q^.
// ===========================================================================
template <class Op>
__device__ __forceinline__ bool standard_prec_loop(const Op &A, const SolveArgs &a, GridSync &g, double (*sm)[32],
                                                   int *sflag, int lo, int hi, Outcome &o, int &spmvs) {
    const Vectors &V = a.V;
    double *x = a.x;
    const double *mi = a.minv;
    double *ph = V.z, *qh = a.qh;
    const bool fixed = a.fixed != 0;

    double d0[1] = {0.0};
    PBCG_ROWS(i) {
        const double ri = a.b[i] - A.row(i, VecLoad{x});
        V.r[i] = ri;
        V.r0[i] = ri;
        V.p[i] = 0.0;
        V.s[i] = 0.0;
        d0[0] = fma(ri, ri, d0[0]);
    }
    ++spmvs;
    if (!grid_sum<1>(g, d0, sm, sflag)) return false;
    double rho = d0[0];
    o.nr0 = sqrt(rho);
    o.nr = o.nr0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[0] = o.nr0;
    const double tol = __dmul_rn(a.rtol, o.nr0), tol2 = __dmul_rn(tol, tol);
    if (o.nr0 == 0.0) { o.status = PBCG_OK; return true; }
    double beta = 0.0, omega = 0.0;

    int it = 0;
    while (it < a.limit) {
        // p_i := r_i + beta (p_{i-1} - omega s_{i-1}); p^_i := M^{-1} p_i; s_i := A p^_i
        PBCG_ROWS(i) {
            const double pn = fma(beta, fma(-omega, V.s[i], V.p[i]), V.r[i]);
            V.p[i] = pn;
            ph[i] = mi[i] * pn;
        }
        if (!grid_sync(g, sm, sflag)) return false;
        double d1[1] = {0.0};
        PBCG_ROWS(i) {
            const double si = A.row(i, VecLoad{ph});
            V.s[i] = si;
            d1[0] = fma(V.r0[i], si, d1[0]);
        }
        ++spmvs;
        if (!grid_sum<1>(g, d1, sm, sflag)) return false;
        if (!isfinite(d1[0])) { o.status = PBCG_NONFINITE; break; }
        if (d1[0] == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        const double alpha = __ddiv_rn(rho, d1[0]);
        // q_i := r_i - alpha s_i; q^_i := M^{-1} q_i; y_i := A q^_i
        PBCG_ROWS(i) {
            const double qi = fma(-alpha, V.s[i], V.r[i]);
            V.q[i] = qi;
            qh[i] = mi[i] * qi;
        }
        if (!grid_sync(g, sm, sflag)) return false;
        double d2[3] = {0.0, 0.0, 0.0};
        PBCG_ROWS(i) {
            const double yi = A.row(i, VecLoad{qh});
            const double qi = V.q[i];
            V.y[i] = yi;
            d2[0] = fma(qi, yi, d2[0]);
            d2[1] = fma(yi, yi, d2[1]);
            d2[2] = fma(qi, qi, d2[2]);
        }
        ++spmvs;
        if (!grid_sum<3>(g, d2, sm, sflag)) return false;
        const double qy = d2[0], yy = d2[1], qq = d2[2];
        if (!all_finite(d2)) { o.status = PBCG_NONFINITE; break; }
        const bool small_q = !fixed && norm_below(qq, tol, tol2);
        if (small_q || yy == 0.0) {
            if (!small_q && qq != 0.0) { o.status = PBCG_BREAKDOWN; break; }
            PBCG_ROWS(i) { x[i] = fma(alpha, ph[i], x[i]); }
            if (!grid_sync(g, sm, sflag)) return false;
            ++it;
            o.nr = qq;
            o.half = 1;
            o.status = PBCG_OK;
            if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[it] = qq;
            break;
        }
        omega = __ddiv_rn(qy, yy);
        if (omega == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        // x_{i+1} := x_i + alpha p^_i + omega q^_i; r_{i+1} := q_i - omega y_i
        double d3[2] = {0.0, 0.0};
        PBCG_ROWS(i) {
            x[i] = fma(omega, qh[i], fma(alpha, ph[i], x[i]));
            const double rn = fma(-omega, V.y[i], V.q[i]);
            V.r[i] = rn;
            d3[0] = fma(V.r0[i], rn, d3[0]);
            d3[1] = fma(rn, rn, d3[1]);
        }
        if (!grid_sum<2>(g, d3, sm, sflag)) return false;
        ++it;
        const double rho_n = d3[0];
        o.nr = d3[1];
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[it] = d3[1];
        if (!all_finite(d3)) { o.status = PBCG_NONFINITE; break; }
        if (!fixed && norm_below(d3[1], tol, tol2)) { o.status = PBCG_OK; break; }
        if (rho_n == 0.0) { o.status = PBCG_BREAKDOWN; break; }
        beta = beta_of(alpha, omega, rho_n, rho, sm[kMaxDots - 1]);
        rho = rho_n;
    }
    o.iters = it;
    if (it == a.limit && o.status == PBCG_NOT_CONVERGED && fixed) o.status = PBCG_OK;
    return true;
}

template <class Op, bool Prec>
__global__ void __launch_bounds__(kTPB, TunePlain<Op>::kMinBlocks) bicgstab_kernel(const Op A, const SolveArgs a) {
    __shared__ double sm[kMaxDots][32];
    __shared__ int sflag;
    if (threadIdx.x == 0) sflag = 1;   // read only after the first exchange's barrier
    GridSync g{a.ctl, a.partials, 0u, 0};   // partials: the exchange slots
    const int lo = (int)((long long)blockIdx.x * a.n / gridDim.x);
    const int hi = (int)((long long)(blockIdx.x + 1) * a.n / gridDim.x);
    Outcome o{0, PBCG_NOT_CONVERGED, 0, 0, 0.0, 0.0};
    int spmvs = 0;
    bool ok;
    if constexpr (Prec)
        ok = standard_prec_loop(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    else
        ok = standard_loop(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    if (!ok) return;
    finish(A, a, g, sm, &sflag, lo, hi, o, spmvs);
}

// ===========================================================================
// Mixed precision: FP64 iterative refinement around an FP32 pipelined solve.
// Each refinement step computes the true residual r = b - A x with the FP64
// matrix and FP64 vectors, rounds it to float, solves A d = r with Algorithm 9
// on float vectors and the low-precision copy of A (FP32 or BF16 values; dot
// products summed per thread in compensated FP32 and across threads in FP64),
// and adds d to x in FP64. The inner solve runs without residual replacement:
// the FP64 residual of every refinement step plays that role.
//
// Refinement contracts only while the low-precision operator is close enough
// to A (roughly cond(A) times the value rounding below 1). So the loop also
// stops when `stall_steps` steps in a row fail to bring the FP64 residual
// below the best one so far, and returns the best iterate with
// PBCG_NOT_CONVERGED. A converging refinement can have an occasional step
// without progress: an inner solve capped at inner_maxit may end on one of
// BiCGStab's residual peaks. The best iterate is kept without an extra sweep: the
// sweep that adds d to x first saves x in `xbest` when x is the best so far,
// i.e. exactly when the loop is about to move away from it.
// ===========================================================================
// Default of stall_steps. Measured on the 192^3 convection-diffusion system
// (40 FP32 refinements to 1e-10: both forms, inner tolerance and cap 0.1/50
// and 0.03/150, five grids, two roundings of b): runs of up to 4 steps
// without a new best occur in converging refinements, so 6.
constexpr int kMixedStallSteps = 6;

struct MixedArgs {
    int n;
    const double *b;
    double *x;
    double *xbest;       // FP64 copy of the best iterate, written when the loop leaves it
    float *d;            // correction of the current step (inner solution)
    float *rhs;          // residual of the current step, rounded to float
    VectorsT<float> V;   // inner work vectors
    Control *ctl;
    double *partials;
    double *hist;        // nullable: true residual norm before each step, length max_outer + 1
    double *inner_hist;  // nullable: recursive residual norms of the first step's inner solve
    double rtol;
    int max_outer;
    double inner_rtol;
    int inner_maxit;
    int inner_fixed;     // > 0: every inner solve runs exactly this many iterations
    int stall_steps;     // steps in a row without a new best residual that stop the loop
};

// 9 resident blocks per SM (56 registers). The FP32 inner sweeps are bound by
// load latency; with rows in aligned pairs, 9 blocks measured fastest (192^3:
// 281 us per stencil inner iteration and 331 us CSR, against 288 / 335 at 8
// blocks and 315 / 339 at 10, where the pairs spill more).
template <class Op64, class Op32>
__global__ void __launch_bounds__(kTPB, 9) mixed_kernel(const Op64 A, const Op32 A32, const MixedArgs m) {
    __shared__ double sm[kMaxDots][32];
    __shared__ int sflag;
    __shared__ uint64_t stage_full[kStages], stage_empty[kStages];
    extern __shared__ __align__(128) char stage_buf[];   // kStageSmemBytes when the sweeps are staged
    constexpr bool kStaged = HasRow2<Op32>::value;
    if (threadIdx.x == 0) {
        sflag = 1;   // read only after the first exchange's barrier
        if (kStaged) {
            for (int k = 0; k < kStages; ++k) {
                mbar_init(&stage_full[k], 1);
                mbar_init(&stage_empty[k], kTPB);
            }
            mbar_init_fence();
        }
    }
    __syncthreads();
    Stager stager{stage_buf, stage_full, stage_empty, 0u, m.ctl};
    GridSync g{m.ctl, m.partials, 0u, 0};
    // row ranges start on multiples of 4 rows: the FP32 sweeps access rows in
    // aligned pairs, and the staged ones copy 16-byte aligned tiles
    const long long quads = (m.n + 3) / 4;
    const int lo = (int)(4 * ((long long)blockIdx.x * quads / gridDim.x));
    const int hi_quad = (int)(4 * ((long long)(blockIdx.x + 1) * quads / gridDim.x));
    const int hi = hi_quad < m.n ? hi_quad : m.n;
    int outer = 0, inner_total = 0, status = PBCG_NOT_CONVERGED, spmvs = 0, stalls = 0;
    double nr0 = 0.0, tol = 0.0, tol2 = 0.0, last = 0.0;
    double best = 0.0;        // smallest squared FP64 residual so far (valid when have_best)
    bool have_best = false;
    bool at_best = false;     // x is the best iterate so far
    for (;;) {
        if (outer > 0) {
            const bool save = at_best;   // the same in every block
            PBCG_ROWS(i) {
                const double xi = m.x[i];
                if (save) m.xbest[i] = xi;
                m.x[i] = xi + (double)m.d[i];
            }
            if (!grid_sync(g, sm, &sflag)) return;
        }
        double d[1] = {0.0};
        PBCG_ROWS(i) {
            const double r = m.b[i] - A.row(i, VecLoad{m.x});
            m.rhs[i] = (float)r;
            m.d[i] = 0.0f;
            d[0] = fma(r, r, d[0]);
        }
        ++spmvs;
        if (!grid_sum<1>(g, d, sm, &sflag)) return;
        last = d[0];
        if (outer == 0) {
            nr0 = sqrt(d[0]);
            tol = __dmul_rn(m.rtol, nr0);
            tol2 = __dmul_rn(tol, tol);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && m.hist) m.hist[outer] = d[0];
        if (!isfinite(d[0])) { at_best = false; status = PBCG_NONFINITE; break; }
        if (nr0 == 0.0 || norm_below(d[0], tol, tol2)) { at_best = true; status = PBCG_OK; break; }
        if (!have_best || d[0] < best) {
            best = d[0];
            have_best = true;
            at_best = true;
            stalls = 0;
        } else {
            at_best = false;
            if (++stalls >= m.stall_steps) break;   // refinement does not contract
        }
        if (outer >= m.max_outer) break;
        SolveArgsT<float> ia;
        ia.n = m.n;
        ia.b = m.rhs;
        ia.x = m.d;
        ia.V = m.V;
        ia.ctl = m.ctl;
        ia.partials = m.partials;
        ia.hist = outer == 0 ? m.inner_hist : nullptr;
        ia.rtol = m.inner_rtol;
        ia.limit = m.inner_fixed > 0 ? m.inner_fixed : m.inner_maxit;
        ia.fixed = m.inner_fixed > 0 ? 1 : 0;
        ia.replace_period = 0;
        ia.max_repl = -1;
        ia.variant = 0;
        Outcome io{0, PBCG_NOT_CONVERGED, 0, 0, 0.0, 0.0};
        if (!pipelined_loop<Op32, float>(A32, ia, g, sm, &sflag, lo, hi, io, spmvs, kStaged ? &stager : nullptr))
            return;
        // the inner history holds squared norms after entry 0 (thread 0 of block 0 wrote them)
        if (blockIdx.x == 0 && threadIdx.x == 0 && ia.hist)
            for (int i = 1; i <= io.iters; ++i) ia.hist[i] = sqrt(ia.hist[i]);
        inner_total += io.iters;
        ++outer;
        if (io.status == PBCG_NONFINITE) { status = PBCG_NONFINITE; break; }
    }
    // A solve that stops unconverged returns the best iterate: x := xbest when x is not it.
    const bool restore = status != PBCG_OK && have_best && !at_best;
    if (restore) {
        PBCG_ROWS(i) { m.x[i] = m.xbest[i]; }
        last = best;
    }
    if (blockIdx.x == 0) {
        if (m.hist)
            for (int i = (int)threadIdx.x; i <= outer; i += kTPB) m.hist[i] = sqrt(m.hist[i]);
        if (threadIdx.x == 0) {
            Control *c = m.ctl;
            c->iters = outer;
            c->inner_iters = inner_total;
            c->status = status;
            c->grid_syncs = g.count;
            c->spmvs = spmvs;
            c->nr0 = nr0;
            c->rel_true = nr0 > 0.0 ? sqrt(last) / nr0 : sqrt(last);
            c->rel_rec = c->rel_true;
            c->half_step = restore ? 1 : 0;   // mixed solves: 1 if x was reset to the best iterate
        }
    }
}

// ===========================================================================
// Single small systems on one thread-block cluster. A cooperative grid pays a
// round trip through L2 and an arrival counter per exchange (several us at a
// few thousand unknowns); the CTAs of one cluster instead cross the hardware
// cluster barrier and exchange their block sums through distributed shared
// memory (ClusterSync). The solver loops are the same code as on the grid.
// Rows are split into `size` contiguous ranges, one per CTA; CTA rank 0
// writes the result record. Every CTA takes the same branches (identical
// scalars), so all of them execute the same sequence of cluster barriers.
// ===========================================================================
template <class Op, bool Pipelined>
__global__ void __launch_bounds__(kTPB, 1) cluster_solve_kernel(const Op A, const SolveArgs a) {
    __shared__ double sm[kMaxDots][32];
    __shared__ double slots[2][kMaxCluster][kSlotDoubles];
    __shared__ int sflag;
    const unsigned size = cluster_ctas(), rank = cluster_rank();
    if (threadIdx.x == 0) sflag = 1;
    cluster_barrier();   // every CTA started before its shared memory is written by the others
    ClusterSync g{slots, rank, size, 0u, 0};
    const int lo = (int)((long long)rank * a.n / size);
    const int hi = (int)((long long)(rank + 1) * a.n / size);
    Outcome o{0, PBCG_NOT_CONVERGED, 0, 0, 0.0, 0.0};
    int spmvs = 0;
    if constexpr (Pipelined)
        pipelined_loop<Op, double, ClusterSync>(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    else
        standard_loop<Op, ClusterSync>(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    finish(A, a, g, sm, &sflag, lo, hi, o, spmvs);
    cluster_barrier();   // no CTA leaves while another may still address its shared memory
}

// M^{-1} = 1 / diag(A) (Jacobi). A zero or non-finite diagonal entry sets *bad.
__global__ void jacobi_csr_kernel(int n, const int *rowptr, const int *col, const double *val, double *minv, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] == i) d = val[k];
        const double m = 1.0 / d;
        if (d == 0.0 || !isfinite(m)) atomicOr(bad, 1);
        minv[i] = m;
    }
}
__global__ void jacobi_stencil_kernel(const StencilOp A, double *minv, int *bad) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < A.n; r += gridDim.x * blockDim.x) {
        const int t = (int)A.dx.div((uint32_t)r);
        const int i = r - t * A.nx;
        const int k = (int)A.dy.div((uint32_t)t);
        const int j = t - k * A.ny;
        const double d = A.coef(PBCG_C, i, j, k);
        const double m = 1.0 / d;
        if (d == 0.0 || !isfinite(m)) atomicOr(bad, 1);
        minv[r] = m;
    }
}

// ===========================================================================
// Batched solves: many independent systems in one launch. The launch is made
// of thread-block clusters of `size` CTAs (size 1: plain blocks). The first
// CTA of a cluster takes the next system from an atomic counter; a system with
// at least `cluster_min_rows` rows is solved by the whole cluster (rows split
// into `size` contiguous ranges, reductions through distributed shared memory
// and the hardware cluster barrier, ClusterSync); otherwise the first CTA
// takes `size` - 1 further systems and every CTA solves one alone (block-level
// reductions and barriers, BlockSync). Clusters never wait on each other, so
// no co-residency beyond the cluster is needed and the launch can be captured
// in a CUDA graph. System s owns the global rows [row_offset[s],
// row_offset[s+1]) of the concatenated CSR arrays (row pointers index the
// shared col/val arrays; column indices are local to the system) and of b, x
// and the work vectors. Systems are taken in index order; ordering them
// largest first balances the load.
// ===========================================================================
struct BatchArgs {
    int nsys;
    int nnz;
    long long total_rows;
    const long long *row_offset;   // [nsys + 1]
    const int *rowptr;             // [total rows + 1], global offsets into col/val
    const int *col;                // local column indices
    const double *val;
    const double *b;
    double *x;
    Vectors V;                     // global work vectors (total rows each)
    unsigned *next;                // work counter, zero before the launch
    pbcg_batch_result *out;        // [nsys]
    double rtol;
    int maxit;
    int replace_period;
    long long cluster_min_rows;    // systems this large are solved by a whole cluster
    int fixed;                     // > 0: every system runs exactly this many iterations
    double *hist;                  // nullable: ||r_i|| of system s at hist[s * hist_stride + i]
    long long hist_stride;
};

// Solve system `sys` on rows [lo, hi) of it (the whole system for BlockSync,
// this CTA's share for ClusterSync); the first CTA writes the result.
template <class Sync>
__device__ __forceinline__ void batched_system(const BatchArgs &B, int sys, Sync &g, unsigned part, unsigned parts,
                                               double (*sm)[32], int *sflag) {
    const long long r0 = B.row_offset[sys], r1 = B.row_offset[sys + 1];
    // structure check of this system: its rows inside the batch, entries inside
    // the shared arrays, columns local to the system (each CTA checks its rows)
    int bad = (r0 < 0 || r1 < r0 || r1 > B.total_rows || r1 - r0 >= (1ll << 31)) ? 1 : 0;
    const int n = bad ? 0 : (int)(r1 - r0);
    const int lo = (int)((long long)part * n / parts), hi = (int)((long long)(part + 1) * n / parts);
    const CsrOpGatherL2 A{{n, B.rowptr + (bad ? 0 : r0), B.col, B.val, B.nnz}};
    PBCG_ROWS(i) {
        const int e0 = A.rowptr[i], e1 = A.rowptr[i + 1];
        if (e0 < 0 || e1 < e0 || e1 > B.nnz) { bad = 1; continue; }
        for (int k = e0; k < e1 && !bad; ++k)
            if (B.col[k] < 0 || B.col[k] >= n) bad = 1;
    }
    double fb[1] = {(double)bad};
    grid_sum<1>(g, fb, sm, sflag);
    pbcg_batch_result res{0, PBCG_ERR_ARG, 0, 0, 0.0, 0.0};
    if (fb[0] == 0.0) {
        SolveArgs a;
        a.n = n;
        a.b = B.b + r0;
        a.x = B.x + r0;
        a.V = Vectors{B.V.r + r0, B.V.r0 + r0, B.V.p + r0, B.V.s + r0, B.V.z + r0,
                      B.V.q + r0, B.V.y + r0, B.V.w + r0, B.V.t + r0, B.V.v + r0};
        a.ctl = nullptr;
        a.partials = nullptr;
        a.hist = B.hist ? B.hist + (size_t)sys * (size_t)B.hist_stride : nullptr;
        a.rtol = B.rtol;
        a.limit = B.fixed > 0 ? B.fixed : B.maxit;
        a.fixed = B.fixed > 0 ? 1 : 0;
        a.replace_period = B.replace_period;
        a.max_repl = -1;
        a.variant = 0;
        a.minv = nullptr;
        a.rh = a.sh = a.zh = a.qh = a.wh = nullptr;
        Outcome o{0, PBCG_NOT_CONVERGED, 0, 0, 0.0, 0.0};
        int spmvs = 0;
        pipelined_loop<CsrOpGatherL2, double, Sync>(A, a, g, sm, sflag, lo, hi, o, spmvs);
        // the history holds squared norms after entry 0 (written by this thread)
        if (a.hist && part == 0 && threadIdx.x == 0)
            for (int i = 1; i <= o.iters; ++i) a.hist[i] = sqrt(a.hist[i]);
        // true residual of the returned x
        double d[1] = {0.0};
        PBCG_ROWS(i) {
            const double rr = a.b[i] - A.row(i, VecLoad{a.x});
            d[0] = fma(rr, rr, d[0]);
        }
        grid_sum<1>(g, d, sm, sflag);
        res.iters = o.iters;
        res.status = o.status;
        res.half_step = o.half;
        res.n_replacements = o.nrr;
        const double nr = o.iters > 0 ? sqrt(o.nr) : o.nr0;
        res.rel_res_recursive = o.nr0 > 0.0 ? nr / o.nr0 : 0.0;
        res.rel_res_true = o.nr0 > 0.0 ? sqrt(d[0]) / o.nr0 : sqrt(d[0]);
    }
    if (part == 0 && threadIdx.x == 0) B.out[sys] = res;
}

__global__ void __launch_bounds__(kTPB, 6) batched_kernel(const BatchArgs B) {
    __shared__ double sm[kMaxDots][32];
    __shared__ double slots[2][kMaxCluster][kSlotDoubles];   // cluster reductions: every CTA's block sums
    __shared__ int item[2];   // system of this CTA (-1: none), whole-cluster flag (-1: no work left)
    __shared__ int sflag;
    const unsigned size = cluster_ctas(), rank = cluster_rank();
    if (size > 1) cluster_barrier();   // every CTA started before its shared memory is addressed
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int s = (int)atomicAdd(B.next, 1u);
            int whole = 0;
            if (s >= B.nsys) {
                whole = -1;
            } else if (size > 1) {
                const long long rows = B.row_offset[s + 1] - B.row_offset[s];
                whole = rows >= B.cluster_min_rows ? 1 : 0;
            }
            int extra = 0;
            if (whole == 0 && size > 1) extra = (int)atomicAdd(B.next, size - 1);
            for (unsigned r = 0; r < size; ++r) {
                int mine = s;
                if (whole == -1) mine = -1;
                else if (whole == 0 && r > 0) mine = extra + (int)r - 1 < B.nsys ? extra + (int)r - 1 : -1;
                if (size > 1) {
                    st_cluster_s32(cluster_map(&item[0], r), mine);
                    st_cluster_s32(cluster_map(&item[1], r), whole);
                } else {
                    item[0] = mine;
                    item[1] = whole;
                }
            }
        }
        if (size > 1) cluster_barrier();
        else __syncthreads();
        const int sys = item[0], whole = item[1];
        if (whole < 0) return;   // the same for every CTA of the cluster
        if (whole == 1) {
            ClusterSync g{slots, rank, size, 0u, 0};
            batched_system(B, sys, g, rank, size, sm, &sflag);
        } else if (sys >= 0) {
            BlockSync g{0};
            batched_system(B, sys, g, 0u, 1u, sm, &sflag);
        }
        // every CTA is done with this item (and with the slots) before the next claim
        if (size > 1) cluster_barrier();
        else __syncthreads();
    }
}

// Diagnostic of the bounded grid-wide wait: every block but the last enters a
// grid synchronisation that the last block never joins, so the wait cannot
// complete and must end at its limit. The first block to give up records
// PBCG_ERR_TIMEOUT in the abort flag; the others see the flag (or their own
// limit) and return. Block 0 then reports the flag.
__global__ void sync_timeout_probe_kernel(Control *ctl, double *slots, uint64_t limit_ns) {
    __shared__ double sm[kMaxDots][32];
    __shared__ int sflag;
    if (blockIdx.x == gridDim.x - 1) return;
    if (threadIdx.x == 0) sflag = 1;
    GridSync g{ctl, slots, 0u, 0, limit_ns};
    const bool ok = grid_sync(g, sm, &sflag);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->status = ok ? (int)PBCG_OK : ld_relaxed_s32(&ctl->abort);
}

// out[k] = (float)in[k], k < len (FP32 copies of stencil coefficient tables).
__global__ void to_float_kernel(const double *in, float *out, long long len) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len; k += (long long)gridDim.x * blockDim.x)
        out[k] = (float)in[k];
}

// y = A x, one row per thread, grid-stride.
template <class Op>
__global__ void __launch_bounds__(kTPB) spmv_kernel(const Op A, const double *x, double *y) {
    const VecLoad u{x};
    for (int i = blockIdx.x * kTPB + threadIdx.x; i < A.n; i += gridDim.x * kTPB) y[i] = A.row(i, u);
}

// CSR structure check: rowptr[0] == 0, non-decreasing, rowptr[n] == nnz, 0 <= col < n.
__global__ void csr_check_kernel(int n, int nnz, const int *rowptr, const int *col, int *bad) {
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
        const int a = rowptr[i];
        if (i == 0 && a != 0) atomicOr(bad, 1);
        if (i == n && a != nnz) atomicOr(bad, 2);
        if (i < n && rowptr[i + 1] < a) atomicOr(bad, 4);
        if (a < 0 || a > nnz) atomicOr(bad, 8);
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const int c = col[k];
        if (c < 0 || c >= n) atomicOr(bad, 16);
    }
}

#undef PBCG_ROWS

}  // namespace pbcg
