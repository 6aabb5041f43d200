// The sparse operators A of A x = b: CSR and 5/7-point stencil.
//
// Each operator computes one row of a product, (A u)_row = sum_j a_{row,j} u_j,
// where u_j is produced by a loader functor. The plain loader reads a vector;
// other loaders form a vector on the fly (e.g. p = r + beta (p - omega s) for
// neighbours), which lets a solver phase fuse an AXPY into its SpMV.
//
// Summation order of a row: its stored entries in order (CSR); B, S, W, C, E,
// N, T (stencil) -- ascending column index, so a stencil and its sorted CSR
// assembly give bitwise identical rows. Products are accumulated with FMA.
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"

namespace pbcg {

// fma for the arithmetic type of a sweep (FP64 path, or FP32 inner solves).
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// A stored matrix value as the arithmetic type T of a sweep.
template <typename T>
__device__ __forceinline__ T value_as(double v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T value_as(float v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T value_as(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

// u_j = x[j]
template <typename T>
struct VecLoadT {
    const T *x;
    __device__ __forceinline__ T operator()(int j) const { return x[j]; }
};
using VecLoad = VecLoadT<double>;

// u_j = r_j + beta (p_j - omega s_j): the p-recurrence of Algorithm 7
struct PLoad {
    const double *r, *p, *s;
    double beta, omega;
    __device__ __forceinline__ double operator()(int j) const { return fma(beta, fma(-omega, s[j], p[j]), r[j]); }
};

// u_j = r_j - alpha s_j: q of Algorithm 7
struct QLoad {
    const double *r, *s;
    double alpha;
    __device__ __forceinline__ double operator()(int j) const { return fma(-alpha, s[j], r[j]); }
};

// CSR with values stored as V (double; float or bfloat16 for low-precision
// inner solves). A row is accumulated in the loader's type, in storage order.
// kChunk > 1 takes a row's entries kChunk at a time: all column indices and
// values of a chunk in flight together, then all gathers, then the FMAs in
// storage order (the same sum as the one-by-one loop). The entries missing
// from a row's last chunk are predicated off. kChunk = 1 is the plain loop.
// Which one pays was measured per matrix class (time per iteration, both
// methods, FP64):
// * 7-point rows (256^3): 7 at a time 5.5 % (Algorithm 9) and 6 % (Algorithm
//   7) faster than one at a time; 8 at a time spilled registers and gained
//   half as much, 4 at a time lost. Taking only whole chunks and the rest one
//   at a time lost 10 %: warps holding a boundary row ran both paths.
// * Random rows of 9-33 entries (2^20 rows): 7 at a time 4-5 % faster.
// * 5-point rows (1024^2): one at a time fastest; 5 at a time 4 % and 7 at a
//   time 3-9 % slower. A predicated-off FP64 FMA occupies the FP64 pipe like
//   a live one, and 2 of every 7 were dead.
// The library therefore uses 7 at a time for matrices averaging more than 6
// entries per row and the plain loop otherwise. FP32 and BF16 values (the
// inner solves) take 8 at a time (4 and 6 measured slower); the batched
// solver keeps the plain loop (its rows gained nothing from chunks), with
// its gathers through L2 only (CsrOpGatherL2).
template <typename V, int kChunk = 8>
struct CsrOpT {
    int n;
    const int *__restrict__ rowptr;
    const int *__restrict__ col;
    const V *__restrict__ val;
    int nnz;   // entries readable at col and val (the bounds of a checked build)

    template <class L>
    __device__ __forceinline__ auto row(int r, const L &u) const -> decltype(u(0)) {
        using T = decltype(u(0));
        const int b = __ldg(rowptr + PBCG_SAFE(r, n)), e = __ldg(rowptr + PBCG_SAFE(r, n) + 1);
        T acc = T(0);
        if constexpr (kChunk <= 1) {
            for (int k = b; k < e; ++k) {
                const int kk = PBCG_SAFE(k, nnz);
                acc = fmaT(value_as<T>(__ldg(val + kk)), u(PBCG_SAFE(__ldg(col + kk), n)), acc);
            }
        } else {
            for (int k0 = b; k0 < e; k0 += kChunk) {
                int c[kChunk] = {};
                V v[kChunk] = {};
                T xv[kChunk] = {};
#pragma unroll
                for (int j = 0; j < kChunk; ++j)
                    if (k0 + j < e) {
                        const int kk = PBCG_SAFE(k0 + j, nnz);
                        c[j] = __ldg(col + kk);
                        v[j] = __ldg(val + kk);
                    }
#pragma unroll
                for (int j = 0; j < kChunk; ++j)
                    if (k0 + j < e) xv[j] = u(PBCG_SAFE(c[j], n));
#pragma unroll
                for (int j = 0; j < kChunk; ++j)
                    if (k0 + j < e) acc = fmaT(value_as<T>(v[j]), xv[j], acc);
            }
        }
        return acc;
    }
};
using CsrOpScalar = CsrOpT<double, 1>;    // one entry at a time
using CsrOpChunked = CsrOpT<double, 7>;   // 7 entries at a time

// A loader whose vector reads bypass L1 (ld.global.cg: cached in L2 only).
template <class L>
struct L2Gather {
    L u;
    __device__ __forceinline__ auto operator()(int j) const -> decltype(u(0)) { return u(j); }
};
template <typename T>
struct L2Gather<VecLoadT<T>> {
    VecLoadT<T> u;
    __device__ __forceinline__ T operator()(int j) const { return __ldcg(u.x + j); }
};

// The batched solver's CSR operator (random systems, 9-33 entries a row with
// uniformly random columns). Each lane streams its own row's column indices
// and values, and a sector of them serves 4 to 8 consecutive entries if it
// stays in L1 that long. So everything else bypasses L1 (ld.global.cg, cached
// in L2 only): the SpMV's gathers, and the fused sweeps' vector loads, which
// are used once (SweepLoadsL2). On the 512-system batch, the gathers alone
// took 52.4 against 55.1 ms, the gathers and sweep loads 50.6 against 52.8
// ms; an evict_last priority on the row streams' loads changed nothing
// (52.4 ms). The results are bit for bit the same.
struct CsrOpGatherL2 : CsrOpScalar {
    template <class L>
    __device__ __forceinline__ auto row(int r, const L &u) const -> decltype(u(0)) {
        return CsrOpScalar::row(r, L2Gather<L>{u});
    }
};
// Rows averaging more than this many entries take the chunked operator.
constexpr long long kChunkedMinAvgRow = 6;

// One coefficient: t1[i*a1 + j*b1 + k*c1] (or `value` when t1 is null) plus
// t2[i*a2 + j*b2 + k*c2] when t2 is set (n2 = 1, else 0). Indices fit 31 bits
// (checked at create). C is the type of the tables: double, or float for the
// low-precision inner solves (tables rounded to FP32 by the library).
template <typename C>
struct StCoefT {
    const C *t1, *t2;
    int a1, b1, c1, a2, b2, c2;
    int n2;
    C value;
    int len1, len2;   // elements readable at t1 and t2 (the bounds of a checked build)
};
using StCoef = StCoefT<double>;

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

template <typename C>
struct StencilOpT {
    int n, nx, ny, nz;
    int nxy;
    FastDiv dx, dy;
    StCoefT<C> c[7];   // C, W, E, S, N, B, T

    __device__ __forceinline__ C coef(int d, int i, int j, int k) const {
        const StCoefT<C> &q = c[d];
        C v = q.t1 ? __ldg(q.t1 + PBCG_SAFE(i * q.a1 + j * q.b1 + k * q.c1, q.len1)) : q.value;
        // The second table is rare (a coefficient varying along two separate
        // directions), and its addition is written as a loop of n2 (0 or 1)
        // trips so that the compiler jumps over it rather than predicating it:
        // a DADD whose lanes are all predicated off still occupies the FP64
        // pipe for a whole warp instruction (64 cycles per sub-partition on
        // this GPU), which as an if-converted branch cost 6 dead DADDs per row
        // of a 7-point stencil with one summed coefficient.
#pragma unroll 1
        for (int m = 0; m < q.n2; ++m) v = add_rn(v, __ldg(q.t2 + PBCG_SAFE(i * q.a2 + j * q.b2 + k * q.c2, q.len2)));
        return v;
    }

    template <class L>
    __device__ __forceinline__ auto row(int r, const L &u) const -> decltype(u(0)) {
        using T = decltype(u(0));
        const int t = (int)dx.div((uint32_t)r);
        const int i = r - t * nx;
        const int k = (int)dy.div((uint32_t)t);
        const int j = t - k * ny;
        T acc = T(0);
        if (k > 0) acc = fmaT((T)coef(PBCG_B, i, j, k), u(PBCG_SAFE(r - nxy, n)), acc);
        if (j > 0) acc = fmaT((T)coef(PBCG_S, i, j, k), u(PBCG_SAFE(r - nx, n)), acc);
        if (i > 0) acc = fmaT((T)coef(PBCG_W, i, j, k), u(PBCG_SAFE(r - 1, n)), acc);
        acc = fmaT((T)coef(PBCG_C, i, j, k), u(PBCG_SAFE(r, n)), acc);
        if (i < nx - 1) acc = fmaT((T)coef(PBCG_E, i, j, k), u(PBCG_SAFE(r + 1, n)), acc);
        if (j < ny - 1) acc = fmaT((T)coef(PBCG_N, i, j, k), u(PBCG_SAFE(r + nx, n)), acc);
        if (k < nz - 1) acc = fmaT((T)coef(PBCG_T, i, j, k), u(PBCG_SAFE(r + nxy, n)), acc);
        return acc;
    }

    // Coefficient d at the nodes (i, j, k) and (i+1, j, k): one load when the
    // table does not vary along x (stride 0), else one per node; each sum of
    // two tables formed per node as in coef().
    __device__ __forceinline__ void coef2(int d, int i, int j, int k, C &v0, C &v1) const {
        const StCoefT<C> &q = c[d];
        if (q.t1) {
            const int at = i * q.a1 + j * q.b1 + k * q.c1;
            v0 = __ldg(q.t1 + PBCG_SAFE(at, q.len1));
            v1 = q.a1 == 0 ? v0 : __ldg(q.t1 + PBCG_SAFE(at + q.a1, q.len1));
        } else {
            v0 = v1 = q.value;
        }
#pragma unroll 1
        for (int m = 0; m < q.n2; ++m) {
            const int at = i * q.a2 + j * q.b2 + k * q.c2;
            const C w0 = __ldg(q.t2 + PBCG_SAFE(at, q.len2));
            const C w1 = q.a2 == 0 ? w0 : __ldg(q.t2 + PBCG_SAFE(at + q.a2, q.len2));
            v0 = add_rn(v0, w0);
            v1 = add_rn(v1, w1);
        }
    }

    // Rows r and r+1 (r even) lie on one x-line for every even r when nx is
    // even. The sweeps use row2 only then: with odd nx some pairs span two
    // lines, and a warp holding one runs both of row2's paths.
    __device__ __forceinline__ bool pairs_on_lines() const { return (nx & 1) == 0; }

    // Rows r and r+1 (r even) of the FP32 inner sweeps, y[0] and y[1], each
    // summed exactly as row() sums it: the same products in the same order,
    // so the results are bitwise those of two row() calls. When both rows lie
    // on one x-line they share the decomposition of r, the coefficient loads
    // that do not vary along x, and their neighbour loads, taken as 64-bit
    // pairs where both values are 8-byte aligned (r even; the offsets nx and
    // nx*ny even). A pair that spans two x-lines (odd nx) takes two row()s.
    template <class T>
    __device__ __forceinline__ void row2(int r, const T *u, T (&y)[2]) const {
        static_assert(sizeof(T) == 4 && sizeof(C) == 4, "pairs of FP32 rows");
        const int t = (int)dx.div((uint32_t)r);
        const int i = r - t * nx;
        if (i + 1 >= nx) {
            const VecLoadT<T> L{u};
            y[0] = row(r, L);
            y[1] = row(r + 1, L);
            return;
        }
        const int k = (int)dy.div((uint32_t)t);
        const int j = t - k * ny;
        // u at offset o and o + 1 from r (o even when `even`)
        auto pair_at = [&](int o, bool even, T &a, T &b) {
            const int at = PBCG_SAFE(r + o, n - 1);   // both at and at + 1 in range
            if (even) {
                const float2 v = *reinterpret_cast<const float2 *>(u + at);
                a = v.x;
                b = v.y;
            } else {
                a = u[at];
                b = u[at + 1];
            }
        };
        T a0 = T(0), a1 = T(0);
        C c0, c1;
        if (k > 0) {
            T v0, v1;
            pair_at(-nxy, (nxy & 1) == 0, v0, v1);
            coef2(PBCG_B, i, j, k, c0, c1);
            a0 = fmaT((T)c0, v0, a0);
            a1 = fmaT((T)c1, v1, a1);
        }
        if (j > 0) {
            T v0, v1;
            pair_at(-nx, (nx & 1) == 0, v0, v1);
            coef2(PBCG_S, i, j, k, c0, c1);
            a0 = fmaT((T)c0, v0, a0);
            a1 = fmaT((T)c1, v1, a1);
        }
        T u0, u1;
        pair_at(0, true, u0, u1);
        coef2(PBCG_W, i, j, k, c0, c1);
        if (i > 0) a0 = fmaT((T)c0, u[PBCG_SAFE(r - 1, n)], a0);
        a1 = fmaT((T)c1, u0, a1);
        coef2(PBCG_C, i, j, k, c0, c1);
        a0 = fmaT((T)c0, u0, a0);
        a1 = fmaT((T)c1, u1, a1);
        coef2(PBCG_E, i, j, k, c0, c1);
        a0 = fmaT((T)c0, u1, a0);
        if (i + 2 < nx) a1 = fmaT((T)c1, u[PBCG_SAFE(r + 2, n)], a1);
        if (j < ny - 1) {
            T v0, v1;
            pair_at(nx, (nx & 1) == 0, v0, v1);
            coef2(PBCG_N, i, j, k, c0, c1);
            a0 = fmaT((T)c0, v0, a0);
            a1 = fmaT((T)c1, v1, a1);
        }
        if (k < nz - 1) {
            T v0, v1;
            pair_at(nxy, (nxy & 1) == 0, v0, v1);
            coef2(PBCG_T, i, j, k, c0, c1);
            a0 = fmaT((T)c0, v0, a0);
            a1 = fmaT((T)c1, v1, a1);
        }
        y[0] = a0;
        y[1] = a1;
    }
};
using StencilOp = StencilOpT<double>;

// Operators whose fused sweeps load their vectors through L2 only.
template <class Op>
struct SweepLoadsL2 {
    static constexpr bool value = false;
};
template <>
struct SweepLoadsL2<CsrOpGatherL2> {
    static constexpr bool value = true;
};

// Operators with row2 (pairs of FP32 rows).
template <class Op>
struct HasRow2 {
    static constexpr bool value = false;
};
template <>
struct HasRow2<StencilOpT<float>> {
    static constexpr bool value = true;
};

}  // namespace pbcg
