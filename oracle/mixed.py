"""Mixed-precision oracle -- test infrastructure only.

FP64 iterative refinement around pipelined BiCGStab (Algorithm 9) run in a
lower precision: each step computes r = b - A x in FP64 (the C oracle's SpMV),
solves A d = fl(r) with Algorithm 9 on vectors of the working type (float32 by
default) and the matrix values in that type, SpMV in that type (scipy.sparse),
but dot products accumulated in float64, then sets x := x + d in FP64.
Written with numpy vector operations in the order of Algorithm 9; the only
library primitives are the SpMV and the dot product.

``pbicgstab_lowp`` is generic in the working type: run in float64 it is plain
Algorithm 9 and is pinned against the C oracle's Algorithm 9 (its residual
history agrees to rounding), which ties this code to the algorithm before it
is trusted in float32.

Reading for the refinement's stopping rule (the paper has no mixed-precision
passage): refinement contracts only while the low-precision operator is close
enough to A, so it also stops when ``stall_limit`` steps in a row fail to bring
the FP64 residual below the best one so far, and returns the best iterate.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import oracle

f32 = np.float32


def dot64(a, b):
    """Dot product accumulated in float64 (float32 products are exact in float64)."""
    return float(np.dot(a.astype(np.float64), b.astype(np.float64)))


def pbicgstab_lowp(A_lp, b_lp, rtol, maxit, fixed_iters=0):
    """Algorithm 9 (no residual replacement) from x0 = 0 on vectors of b_lp's
    dtype and the sparse matrix A_lp of the same dtype. The scalars alpha, beta,
    omega, rho are float64, rounded to the working type where a vector update
    uses them; dot products are accumulated in float64.

    fixed_iters > 0 runs exactly that many iterations (no stopping test).
    Returns (x, iterations, history) with history[i] = ||r_i||_2 (recursive
    residual) for i = 0..iterations (the last entry is ||q|| after a half step).
    """
    dt = b_lp.dtype.type
    n = b_lp.size
    limit = fixed_iters if fixed_iters > 0 else maxit
    fixed = fixed_iters > 0
    x = np.zeros(n, dtype=dt)
    r = b_lp.copy()                      # b - A 0
    r0 = r.copy()
    w = A_lp @ r
    t = A_lp @ w
    p = np.zeros(n, dtype=dt); s = p.copy(); z = p.copy(); v = p.copy()
    rho = dot64(r0, r)
    nr0 = np.sqrt(rho)
    hist = [nr0]
    if nr0 == 0.0:
        return x, 0, np.array(hist)
    r0w = dot64(r0, w)
    if r0w == 0.0:
        return x, 0, np.array(hist)
    alpha, beta, omega = rho / r0w, 0.0, 0.0
    for i in range(limit):
        al, be, om = dt(alpha), dt(beta), dt(omega)
        p = r + be * (p - om * s)
        s = w + be * (s - om * z)
        z = t + be * (z - om * v)
        q = r - al * s
        y = w - al * z
        qy, yy, qq = dot64(q, y), dot64(y, y), dot64(q, q)
        v = A_lp @ z
        if (not fixed and np.sqrt(qq) <= rtol * nr0) or yy == 0.0:
            x = x + al * p
            hist.append(np.sqrt(qq))
            return x, i + 1, np.array(hist)
        omega = qy / yy
        om = dt(omega)
        x = x + al * p + om * q
        r = q - om * y
        w = y - om * (t - al * v)
        rho_n, r0w, r0s, r0z = dot64(r0, r), dot64(r0, w), dot64(r0, s), dot64(r0, z)
        t = A_lp @ w
        hist.append(np.sqrt(dot64(r, r)))
        if (not fixed and hist[-1] <= rtol * nr0) or rho_n == 0.0:
            return x, i + 1, np.array(hist)
        beta = (alpha / omega) * (rho_n / rho)
        alpha = rho_n / (r0w + beta * r0s - beta * omega * r0z)
        rho = rho_n
    return x, limit, np.array(hist)


def pbicgstab_f32(A32, b32, rtol, maxit):
    """Algorithm 9 on float32 vectors from x0 = 0; returns (x, iterations)."""
    x, its, _ = pbicgstab_lowp(A32, b32, rtol, maxit)
    return x, its


def refine(A, b, rtol=1e-10, max_outer=20, inner_rtol=1e-4, inner_maxit=1000, values32=None, inner_fixed=0,
           stall_limit=6):
    """FP64 iterative refinement with FP32 inner Algorithm 9. ``values32``: the
    float32 values of A's CSR structure (default: A's values rounded).
    inner_fixed > 0: every inner solve runs exactly that many iterations.
    Stops at the tolerance (status CONVERGED), after max_outer steps, or when
    stall_limit steps in a row do not reduce the FP64 residual below the best
    so far (both NOT_CONVERGED, returning the best iterate).
    Returns dict(x, outer, inner_iters, rel_res_true, history, status,
    restored, inner_history) -- history: the FP64 residual norm before each
    step; inner_history: the first inner solve's residual norms."""
    vals = A.val.astype(f32) if values32 is None else np.asarray(values32, dtype=f32)
    A32 = sp.csr_matrix((vals, A.col, A.rowptr), shape=(A.n, A.n))
    x = np.zeros(A.n)
    hist = []
    inner_total = 0
    nr0 = None
    best, x_best, stalls = None, None, 0
    status = oracle.NOT_CONVERGED
    inner_hist = None
    outer = 0
    while True:
        r = b - oracle.spmv(A, x)
        nr = np.linalg.norm(r)
        if nr0 is None:
            nr0 = nr
        hist.append(nr)
        if not np.isfinite(nr):
            status = oracle.NONFINITE
            break
        if nr0 == 0.0 or nr <= rtol * nr0:
            status = oracle.CONVERGED
            x_best, best = x, nr
            break
        if best is None or nr < best:
            best, x_best, stalls = nr, x, 0
        else:
            stalls += 1
            if stalls >= stall_limit:
                break
        if outer == max_outer:
            break
        d, its, ih = pbicgstab_lowp(A32, r.astype(f32), inner_rtol, inner_maxit, fixed_iters=inner_fixed)
        if inner_hist is None:
            inner_hist = ih
        inner_total += its
        x = x + d.astype(np.float64)
        outer += 1
    restored = status != oracle.CONVERGED and x_best is not None and x_best is not x
    if restored:
        x = x_best
    final = best if restored else hist[-1]
    return dict(x=x, outer=outer, inner_iters=inner_total, rel_res_true=final / nr0, history=np.array(hist),
                status=status, restored=restored, inner_history=inner_hist)
