"""Mixed-precision oracle -- test infrastructure only.

FP64 iterative refinement around pipelined BiCGStab (Algorithm 9) run in
FP32: each step computes r = b - A x in FP64 (the C oracle's SpMV), solves
A d = fl32(r) with Algorithm 9 on float32 vectors, a float32 matrix and float32
SpMV (scipy.sparse, float32 accumulation) but dot products accumulated in
float64, then sets x := x + d in FP64. Written with numpy vector operations in
the order of Algorithm 9; the only library primitives are the SpMV and the dot
product.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import oracle

f32 = np.float32


def dot64(a, b):
    """Dot product of float32 vectors accumulated in float64 (products exact)."""
    return float(np.dot(a.astype(np.float64), b.astype(np.float64)))


def pbicgstab_f32(A32, b32, rtol, maxit):
    """Algorithm 9 on float32 vectors from x0 = 0; returns (x, iterations)."""
    n = b32.size
    x = np.zeros(n, dtype=f32)
    r = b32.copy()                       # b - A 0
    r0 = r.copy()
    w = A32 @ r
    t = A32 @ w
    p = np.zeros(n, dtype=f32); s = p.copy(); z = p.copy(); v = p.copy()
    rho = dot64(r0, r)
    nr0 = np.sqrt(dot64(r, r))
    if nr0 == 0.0:
        return x, 0
    r0w = dot64(r0, w)
    if r0w == 0.0:
        return x, 0
    alpha, beta, omega = rho / r0w, 0.0, 0.0
    for i in range(maxit):
        al, be, om = f32(alpha), f32(beta), f32(omega)
        p = r + be * (p - om * s)
        s = w + be * (s - om * z)
        z = t + be * (z - om * v)
        q = r - al * s
        y = w - al * z
        qy, yy, qq = dot64(q, y), dot64(y, y), dot64(q, q)
        v = A32 @ z
        if np.sqrt(qq) <= rtol * nr0 or yy == 0.0:
            x = x + al * p
            return x, i + 1
        omega = qy / yy
        om = f32(omega)
        x = x + al * p + om * q
        r = q - om * y
        w = y - om * (t - al * v)
        rho_n, r0w, r0s, r0z = dot64(r0, r), dot64(r0, w), dot64(r0, s), dot64(r0, z)
        t = A32 @ w
        if np.sqrt(dot64(r, r)) <= rtol * nr0 or rho_n == 0.0:
            return x, i + 1
        beta = (alpha / omega) * (rho_n / rho)
        alpha = rho_n / (r0w + beta * r0s - beta * omega * r0z)
        rho = rho_n
    return x, maxit


def refine(A, b, rtol=1e-10, max_outer=20, inner_rtol=1e-4, inner_maxit=1000, values32=None):
    """FP64 iterative refinement with FP32 inner Algorithm 9. ``values32``: the
    float32 values of A's CSR structure (default: A's values rounded).
    Returns dict(x, outer, inner_iters, rel_res_true, history)."""
    vals = A.val.astype(f32) if values32 is None else np.asarray(values32, dtype=f32)
    A32 = sp.csr_matrix((vals, A.col, A.rowptr), shape=(A.n, A.n))
    x = np.zeros(A.n)
    hist = []
    inner_total = 0
    nr0 = None
    for outer in range(max_outer + 1):
        r = b - oracle.spmv(A, x)
        nr = np.linalg.norm(r)
        if nr0 is None:
            nr0 = nr
        hist.append(nr)
        if nr <= rtol * nr0 or outer == max_outer:
            break
        d, its = pbicgstab_f32(A32, r.astype(f32), inner_rtol, inner_maxit)
        inner_total += its
        x = x + d.astype(np.float64)
    return dict(x=x, outer=len(hist) - 1, inner_iters=inner_total, rel_res_true=hist[-1] / nr0,
                history=np.array(hist))
