"""Exact rational BiCGStab variants for tiny systems -- test infrastructure only.

Algorithms 7, 8 and 9 of Cools & Vanroose (arXiv:1612.01395), plus the eq. (5)
form of alpha and the residual replacement of Section 4.2, in exact arithmetic
with ``fractions.Fraction``. In exact arithmetic the three algorithms produce
the same iterates (Section 3.2, Section 3.3), and residual replacement changes
nothing, so any wrong coefficient or index in one of them breaks equality.

The iteration stops when the residual is exactly zero (or the half step makes
it zero), on breakdown, or after ``maxit`` iterations. The returned dictionary
holds the iterates ``x[i]``, ``r[i]`` (lists of Fractions) for every completed
iteration and a ``status`` string.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence

Vec = List[Fraction]


def _vec(v: Sequence) -> Vec:
    return [Fraction(e) for e in v]


def matvec(A, x: Vec) -> Vec:
    return [sum((Fraction(a) * xi for a, xi in zip(row, x)), Fraction(0)) for row in A]


def dot(a: Vec, b: Vec) -> Fraction:
    return sum((ai * bi for ai, bi in zip(a, b)), Fraction(0))


def lin(a: Vec, c: Fraction, b: Vec) -> Vec:
    """a + c * b"""
    return [ai + c * bi for ai, bi in zip(a, b)]


def _is_zero(v: Vec) -> bool:
    return all(e == 0 for e in v)


def bicgstab(A, b, x0=None, maxit=50):
    """Algorithm 7."""
    n = len(b)
    b = _vec(b)
    x = _vec(x0) if x0 is not None else [Fraction(0)] * n
    r = lin(b, Fraction(-1), matvec(A, x))
    r0 = list(r)
    p = list(r)
    rho = dot(r0, r)
    xs, rs = [list(x)], [list(r)]
    if _is_zero(r):
        return dict(x=xs, r=rs, status="converged", half_step=False, angles=[])
    angles = []   # per iteration: squared cosines of (r0, s_i) and (q_i, y_i)
    for _ in range(maxit):
        s = matvec(A, p)
        r0s = dot(r0, s)
        if r0s == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, angles=angles)
        alpha = rho / r0s
        q = lin(r, -alpha, s)
        y = matvec(A, q)
        qy, yy = dot(q, y), dot(y, y)
        qq = dot(q, q)
        angles.append((r0s * r0s / (dot(r0, r0) * dot(s, s)), qy * qy / (qq * yy) if qq and yy else Fraction(1)))
        if yy == 0:
            if not _is_zero(q):
                return dict(x=xs, r=rs, status="breakdown", half_step=False, angles=angles)
            x = lin(x, alpha, p)
            xs.append(list(x)); rs.append(list(q))
            return dict(x=xs, r=rs, status="converged", half_step=True, angles=angles)
        omega = qy / yy
        if omega == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, angles=angles)
        x = lin(lin(x, alpha, p), omega, q)
        r = lin(q, -omega, y)
        xs.append(list(x)); rs.append(list(r))
        if _is_zero(r):
            return dict(x=xs, r=rs, status="converged", half_step=False, angles=angles)
        rho_new = dot(r0, r)
        if rho_new == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, angles=angles)
        beta = (alpha / omega) * (rho_new / rho)
        rho = rho_new
        p = lin(r, beta, lin(p, -omega, s))
    return dict(x=xs, r=rs, status="maxit", half_step=False, angles=angles)


def cabicgstab(A, b, x0=None, maxit=50):
    """Algorithm 8 (alpha by eq. (3))."""
    n = len(b)
    b = _vec(b)
    x = _vec(x0) if x0 is not None else [Fraction(0)] * n
    r = lin(b, Fraction(-1), matvec(A, x))
    r0 = list(r)
    w = matvec(A, r)
    zero = [Fraction(0)] * n
    p, s, z = list(zero), list(zero), list(zero)
    xs, rs = [list(x)], [list(r)]
    if _is_zero(r):
        return dict(x=xs, r=rs, status="converged", half_step=False)
    rho = dot(r0, r)
    if dot(r0, w) == 0:
        return dict(x=xs, r=rs, status="breakdown", half_step=False)
    alpha, beta, omega = rho / dot(r0, w), Fraction(0), Fraction(0)
    for _ in range(maxit):
        p = lin(r, beta, lin(p, -omega, s))
        s = lin(w, beta, lin(s, -omega, z))
        z = matvec(A, s)
        q = lin(r, -alpha, s)
        y = lin(w, -alpha, z)
        qy, yy = dot(q, y), dot(y, y)
        if yy == 0:
            if not _is_zero(q):
                return dict(x=xs, r=rs, status="breakdown", half_step=False)
            x = lin(x, alpha, p)
            xs.append(list(x)); rs.append(list(q))
            return dict(x=xs, r=rs, status="converged", half_step=True)
        omega = qy / yy
        if omega == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False)
        x = lin(lin(x, alpha, p), omega, q)
        r = lin(q, -omega, y)
        w = matvec(A, r)
        xs.append(list(x)); rs.append(list(r))
        if _is_zero(r):
            return dict(x=xs, r=rs, status="converged", half_step=False)
        rho_new, r0w, r0s, r0z = dot(r0, r), dot(r0, w), dot(r0, s), dot(r0, z)
        if rho_new == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False)
        beta = (alpha / omega) * (rho_new / rho)
        den = r0w + beta * r0s - beta * omega * r0z
        if den == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False)
        alpha = rho_new / den
        rho = rho_new
    return dict(x=xs, r=rs, status="maxit", half_step=False)


def pbicgstab(A, b, x0=None, maxit=50, replace_period=0, alpha_eq5=False, rr_placement=0):
    """Algorithm 9, with residual replacement every ``replace_period`` iterations.

    ``rr_placement`` 0: r, w are replaced after x_i, r_i, w_i are formed and
    before the second reduction, s, z after p_i (the placement the FP64 oracle
    uses by default); 1: all four after p_i. Both leave every iterate unchanged
    in exact arithmetic.
    """
    n = len(b)
    b = _vec(b)
    x = _vec(x0) if x0 is not None else [Fraction(0)] * n
    r = lin(b, Fraction(-1), matvec(A, x))
    r0 = list(r)
    w = matvec(A, r)
    t = matvec(A, w)
    zero = [Fraction(0)] * n
    p, s, z, v = list(zero), list(zero), list(zero), list(zero)
    xs, rs = [list(x)], [list(r)]
    if _is_zero(r):
        return dict(x=xs, r=rs, status="converged", half_step=False, replacements=0)
    rho = dot(r0, r)
    if dot(r0, w) == 0:
        return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=0)
    alpha, beta, omega = rho / dot(r0, w), Fraction(0), Fraction(0)
    nrr = 0
    replaced_rw = False
    for i in range(maxit):
        p = lin(r, beta, lin(p, -omega, s))
        late = rr_placement == 1 and replace_period > 0 and i > 0 and i % replace_period == 0
        if replaced_rw:
            s = matvec(A, p)
            z = matvec(A, s)
        elif late:
            r = lin(b, Fraction(-1), matvec(A, x))
            w = matvec(A, r)
            s = matvec(A, p)
            z = matvec(A, s)
            nrr += 1
        else:
            s = lin(w, beta, lin(s, -omega, z))
            z = lin(t, beta, lin(z, -omega, v))
        q = lin(r, -alpha, s)
        y = lin(w, -alpha, z)
        qy, yy = dot(q, y), dot(y, y)
        v = matvec(A, z)
        if yy == 0:
            if not _is_zero(q):
                return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
            x = lin(x, alpha, p)
            xs.append(list(x)); rs.append(list(q))
            return dict(x=xs, r=rs, status="converged", half_step=True, replacements=nrr)
        omega = qy / yy
        if omega == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
        x = lin(lin(x, alpha, p), omega, q)
        r = lin(q, -omega, y)
        w = lin(y, -omega, lin(t, -alpha, v))
        replaced_rw = rr_placement == 0 and replace_period > 0 and (i + 1) % replace_period == 0
        if replaced_rw:
            r = lin(b, Fraction(-1), matvec(A, x))
            w = matvec(A, r)
            nrr += 1
        rho_new, r0w, r0s, r0z = dot(r0, r), dot(r0, w), dot(r0, s), dot(r0, z)
        t = matvec(A, w)
        xs.append(list(x)); rs.append(list(r))
        if _is_zero(r):
            return dict(x=xs, r=rs, status="converged", half_step=False, replacements=nrr)
        if rho_new == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
        beta = (alpha / omega) * (rho_new / rho)
        if alpha_eq5:
            inv = 1 / omega + r0w / rho_new - beta * omega * (r0z / rho_new)
            if inv == 0:
                return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
            alpha = 1 / inv
        else:
            den = r0w + beta * r0s - beta * omega * r0z
            if den == 0:
                return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
            alpha = rho_new / den
        rho = rho_new
    return dict(x=xs, r=rs, status="maxit", half_step=False, replacements=nrr)


def _prec(minv, u: Vec) -> Vec:
    return [m * e for m, e in zip(minv, u)]


def bicgstab_prec(A, minv, b, x0=None, maxit=50):
    """Algorithm 10 with M^{-1} u = minv * u (minv: Fractions)."""
    n = len(b)
    b = _vec(b)
    minv = _vec(minv)
    x = _vec(x0) if x0 is not None else [Fraction(0)] * n
    r = lin(b, Fraction(-1), matvec(A, x))
    r0 = list(r)
    p = list(r)
    rho = dot(r0, r)
    xs, rs = [list(x)], [list(r)]
    if _is_zero(r):
        return dict(x=xs, r=rs, status="converged", half_step=False)
    for _ in range(maxit):
        ph = _prec(minv, p)
        s = matvec(A, ph)
        r0s = dot(r0, s)
        if r0s == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False)
        alpha = rho / r0s
        q = lin(r, -alpha, s)
        qh = _prec(minv, q)
        y = matvec(A, qh)
        qy, yy = dot(q, y), dot(y, y)
        if yy == 0:
            if not _is_zero(q):
                return dict(x=xs, r=rs, status="breakdown", half_step=False)
            x = lin(x, alpha, ph)
            xs.append(list(x)); rs.append(list(q))
            return dict(x=xs, r=rs, status="converged", half_step=True)
        omega = qy / yy
        if omega == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False)
        x = lin(lin(x, alpha, ph), omega, qh)
        r = lin(q, -omega, y)
        xs.append(list(x)); rs.append(list(r))
        if _is_zero(r):
            return dict(x=xs, r=rs, status="converged", half_step=False)
        rho_new = dot(r0, r)
        if rho_new == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False)
        beta = (alpha / omega) * (rho_new / rho)
        rho = rho_new
        p = lin(r, beta, lin(p, -omega, s))
    return dict(x=xs, r=rs, status="maxit", half_step=False)


def pbicgstab_prec(A, minv, b, x0=None, maxit=50, replace_period=0):
    """Algorithm 11 with M^{-1} u = minv * u and residual replacement (split placement)."""
    n = len(b)
    b = _vec(b)
    minv = _vec(minv)
    x = _vec(x0) if x0 is not None else [Fraction(0)] * n
    r = lin(b, Fraction(-1), matvec(A, x))
    r0 = list(r)
    rh = _prec(minv, r)
    w = matvec(A, rh)
    wh = _prec(minv, w)
    t = matvec(A, wh)
    zero = [Fraction(0)] * n
    ph, s, sh, z, zh, v = (list(zero) for _ in range(6))
    xs, rs = [list(x)], [list(r)]
    if _is_zero(r):
        return dict(x=xs, r=rs, status="converged", half_step=False, replacements=0)
    rho = dot(r0, r)
    if dot(r0, w) == 0:
        return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=0)
    alpha, beta, omega = rho / dot(r0, w), Fraction(0), Fraction(0)
    nrr = 0
    replaced = False
    for i in range(maxit):
        ph = lin(rh, beta, lin(ph, -omega, sh))
        if replaced:
            s = matvec(A, ph)
            sh = _prec(minv, s)
            z = matvec(A, sh)
        else:
            s = lin(w, beta, lin(s, -omega, z))
            sh = lin(wh, beta, lin(sh, -omega, zh))
            z = lin(t, beta, lin(z, -omega, v))
        q = lin(r, -alpha, s)
        qh = lin(rh, -alpha, sh)
        y = lin(w, -alpha, z)
        qy, yy = dot(q, y), dot(y, y)
        zh = _prec(minv, z)
        v = matvec(A, zh)
        if yy == 0:
            if not _is_zero(q):
                return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
            x = lin(x, alpha, ph)
            xs.append(list(x)); rs.append(list(q))
            return dict(x=xs, r=rs, status="converged", half_step=True, replacements=nrr)
        omega = qy / yy
        if omega == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
        x = lin(lin(x, alpha, ph), omega, qh)
        r = lin(q, -omega, y)
        rh = lin(qh, -omega, lin(wh, -alpha, zh))
        w = lin(y, -omega, lin(t, -alpha, v))
        replaced = replace_period > 0 and (i + 1) % replace_period == 0
        if replaced:
            r = lin(b, Fraction(-1), matvec(A, x))
            rh = _prec(minv, r)
            w = matvec(A, rh)
            nrr += 1
        rho_new, r0w, r0s, r0z = dot(r0, r), dot(r0, w), dot(r0, s), dot(r0, z)
        wh = _prec(minv, w)
        t = matvec(A, wh)
        xs.append(list(x)); rs.append(list(r))
        if _is_zero(r):
            return dict(x=xs, r=rs, status="converged", half_step=False, replacements=nrr)
        if rho_new == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
        beta = (alpha / omega) * (rho_new / rho)
        den = r0w + beta * r0s - beta * omega * r0z
        if den == 0:
            return dict(x=xs, r=rs, status="breakdown", half_step=False, replacements=nrr)
        alpha = rho_new / den
        rho = rho_new
    return dict(x=xs, r=rs, status="maxit", half_step=False, replacements=nrr)
