"""Seeded synthetic inputs: test matrices, right-hand sides and random vectors.

This module only *builds inputs*. It holds none of the solver's arithmetic (no
matrix-vector product, dot product or recurrence), so both the CUDA path and the
CPU oracle can take their inputs from it without sharing any of the method.

Contents
--------
* ``splitmix64_uniform``: U[-1, 1) doubles from SplitMix64 (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014).
* ``convection_diffusion``: 2-D 5-point / 3-D 7-point first-order upwind
  convection-diffusion operators on the unit square/cube with Dirichlet
  boundaries eliminated, in CSR form and in the equivalent stencil form. Both
  forms hold the same coefficients bit for bit and list a row's entries in the
  same order (B, S, W, C, E, N, T = ascending column index), so an SpMV that
  sums a row in that order gives identical results on both forms.
* ``ptp1`` / ``ptp2``: the paper's two parallel test problems (Section 5,
  equations PTP1 and PTP2), constant 5-point stencils on an n x n grid.

Grid ordering is lexicographic with x fastest: ``row = i + nx*(j + ny*k)``.
Stencil directions are indexed ``0=C, 1=W(i-1), 2=E(i+1), 3=S(j-1), 4=N(j+1),
5=B(k-1), 6=T(k+1)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

# Direction indices of the stencil form.
C, W, E, S, N, B, T = range(7)
# Grid offset (di, dj, dk) of each direction.
OFFSETS = {C: (0, 0, 0), W: (-1, 0, 0), E: (1, 0, 0), S: (0, -1, 0),
           N: (0, 1, 0), B: (0, 0, -1), T: (0, 0, 1)}
# Order in which a row's entries appear in CSR (ascending column index).
CSR_ORDER = (B, S, W, C, E, N, T)

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream seeded with ``seed``.

    Output j is ``mix(seed + (j+1)*GAMMA)`` with the published finaliser
    (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31), all mod 2^64.
    """
    j = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + j * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_uniform(seed: int, count: int, start: int = 0) -> np.ndarray:
    """U[-1, 1) doubles: u = (z >> 11) * 2^-53 in [0, 1), value = 2u - 1 (exact)."""
    z = splitmix64(seed, count, start)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


@dataclass
class Coef:
    """One stencil coefficient as a function of the node (i, j, k).

    ``value`` is used when ``table`` is None. Otherwise the coefficient is
    ``table[i*stride[0] + j*stride[1] + k*stride[2]]`` plus, when ``table2`` is
    given, ``table2[i*stride2[0] + j*stride2[1] + k*stride2[2]]`` (added second).
    """
    value: float = 0.0
    table: Optional[np.ndarray] = None
    stride: tuple = (0, 0, 0)
    table2: Optional[np.ndarray] = None
    stride2: tuple = (0, 0, 0)

    def on_grid(self, nx: int, ny: int, nz: int) -> np.ndarray:
        """The coefficient at every node, shape (nz, ny, nx), same rounding as a kernel."""
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        if self.table is None:
            out = np.full((nz, ny, nx), self.value, dtype=np.float64)
        else:
            s = self.stride
            out = self.table[i * s[0] + j * s[1] + k * s[2]].astype(np.float64)
        if self.table2 is not None:
            s = self.stride2
            out = out + self.table2[i * s[0] + j * s[1] + k * s[2]]
        return out


@dataclass
class Stencil:
    """A 5-point (nz == 1) or 7-point stencil operator with Dirichlet elimination."""
    nx: int
    ny: int
    nz: int
    coefs: list = field(default_factory=list)   # 7 Coef, indexed by direction

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dim(self) -> int:
        return 2 if self.nz == 1 else 3


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray   # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.col] = self.val
        return a


def stencil_to_csr(st: Stencil) -> CSR:
    """Assemble the stencil as CSR with entries in ascending column order.

    Neighbours outside the grid are dropped (Dirichlet elimination). Values are
    copied from ``Coef.on_grid``, so both forms hold identical doubles.
    """
    nx, ny, nz = st.nx, st.ny, st.nz
    n = st.n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    dirs = [d for d in CSR_ORDER if st.dim == 3 or d not in (B, T)]
    masks, vals = [], []
    for d in dirs:
        di, dj, dk = OFFSETS[d]
        m = (i + di >= 0) & (i + di < nx) & (j + dj >= 0) & (j + dj < ny) & (k + dk >= 0) & (k + dk < nz)
        masks.append(m)
        vals.append(st.coefs[d].on_grid(nx, ny, nz).ravel())
    counts = np.zeros(n, dtype=np.int64)
    for m in masks:
        counts += m
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    if nnz >= 2 ** 31:
        raise ValueError("nnz does not fit int32")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = rowptr[:-1].copy()
    rows = np.arange(n, dtype=np.int64)
    for d, m, v in zip(dirs, masks, vals):
        di, dj, dk = OFFSETS[d]
        delta = di + nx * (dj + ny * dk)
        p = pos[m]
        col[p] = (rows[m] + delta).astype(np.int32)
        val[p] = v[m]
        pos[m] += 1
    return CSR(n=n, rowptr=rowptr.astype(np.int32), col=col, val=val)


def convection_diffusion(shape: Sequence[int], velocity: Sequence[np.ndarray]) -> Stencil:
    """First-order upwind convection-diffusion, operator scaled by h^2.

    ``-Laplace(u) + c . grad(u)`` on the unit square (2-D) or cube (3-D),
    ``h = 1/(n+1)`` per axis (all axes must have the same n), node coordinate
    ``(i+1) h``. Each velocity component depends on one other coordinate and is
    given as a 1-D table: 2-D ``(c_x over j, c_y over i)``; 3-D
    ``(c_x over j, c_y over k, c_z over i)``.

    Per axis with velocity c: minus-side neighbour ``-1 - h*max(c, 0)``,
    plus-side neighbour ``-1 - h*max(-c, 0)``, diagonal contribution
    ``2 + h*|c|``. The diagonal is summed as ``(a_x + a_y) + a_z``.
    """
    if len(shape) == 2:
        nx, ny = shape
        nz = 1
    else:
        nx, ny, nz = shape
    if len(set(s for s in (nx, ny, nz) if s > 1)) != 1:
        raise ValueError("all axes must have the same number of points")
    nn = nx
    h = 1.0 / (nn + 1)

    def minus(c):
        return -1.0 - h * np.maximum(c, 0.0)

    def plus(c):
        return -1.0 - h * np.maximum(-c, 0.0)

    def diag(c):
        return 2.0 + h * np.abs(c)

    coefs = [None] * 7
    if len(shape) == 2:
        cx, cy = (np.asarray(v, dtype=np.float64) for v in velocity)   # cx over j, cy over i
        ax, ay = diag(cx), diag(cy)
        coefs[C] = Coef(table=ax, stride=(0, 1, 0), table2=ay, stride2=(1, 0, 0))
        coefs[W] = Coef(table=minus(cx), stride=(0, 1, 0))
        coefs[E] = Coef(table=plus(cx), stride=(0, 1, 0))
        coefs[S] = Coef(table=minus(cy), stride=(1, 0, 0))
        coefs[N] = Coef(table=plus(cy), stride=(1, 0, 0))
        coefs[B] = Coef(value=0.0)
        coefs[T] = Coef(value=0.0)
    else:
        cx, cy, cz = (np.asarray(v, dtype=np.float64) for v in velocity)  # over j, k, i
        ax, ay, az = diag(cx), diag(cy), diag(cz)
        axy = (ax[:, None] + ay[None, :]).T.ravel()    # index j + ny*k
        coefs[C] = Coef(table=axy, stride=(0, 1, ny), table2=az, stride2=(1, 0, 0))
        coefs[W] = Coef(table=minus(cx), stride=(0, 1, 0))
        coefs[E] = Coef(table=plus(cx), stride=(0, 1, 0))
        coefs[S] = Coef(table=minus(cy), stride=(0, 0, 1))
        coefs[N] = Coef(table=plus(cy), stride=(0, 0, 1))
        coefs[B] = Coef(table=minus(cz), stride=(1, 0, 0))
        coefs[T] = Coef(table=plus(cz), stride=(1, 0, 0))
    return Stencil(nx=nx, ny=ny, nz=nz, coefs=coefs)


def cd2d_constant(n: int = 64, c: Sequence[float] = (10.0, 10.0)) -> Stencil:
    """2-D convection-diffusion with constant velocity (c_x, c_y) on an n x n grid."""
    return convection_diffusion((n, n), (np.full(n, c[0]), np.full(n, c[1])))


def cd2d_field(n: int = 1024, cmax: float = 50.0, seed: int = 0) -> Stencil:
    """2-D convection-diffusion with a per-cell velocity (c, c), c ~ U[0, cmax]
    from SplitMix64 (one value per node, lexicographic order): minus-side
    neighbours -1 - h c, plus-side -1, diagonal 4 + 2 h c (c >= 0, upwind)."""
    h = 1.0 / (n + 1)
    c = 0.5 * cmax * (splitmix64_uniform(seed ^ 0xC0FFEE, n * n) + 1.0)
    minus = -1.0 - h * c
    coefs = [None] * 7
    coefs[C] = Coef(table=(2.0 + h * c) + (2.0 + h * c), stride=(1, n, 0))
    coefs[W] = Coef(table=minus, stride=(1, n, 0))
    coefs[E] = Coef(value=-1.0)
    coefs[S] = Coef(table=minus, stride=(1, n, 0))
    coefs[N] = Coef(value=-1.0)
    coefs[B] = Coef(value=0.0)
    coefs[T] = Coef(value=0.0)
    return Stencil(nx=n, ny=n, nz=1, coefs=coefs)


def cd3d_trig(n: int = 256, amp: float = 20.0) -> Stencil:
    """3-D convection-diffusion, velocity (amp sin y, amp cos z, amp sin x), n^3 grid."""
    h = 1.0 / (n + 1)
    coord = (np.arange(n) + 1) * h
    return convection_diffusion((n, n, n), (amp * np.sin(coord), amp * np.cos(coord), amp * np.sin(coord)))


def constant_stencil_2d(n: int, center: float, west: float, east: float, south: float, north: float) -> Stencil:
    coefs = [None] * 7
    coefs[C] = Coef(value=center)
    coefs[W] = Coef(value=west)
    coefs[E] = Coef(value=east)
    coefs[S] = Coef(value=south)
    coefs[N] = Coef(value=north)
    coefs[B] = Coef(value=0.0)
    coefs[T] = Coef(value=0.0)
    return Stencil(nx=n, ny=n, nz=1, coefs=coefs)


def ptp1(n: int = 1000, eps: float = 1.0 - 0.001) -> Stencil:
    """Parallel test problem 1 (Section 5, equation PTP1): centre 4, W = N = -1, E = S = -eps."""
    return constant_stencil_2d(n, 4.0, -1.0, -eps, -eps, -1.0)


def ptp2(n: int = 1000) -> Stencil:
    """Parallel test problem 2 (Section 5, equation PTP2): centre 1, all four neighbours -1."""
    return constant_stencil_2d(n, 1.0, -1.0, -1.0, -1.0, -1.0)


def random_integer_system(n: int, seed: int, lo: int = -3, hi: int = 3, diag_boost: int = 0):
    """Small dense unsymmetric integer matrix and integer right-hand side (rational tests).

    Entries are uniform integers in [lo, hi] from SplitMix64; ``diag_boost`` is
    added to the diagonal. Returns (A as int64 n x n, b as int64 n).
    """
    z = splitmix64(seed, n * n + n)
    span = np.uint64(hi - lo + 1)
    v = (z % span).astype(np.int64) + lo
    a = v[: n * n].reshape(n, n)
    a[np.arange(n), np.arange(n)] += diag_boost
    return a, v[n * n:]


def dense_to_csr(a: np.ndarray) -> CSR:
    n = a.shape[0]
    rows, cols = np.nonzero(a)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n=n, rowptr=rowptr.astype(np.int32), col=cols.astype(np.int32),
               val=a[rows, cols].astype(np.float64))


def random_sparse(n: int, seed: int, nnz_lo: int = 8, nnz_hi: int = 32, dominance: float = 1.1) -> CSR:
    """Random unsymmetric sparse matrix: row r gets k_r ~ U{nnz_lo..nnz_hi}
    off-diagonal entries at distinct uniformly random columns (diagonal
    excluded; duplicates redrawn), values N(0,1) (Box-Muller on SplitMix64
    uniforms), and diagonal = dominance * the row's sum of |off-diagonal|.
    """
    if n < 2:
        raise ValueError("n >= 2 required")
    kspan = nnz_hi - nnz_lo + 1
    counts = nnz_lo + (splitmix64(seed ^ 0x5EED, n) % np.uint64(kspan)).astype(np.int64)
    counts = np.minimum(counts, n - 1)
    total = int(counts.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), counts)
    stream = 0

    def draw(rr, cnt):
        nonlocal stream
        d = (splitmix64(seed, cnt, start=stream) % np.uint64(n - 1)).astype(np.int64)
        stream += cnt
        return d + (d >= rr)          # skip the diagonal

    cols = draw(rows, total)
    for _ in range(1000):
        key = np.sort(rows * n + cols)          # rows sorted, columns sorted within a row
        rows, cols = key // n, key % n
        dup = np.zeros(total, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        m = int(dup.sum())
        if m == 0:
            break
        cols[dup] = draw(rows[dup], m)
    u = (splitmix64(seed ^ 0xA5A5A5A5, 2 * total) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    g = np.sqrt(-2.0 * np.log1p(-u[:total])) * np.cos(2.0 * np.pi * u[total:])
    diag = dominance * np.bincount(rows, weights=np.abs(g), minlength=n)
    allr = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    allc = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    allv = np.concatenate([g, diag])
    order = np.argsort(allr * n + allc)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts + 1, out=rowptr[1:])
    return CSR(n=n, rowptr=rowptr.astype(np.int32), col=allc[order].astype(np.int32), val=allv[order])


@dataclass
class Batch:
    """Independent systems concatenated: system s owns rows row_offset[s]..row_offset[s+1]."""
    sizes: np.ndarray        # int64 [nsys]
    row_offset: np.ndarray   # int64 [nsys+1]
    rowptr: np.ndarray       # int32 [total+1], offsets into col/val
    col: np.ndarray          # int32, local to the system
    val: np.ndarray          # float64
    b: np.ndarray            # float64 [total]

    @property
    def nsys(self) -> int:
        return int(self.sizes.size)

    @property
    def total_rows(self) -> int:
        return int(self.row_offset[-1])

    def system(self, s: int) -> CSR:
        r0, r1 = int(self.row_offset[s]), int(self.row_offset[s + 1])
        rp = self.rowptr[r0:r1 + 1].astype(np.int64)
        e0, e1 = int(rp[0]), int(rp[-1])
        return CSR(n=r1 - r0, rowptr=(rp - e0).astype(np.int32), col=self.col[e0:e1], val=self.val[e0:e1])


def random_batch(nsys: int = 512, seed: int = 0, nmin: int = 1000, nmax: int = 64000,
                 nnz_lo: int = 8, nnz_hi: int = 32) -> Batch:
    """nsys random_sparse systems with sizes log-uniform in [nmin, nmax] and
    b ~ U[-1, 1], ordered largest first (which balances a work queue)."""
    u = (splitmix64(seed ^ 0xB47C4, nsys) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    sizes = np.rint(np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    sizes = np.sort(sizes)[::-1].copy()
    mats = [random_sparse(int(n), seed * 100003 + 17 * s + 1, nnz_lo, nnz_hi) for s, n in enumerate(sizes)]
    row_offset = np.zeros(nsys + 1, dtype=np.int64)
    np.cumsum(sizes, out=row_offset[1:])
    nnz = np.array([m.nnz for m in mats], dtype=np.int64)
    nnz_off = np.zeros(nsys + 1, dtype=np.int64)
    np.cumsum(nnz, out=nnz_off[1:])
    if nnz_off[-1] >= 2 ** 31:
        raise ValueError("total nnz does not fit int32")
    rowptr = np.concatenate([m.rowptr[:-1].astype(np.int64) + nnz_off[s] for s, m in enumerate(mats)] +
                            [nnz_off[-1:]])
    b = splitmix64_uniform(seed ^ 0xBBBB, int(row_offset[-1]))
    return Batch(sizes=sizes, row_offset=row_offset, rowptr=rowptr.astype(np.int32),
                 col=np.concatenate([m.col for m in mats]), val=np.concatenate([m.val for m in mats]), b=b)
