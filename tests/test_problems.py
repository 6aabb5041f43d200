"""Input generators: RNG test vectors, operator definitions and CSR/stencil equality (CPU)."""
import os

import numpy as np
import pytest

from paper_1612_01395_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for seed, *outs in rows:
        got = [int(v) for v in P.splitmix64(int(seed), len(outs))]
        assert got == [int(o, 16) for o in outs]


def test_uniform_range_and_offset_streams():
    u = P.splitmix64_uniform(7, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01
    np.testing.assert_array_equal(P.splitmix64_uniform(7, 10, start=5), u[5:15])


def dense_cd(nx, ny, nz, vel):
    """Upwind convection-diffusion assembled entry by entry from its definition."""
    n = nx * ny * nz
    h = 1.0 / (nx + 1)
    a = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = i + nx * (j + ny * k)
                cs = vel(i, j, k)
                axes = [(1, i, nx), (nx, j, ny)] + ([(nx * ny, k, nz)] if nz > 1 else [])
                diag = 0.0
                for (stride, idx, m), c in zip(axes, cs):
                    diag += 2.0 + h * abs(c)
                    if idx > 0:
                        a[row, row - stride] = -1.0 - h * max(c, 0.0)
                    if idx < m - 1:
                        a[row, row + stride] = -1.0 - h * max(-c, 0.0)
                a[row, row] = diag
    return a


def test_cd2d_matches_definition():
    st = P.cd2d_constant(6, (10.0, -3.0))
    A = P.stencil_to_csr(st)
    ref = dense_cd(6, 6, 1, lambda i, j, k: (10.0, -3.0))
    np.testing.assert_allclose(A.to_dense(), ref, rtol=1e-15, atol=0)


def test_cd3d_matches_definition():
    n = 5
    h = 1.0 / (n + 1)
    c = (np.arange(n) + 1) * h
    st = P.cd3d_trig(n)
    A = P.stencil_to_csr(st)
    ref = dense_cd(n, n, n, lambda i, j, k: (20 * np.sin(c[j]), 20 * np.cos(c[k]), 20 * np.sin(c[i])))
    np.testing.assert_allclose(A.to_dense(), ref, rtol=1e-15, atol=0)


def test_nnz_formulas():
    assert P.stencil_to_csr(P.cd2d_constant(64)).nnz == 5 * 4096 - 4 * 64
    A = P.stencil_to_csr(P.cd3d_trig(16))
    assert A.nnz == 7 * 16 ** 3 - 6 * 16 ** 2


def test_csr_rows_sorted_and_in_range():
    A = P.stencil_to_csr(P.cd3d_trig(7))
    for r in range(A.n):
        cols = A.col[A.rowptr[r]:A.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
        assert cols.min() >= 0 and cols.max() < A.n


def test_stencil_coefficients_identical_to_csr_values():
    """The stencil form evaluates to the very doubles stored in CSR."""
    st = P.cd3d_trig(9)
    A = P.stencil_to_csr(st)
    dense = A.to_dense()
    nx = ny = nz = 9
    for d in range(7):
        grid = st.coefs[d].on_grid(nx, ny, nz)
        di, dj, dk = P.OFFSETS[d]
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        assert dense[i + nx * (j + ny * k), ii + nx * (jj + ny * kk)] == grid[k, j, i]


def test_ptp_stencils():
    a1 = P.stencil_to_csr(P.ptp1(4)).to_dense()
    # centre 4, W and N -1, E and S -eps (lexicographic, x fastest)
    r = 1 + 4 * 1
    assert a1[r, r] == 4.0 and a1[r, r - 1] == -1.0 and a1[r, r + 4] == -1.0
    assert a1[r, r + 1] == -0.999 and a1[r, r - 4] == -0.999
    a2 = P.stencil_to_csr(P.ptp2(4)).to_dense()
    assert a2[r, r] == 1.0 and np.all(a2[r, [r - 1, r + 1, r - 4, r + 4]] == -1.0)


def test_random_sparse_structure():
    A = P.random_sparse(200, seed=3)
    dense = A.to_dense()
    off = dense - np.diag(np.diag(dense))
    counts = np.count_nonzero(off, axis=1)
    assert counts.min() >= 8 and counts.max() <= 32
    np.testing.assert_allclose(np.diag(dense), 1.1 * np.abs(off).sum(axis=1), rtol=1e-15)
