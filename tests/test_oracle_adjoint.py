"""The oracle's adjoint gradient of a sparse solve, pinned by finite differences (CPU)."""
import numpy as np
import scipy.sparse as sp

import oracle
from paper_1612_01395_gb300 import problems as P


def transpose(A):
    """A^T as a problems.CSR via scipy (rows sorted by column)."""
    m = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n)).T.tocsr()
    m.sort_indices()
    return P.CSR(n=A.n, rowptr=m.indptr.astype(np.int32), col=m.indices.astype(np.int32), val=m.data.copy())


def oracle_gradients(A, b, xt, rtol=1e-13):
    """L = 0.5 ||x - xt||^2, x = A^{-1} b: dL/db = lambda, dL/da_ij = -lambda_i x_j."""
    x = oracle.pbicgstab(A, b, rtol=rtol, maxit=5000, replace_period=20).x
    lam = oracle.pbicgstab(transpose(A), x - xt, rtol=rtol, maxit=5000, replace_period=20).x
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return x, lam, -lam[rows] * x[A.col]


def loss(A, b, xt):
    x = oracle.pbicgstab(A, b, rtol=1e-13, maxit=5000, replace_period=20).x
    return 0.5 * float(np.dot(x - xt, x - xt))


def test_oracle_adjoint_matches_central_differences():
    """Central differences with h = 1e-6 carry noise of about L * (solve accuracy)
    / h ~ 1e-9 here, hence the absolute term of the bound."""
    st = P.cd2d_field(12, seed=1)
    A = P.stencil_to_csr(st)
    b = P.splitmix64_uniform(2, A.n)
    xt = P.splitmix64_uniform(3, A.n)
    x, gb, gv = oracle_gradients(A, b, xt)
    h = 1e-6
    idx = (P.splitmix64(4, 8) % np.uint64(A.n)).astype(int)
    for i in idx:
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(A, bp, xt) - loss(A, bm, xt)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-5 * abs(gb[i]) + 1e-8
    kdx = (P.splitmix64(5, 8) % np.uint64(A.nnz)).astype(int)
    for k in kdx:
        Ap = P.CSR(A.n, A.rowptr, A.col, A.val.copy())
        Am = P.CSR(A.n, A.rowptr, A.col, A.val.copy())
        Ap.val[k] += h
        Am.val[k] -= h
        fd = (loss(Ap, b, xt) - loss(Am, b, xt)) / (2 * h)
        assert abs(fd - gv[k]) <= 1e-5 * abs(gv[k]) + 1e-8


def test_field_generator_matches_definition():
    n = 6
    st = P.cd2d_field(n, seed=1)
    A = P.stencil_to_csr(st).to_dense()
    h = 1.0 / (n + 1)
    c = 25.0 * (P.splitmix64_uniform(1 ^ 0xC0FFEE, n * n) + 1.0)
    assert np.all((c >= 0) & (c <= 50))
    r = 2 + n * 3
    assert A[r, r] == (2.0 + h * c[r]) + (2.0 + h * c[r])
    assert A[r, r - 1] == -1.0 - h * c[r] and A[r, r - n] == -1.0 - h * c[r]
    assert A[r, r + 1] == -1.0 and A[r, r + n] == -1.0
