"""CSR rows of every length through both CSR operator forms (needs a GB300).

The library takes a row's entries one at a time when the matrix averages at
most 6 entries per row, and 7 at a time (the last chunk of a row partial)
otherwise. Either way a row of A x is one chain of fused multiply-adds in
storage order, acc = fma(a_k, x_col(k), acc) from acc = 0, as the library
states. That chain has one exact value, computed here with
rational arithmetic and one rounding per step, so the GPU products are
compared bit for bit. Row lengths cover empty rows, rows shorter than a
chunk, exactly one and two chunks, and one entry either side of a chunk
boundary.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def ragged_csr(lengths, n, seed):
    """CSR with the given row lengths, distinct sorted random columns in
    [0, n), and values from SplitMix64 uniforms in [-1, 1)."""
    rng = np.random.default_rng(seed)
    rowptr = np.zeros(len(lengths) + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lengths)
    cols = [np.sort(rng.choice(n, size=k, replace=False)) for k in lengths]
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = P.splitmix64_uniform(seed, int(rowptr[-1]))
    return P.CSR(n=len(lengths), rowptr=rowptr.astype(np.int32), col=col, val=val)


def fma_chain(A, x):
    """Each row as a chain of correctly rounded fused multiply-adds."""
    y = np.zeros(A.n)
    for r in range(A.n):
        acc = 0.0
        for k in range(A.rowptr[r], A.rowptr[r + 1]):
            acc = float(Fraction(A.val[k]) * Fraction(x[A.col[k]]) + Fraction(acc))
        y[r] = acc
    return y


@pytest.mark.parametrize("lengths_of, chunked", [
    (lambda i: [0, 1, 2, 5, 6, 7, 8, 13, 14, 15, 21, 40][i % 12], True),   # average 11: 7 at a time
    (lambda i: [0, 1, 3, 5, 6, 7, 8, 2][i % 8], False),                    # average 4: one at a time
])
def test_spmv_rows_are_storage_order_fma_chains(lengths_of, chunked):
    import torch
    n = 1501   # odd, several warps and blocks, ragged last warp
    lengths = [lengths_of(i) for i in range(n)]
    A = ragged_csr(lengths, n, seed=23)
    assert (len(A.val) > 6 * n) == chunked
    s = native.Solver.from_csr(A)
    x = P.splitmix64_uniform(29, n)
    y = s.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    s.close()
    np.testing.assert_array_equal(y, fma_chain(A, x))
