"""Parity of the extensions at their full benchmark sizes (needs a GB300).

* Mixed precision: 3-D convection-diffusion on a 192^3 grid (7,077,888
  unknowns), stencil and CSR forms, FP32 inner Algorithm 9 with inner
  tolerance 0.1 and cap 50 inside FP64 refinement to a true relative residual
  of 1e-10 -- the benchmark's first mixed-precision setting, on the default
  grid.
* Batched: the benchmark's 512 random sparse systems (7,745,785 rows) in one
  launch with the default launch shape, each to rtol 1e-8.

The oracle cannot solve these in test time; the checks are properties that
hold at any size: the true residual of every returned solution, recomputed
with the oracle's FP64 SpMV, and for the mixed solve the distance to the
library's FP64 p-BiCGStab solution, bounded by the condition of the problem
times the residual.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def cd3d_192():
    st = P.cd3d_trig(192)
    A = P.stencil_to_csr(st)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    return st, A, b


@pytest.mark.parametrize("form", ["stencil", "csr"])
def test_full_size_mixed_precision(cd3d_192, form):
    import torch
    st, A, b = cd3d_192
    s = native.Solver.from_stencil(st) if form == "stencil" else native.Solver.from_csr(A)
    v32 = None if form == "stencil" else dev(A.val).to(torch.float32)
    bd = dev(b)
    x, info = s.solve_mixed(bd, v32, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=60, inner_rtol=0.1,
                            inner_maxit=50)
    assert info["status"] == native.PBCG_OK, info
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(b - oracle.spmv(A, xg)) / np.linalg.norm(b)
    assert true_rel <= 1e-10, (true_rel, info)
    x64, i64 = s.solve(bd, rtol=1e-10, maxit=5000, replace_period=50)
    assert i64["status"] == native.PBCG_OK
    x64 = x64.cpu().numpy()
    assert np.linalg.norm(xg - x64) / np.linalg.norm(x64) <= 1e-6
    s.close()


def test_full_size_batched():
    B = P.random_batch(nsys=512, seed=0)
    bs = native.BatchSolver(B)
    bd = dev(B.b)
    x = bd.new_zeros(bd.shape)
    bs.launch(bd, x, rtol=1e-8, maxit=1000)
    r = bs.fetch_results()
    assert np.all(r["status"] == native.PBCG_OK)
    xg = x.cpu().numpy()
    worst = 0.0
    for k in range(B.nsys):
        r0, r1 = int(B.row_offset[k]), int(B.row_offset[k + 1])
        e0, e1 = int(B.rowptr[r0]), int(B.rowptr[r1])
        A = P.CSR(n=r1 - r0, rowptr=(B.rowptr[r0:r1 + 1] - e0).astype(np.int32), col=B.col[e0:e1],
                  val=B.val[e0:e1])
        bk = B.b[r0:r1]
        rel = np.linalg.norm(bk - oracle.spmv(A, xg[r0:r1])) / np.linalg.norm(bk)
        worst = max(worst, rel)
        # the library's own record of the true residual agrees with the oracle's
        assert abs(rel - r["rel_res_true"][k]) <= 1e-3 * rel + 1e-15
    assert worst <= 1e-8, worst
    del bs
