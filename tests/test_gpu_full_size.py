"""Parity at the full benchmark size: 3-D convection-diffusion on a 256^3 grid
(16,777,216 unknowns), velocity (20 sin y, 20 cos z, 20 sin x), stencil and CSR
forms, in the launch configuration the benchmark uses (automatic grid).

The oracle cannot run a whole solve at this size in test time, so the checks
are: every SpMV row against the oracle; the first 20 iterations step by step
(the parity horizon: residual norms within 1e-8 and x within 1e-9 of the
oracle), without residual replacement and with replacement every 5
iterations (4 replacements inside the window, so the replacement path is
compared at full size too); and, for complete solves, the true residual of
the returned x recomputed by the oracle's SpMV.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu

N1D = 256


@pytest.fixture(scope="module")
def cd3d_256():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()
    st = P.cd3d_trig(N1D)
    A = P.stencil_to_csr(st)
    xs = P.splitmix64_uniform(0, A.n)
    b = oracle.spmv(A, xs)
    return st, A, xs, b


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_full_size_spmv_rows(cd3d_256):
    st, A, xs, b = cd3d_256
    ss = native.Solver.from_stencil(st)
    sc = native.Solver.from_csr(A)
    xd = dev(xs)
    ys = ss.spmv(xd).cpu().numpy()
    yc = sc.spmv(xd).cpu().numpy()
    np.testing.assert_array_equal(ys, yc)
    np.testing.assert_allclose(ys, b, rtol=1e-14, atol=1e-14 * np.max(np.abs(b)))
    ss.close()
    sc.close()


K = 20
_ORACLE = {}


def oracle_window(A, b, rr):
    """The oracle's first K iterations (cached: about 10 s each at this size)."""
    if rr not in _ORACLE:
        _ORACLE[rr] = oracle.pbicgstab(A, b, rtol=0.0, maxit=K, fixed_iters=K, replace_period=rr)
    return _ORACLE[rr]


@pytest.mark.parametrize("rr", [0, 5])
@pytest.mark.parametrize("form", ["stencil", "csr"])
def test_full_size_first_iterations(cd3d_256, form, rr):
    st, A, xs, b = cd3d_256
    ref = oracle_window(A, b, rr)
    assert ref.n_replacements == (K // rr if rr else 0)
    s = native.Solver.from_stencil(st) if form == "stencil" else native.Solver.from_csr(A)
    x, info, hist = s.solve(dev(b), rtol=0.0, maxit=K, fixed_iters=K, replace_period=rr, history=True)
    assert info["status"] == native.PBCG_OK
    assert info["n_replacements"] == ref.n_replacements
    h = hist.cpu().numpy()
    assert h.size == K + 1
    xg = x.cpu().numpy()
    tol = 1e-8 * ref.hist + 1e-13 * ref.nr0
    if rr and K % rr == 0:
        # r_K was replaced by the true residual of x_K: two x_K that differ by
        # dx have true residuals that differ by up to ||A dx|| (triangle
        # inequality), computed here with the oracle's SpMV
        tol[-1] += np.linalg.norm(oracle.spmv(A, xg - ref.x))
    assert np.all(np.abs(h - ref.hist) <= tol), np.abs(h - ref.hist) / ref.hist
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-9
    s.close()


@pytest.mark.parametrize("method,rr", [("pipelined", 50), ("standard", 0)])
def test_full_size_solve_reaches_tolerance(cd3d_256, method, rr):
    st, A, xs, b = cd3d_256
    s = native.Solver.from_stencil(st)
    x, info = s.solve(dev(b), rtol=1e-8, maxit=5000, replace_period=rr, method=method)
    assert info["status"] == native.PBCG_OK, info
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(b - oracle.spmv(A, xg)) / np.linalg.norm(b)
    assert true_rel <= 1e-8, (true_rel, info)
    s.close()
