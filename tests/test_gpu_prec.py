"""Jacobi-preconditioned solves on the GPU (Algorithms 10 and 11) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu

X_TOL, HIST_TOL, HIST_FLOOR = 1e-9, 1e-8, 1e-13


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def scaled_random(n=3001, seed=5):
    """Random sparse system with rows scaled over 4 decades (Jacobi matters)."""
    A = P.random_sparse(n, seed=seed)
    scale = 10.0 ** (4 * P.splitmix64_uniform(8, A.n) ** 2)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    A.val = A.val * scale[rows]
    return None, A


def problem(name):
    if name == "cd2d_64":
        st = P.cd2d_constant(64, (10.0, 10.0))
        return st, P.stencil_to_csr(st)
    if name == "cd3d_20":
        st = P.cd3d_trig(20)
        return st, P.stencil_to_csr(st)
    return scaled_random()


def make(name, form):
    st, A = problem(name)
    if form == "stencil":
        if st is None:
            pytest.skip("no stencil form")
        return native.Solver.from_stencil(st, prec=native.PBCG_PREC_JACOBI), A
    return native.Solver.from_csr(A, prec=native.PBCG_PREC_JACOBI), A


@pytest.mark.parametrize("name", ["cd2d_64", "cd3d_20", "scaled_rand"])
@pytest.mark.parametrize("form", ["csr", "stencil"])
@pytest.mark.parametrize("method", ["pipelined", "standard"])
@pytest.mark.parametrize("grid", [0, 1024], ids=["default_grid", "grid1024"])
def test_preconditioned_first_iterations_match_oracle(name, form, method, grid):
    """grid 1024: the reductions go through the last block to arrive (512
    blocks and more)."""
    s, A = make(name, form)
    minv = oracle.jacobi_minv(A)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    fn = oracle.pbicgstab_prec if method == "pipelined" else oracle.bicgstab_prec
    ref = fn(A, minv, b, rtol=1e-8, maxit=3000)
    assert ref.status == oracle.CONVERGED
    k = min(20, ref.iters - (1 if ref.half_step else 0))
    fx = fn(A, minv, b, rtol=0.0, maxit=k, fixed_iters=k)
    x, info, hist = s.solve(dev(b), rtol=0.0, maxit=k, fixed_iters=k, history=True, method=method, grid=grid)
    assert info["status"] == native.PBCG_OK and info["iters"] == k
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - fx.x) / np.linalg.norm(fx.x) <= X_TOL
    h = hist.cpu().numpy()
    assert np.all(np.abs(h - fx.hist) <= HIST_TOL * fx.hist + HIST_FLOOR * fx.nr0)
    s.close()


@pytest.mark.parametrize("name", ["cd2d_64", "scaled_rand"])
@pytest.mark.parametrize("method", ["pipelined", "standard"])
def test_preconditioned_final_solution_matches_oracle(name, method):
    s, A = make(name, "csr")
    minv = oracle.jacobi_minv(A)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    if method == "pipelined":
        ref = oracle.pbicgstab_prec(A, minv, b, rtol=1e-12, maxit=3000, replace_period=20)
        x, info = s.solve(dev(b), rtol=1e-12, maxit=3000, replace_period=20)
    else:
        ref = oracle.bicgstab_prec(A, minv, b, rtol=1e-12, maxit=3000)
        x, info = s.solve(dev(b), rtol=1e-12, maxit=3000, method="standard")
    assert info["status"] == native.PBCG_OK
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= X_TOL
    s.close()


def test_preconditioned_replacement_matches_oracle():
    s, A = make("cd2d_64", "stencil")
    minv = oracle.jacobi_minv(A)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    fx = oracle.pbicgstab_prec(A, minv, b, rtol=0.0, maxit=12, fixed_iters=12, replace_period=4)
    x, info = s.solve(dev(b), rtol=0.0, maxit=12, fixed_iters=12, replace_period=4)
    assert info["n_replacements"] == fx.n_replacements == 3
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - fx.x) / np.linalg.norm(fx.x) <= X_TOL
    s.close()


def test_jacobi_reduces_iterations_on_scaled_rows():
    _, A = scaled_random()
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    plain = native.Solver.from_csr(A)
    prec = native.Solver.from_csr(A, prec=native.PBCG_PREC_JACOBI)
    _, i0 = plain.solve(dev(b), rtol=1e-10, maxit=5000)
    _, i1 = prec.solve(dev(b), rtol=1e-10, maxit=5000)
    assert i1["status"] == native.PBCG_OK
    assert i1["iters"] < i0["iters"]


def test_zero_diagonal_rejected():
    import torch
    A = P.dense_to_csr(np.array([[0.0, 1.0], [1.0, 0.0]]))
    with pytest.raises(native.PbcgError) as e:
        native.Solver.from_csr(A, prec=native.PBCG_PREC_JACOBI)
    assert e.value.status == native.PBCG_ERR_ARG
