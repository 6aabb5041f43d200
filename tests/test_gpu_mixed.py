"""Mixed precision on the GPU: FP64 refinement around FP32 Algorithm 9 (needs a GB300).

Checked by the FP64 oracle: the true residual of the returned x is recomputed by
the oracle's FP64 SpMV, and the solution is compared with the oracle's FP64
solution of a tight solve; the error against it is the stated accuracy of the
mixed-precision result.
"""
import numpy as np
import pytest

import oracle
from oracle import mixed
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


def systems():
    return {"cd2d_64": P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0))),
            "cd3d_20": P.stencil_to_csr(P.cd3d_trig(20)),
            "rand_3001": P.random_sparse(3001, seed=5)}


@pytest.mark.parametrize("name", ["cd2d_64", "cd3d_20", "rand_3001"])
def test_mixed_fp32_reaches_1e10_true_residual(name):
    import torch
    A = systems()[name]
    xs = P.splitmix64_uniform(0, A.n)
    b = oracle.spmv(A, xs)
    s = native.Solver.from_csr(A)
    v32 = dev(A.val).to(torch.float32)
    x, info, hist = s.solve_mixed(dev(b), v32, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=30,
                                  inner_rtol=1e-3, inner_maxit=2000, history=True)
    assert info["status"] == native.PBCG_OK, info
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(b - oracle.spmv(A, xg)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    assert abs(true_rel - info["rel_res_true"]) <= 1e-2 * true_rel + 1e-16
    h = hist.cpu().numpy()
    assert h[-1] <= 1e-10 * h[0]
    # accuracy against the FP64 oracle's solution of a tight solve
    ref = oracle.pbicgstab(A, b, rtol=1e-12, maxit=3000, replace_period=20)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    # the refinement takes a similar number of steps as the numpy/float32 oracle
    mo = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3, inner_maxit=2000)
    assert abs(info["outer"] - mo["outer"]) <= 2
    s.close()


def test_mixed_bf16_values_converge_on_well_conditioned_system():
    import torch
    A = systems()["rand_3001"]
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_csr(A)
    v16 = dev(A.val).to(torch.bfloat16)
    x, info = s.solve_mixed(dev(b), v16, native.PBCG_VALUES_BF16, rtol=1e-10, max_outer=30, inner_rtol=1e-3)
    assert info["status"] == native.PBCG_OK, info
    true_rel = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    s.close()


STENCILS = {"cd2d_64": lambda: P.cd2d_constant(64, (10.0, 10.0)), "cd3d_20": lambda: P.cd3d_trig(20),
            "cd2d_63": lambda: P.cd2d_constant(63, (10.0, 10.0)), "cd3d_21": lambda: P.cd3d_trig(21)}


@pytest.mark.parametrize("name", list(STENCILS))
def test_mixed_fp32_stencil_form_reaches_1e10_true_residual(name):
    """Stencil handles: the inner solves use the coefficient tables rounded to
    FP32 (a summed coefficient is then added in FP32, so the inner operator can
    differ from the rounded CSR values in the last bit); the FP64 refinement
    still reaches the FP64 solution. Even nx takes the inner sweeps' paired
    rows (one SpMV call per x-line pair), odd nx one call per row."""
    st = STENCILS[name]()
    A = P.stencil_to_csr(st)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_stencil(st)
    x, info = s.solve_mixed(dev(b), None, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=30, inner_rtol=1e-3,
                            inner_maxit=2000)
    assert info["status"] == native.PBCG_OK, info
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(b - oracle.spmv(A, xg)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    ref = oracle.pbicgstab(A, b, rtol=1e-12, maxit=3000, replace_period=20)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    mo = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3, inner_maxit=2000)
    assert abs(info["outer"] - mo["outer"]) <= 2
    s.close()


def test_mixed_on_a_large_grid_is_deterministic_and_converges():
    """1024 blocks on a small system: the reductions go through the last block
    to arrive; two runs give the same bits and reach the FP64 solution."""
    import torch
    A = systems()["cd3d_20"]
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_csr(A)
    v32 = dev(A.val).to(torch.float32)
    kw = dict(rtol=1e-10, max_outer=30, inner_rtol=1e-3, inner_maxit=2000, grid=1024)
    x1, i1 = s.solve_mixed(dev(b), v32, native.PBCG_VALUES_F32, **kw)
    x2, i2 = s.solve_mixed(dev(b), v32, native.PBCG_VALUES_F32, **kw)
    assert i1["status"] == native.PBCG_OK and i1["grid"] == 1024
    np.testing.assert_array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    true_rel = np.linalg.norm(b - oracle.spmv(A, x1.cpu().numpy())) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    s.close()


@pytest.mark.parametrize("grid", [7, 1000])
def test_mixed_odd_size_with_row_pairs_at_block_edges(grid):
    """The FP32 sweeps take rows in aligned pairs and every block's range
    starts on an even row. n = 3001 is odd, so the last row has no partner.
    With 1000 blocks most ranges hold one pair, some none, and the last
    block holds a pair and the lone row; with 7 blocks the ranges are long.
    Both reach the FP64 solution, bit-identically on a repeat."""
    import torch
    A = systems()["rand_3001"]
    b = oracle.spmv(A, P.splitmix64_uniform(3, A.n))
    s = native.Solver.from_csr(A)
    v32 = dev(A.val).to(torch.float32)
    kw = dict(rtol=1e-10, max_outer=30, inner_rtol=1e-3, inner_maxit=2000, grid=grid)
    x1, i1 = s.solve_mixed(dev(b), v32, native.PBCG_VALUES_F32, **kw)
    x2, _ = s.solve_mixed(dev(b), v32, native.PBCG_VALUES_F32, **kw)
    assert i1["status"] == native.PBCG_OK and i1["grid"] == grid, i1
    xg = x1.cpu().numpy()
    np.testing.assert_array_equal(xg, x2.cpu().numpy())
    assert np.linalg.norm(b - oracle.spmv(A, xg)) / np.linalg.norm(b) <= 1e-10
    ref = oracle.pbicgstab(A, b, rtol=1e-12, maxit=3000, replace_period=20)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-7
    s.close()


def test_mixed_rejects_bad_arguments():
    import torch
    s = native.Solver.from_stencil(P.cd2d_constant(16))
    b = torch.ones(256, dtype=torch.float64, device="cuda")
    with pytest.raises(native.PbcgError):   # stencil handles take no values
        s.solve_mixed(b, torch.ones(10, dtype=torch.float32, device="cuda"))
    with pytest.raises(native.PbcgError):   # nor BF16
        s.solve_mixed(b, None, native.PBCG_VALUES_BF16)
    A = P.stencil_to_csr(P.cd2d_constant(16))
    c = native.Solver.from_csr(A)
    st, info = native.pbicgstab_solve_mixed(c.h, dev(A.val).to(torch.float32).data_ptr(), 7, b.data_ptr(),
                                            b.data_ptr(), 1e-10, 10, 1e-3, 100)
    assert st == native.PBCG_ERR_ARG
