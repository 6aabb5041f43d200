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


# Parity of the FP32 inner solve, step by step. Two correct FP32 runs of
# Algorithm 9 that round differently (the oracle's numpy float32 updates and a
# variant with fused multiply-adds, like the kernel's) were measured to differ
# in ||r_i|| by at most 3e-6 relative through iteration 6 and 9e-4 through
# iteration 10 on the 64^2, 20^3, 21^3, 32^3, 48^3 and random 3001-row
# systems, and by 1e-2 to 2 by iterations 15-25: FP32 BiCGStab amplifies
# roundings as FP64 does, from a 2^29 times larger start. So the FP32 parity
# horizon is 10 iterations, with bars 1e-4 through iteration 6 and 1e-2
# through 10 (>= 10x the measured spread); a wrong coefficient moves the
# history by O(1) within two iterations. The GPU's inner dot products
# (compensated FP32) equal the oracle's FP64 sums to ~2^-48. Stencil handles
# use their coefficient tables rounded to FP32 and a summed coefficient added
# in FP32, which can differ from the rounded CSR value by one FP32 ulp: a
# perturbation of the size of the roundings, within the same bars.
INNER_K = 10
INNER_TOL_EARLY, INNER_K_EARLY = 1e-4, 6
INNER_TOL = 1e-2


@pytest.mark.parametrize("name,form", [("cd2d_64", "csr"), ("cd3d_20", "csr"), ("rand_3001", "csr"),
                                       ("cd2d_64", "stencil"), ("cd3d_20", "stencil"), ("cd3d_21", "stencil")])
def test_inner_fp32_history_matches_oracle_per_iteration(name, form):
    import scipy.sparse as sp
    import torch
    if form == "stencil":
        st = STENCILS[name]()
        A = P.stencil_to_csr(st)
        s = native.Solver.from_stencil(st)
        v32 = None
    else:
        A = systems()[name]
        s = native.Solver.from_csr(A)
        v32 = dev(A.val).to(torch.float32)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    x, info, ih = s.solve_mixed(dev(b), v32, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=1, inner_rtol=0.0,
                                inner_maxit=INNER_K, fixed_iters=INNER_K, inner_history=True)
    assert info["outer"] == 1 and info["inner_iters"] == INNER_K, info
    A32 = sp.csr_matrix((A.val.astype(np.float32), A.col, A.rowptr), shape=(A.n, A.n))
    d, its, ref = mixed.pbicgstab_lowp(A32, b.astype(np.float32), 0.0, INNER_K, fixed_iters=INNER_K)
    h = ih.cpu().numpy()
    assert h.size == INNER_K + 1
    assert h[0] == pytest.approx(ref[0], rel=1e-12)   # ||fl32(b)||, an FP64-grade sum on both sides
    rel = np.abs(h - ref) / ref
    assert np.all(rel[:INNER_K_EARLY + 1] <= INNER_TOL_EARLY), rel
    assert np.all(rel <= INNER_TOL), rel
    # the step's correction: x = x0 + d with x0 = 0, i.e. the inner solution in FP64
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - d.astype(np.float64)) / np.linalg.norm(d) <= INNER_TOL
    s.close()


def test_refinement_that_does_not_contract_stops_with_best_iterate():
    """Negated FP32 values make every inner solve return about -A^{-1} r, so
    the FP64 residual doubles each step. The solve must stop after
    `stall_steps` steps without progress (PBCG_NOT_CONVERGED), return the best
    iterate -- x0 = 0 itself, bit for bit -- and report its residual ratio 1.
    The oracle's refinement takes the same decisions."""
    import torch
    A = systems()["cd2d_64"]
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_csr(A)
    vneg = dev(-A.val).to(torch.float32)
    for steps in (2, 0):   # 0: the default, 6
        x, info, hist = s.solve_mixed(dev(b), vneg, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=30,
                                      inner_rtol=1e-3, inner_maxit=2000, history=True, stall_steps=steps)
        limit = steps or 6
        assert info["status"] == native.PBCG_NOT_CONVERGED, info
        assert info["outer"] == limit and info["restored"] == 1, info
        assert info["rel_res_true"] == 1.0
        assert torch.count_nonzero(x).item() == 0
        h = hist.cpu().numpy()
        np.testing.assert_allclose(h / h[0], 2.0 ** np.arange(limit + 1), rtol=1e-3)
        ref = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3, inner_maxit=2000, values32=-A.val.astype(np.float32),
                           stall_limit=limit)
        assert ref["status"] == oracle.NOT_CONVERGED and ref["outer"] == info["outer"] and ref["restored"]
    # from a nonzero start the returned x is that start, bit for bit
    x0 = dev(P.splitmix64_uniform(7, A.n))
    x, info = s.solve_mixed(dev(b), vneg, native.PBCG_VALUES_F32, x0=x0, rtol=1e-10, max_outer=30,
                            inner_rtol=1e-3, inner_maxit=2000)
    assert info["status"] == native.PBCG_NOT_CONVERGED and info["restored"] == 1
    assert torch.equal(x, x0)
    s.close()


def test_converging_refinement_is_not_stopped_by_the_stall_rule():
    """On a system where refinement contracts, the stall rule never fires:
    the same result as the oracle's refinement (status, step count within 2)."""
    import torch
    A = P.stencil_to_csr(P.cd3d_trig(24))
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_csr(A)
    v16 = dev(A.val).to(torch.bfloat16)
    x, info = s.solve_mixed(dev(b), v16, native.PBCG_VALUES_BF16, rtol=1e-10, max_outer=40, inner_rtol=1e-2,
                            inner_maxit=150)
    assert info["status"] == native.PBCG_OK and info["restored"] == 0, info
    true_rel = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    s.close()


def tiny_stencil(nx, ny, nz):
    if nz == 1 and ny == nx and nx > 1:
        return P.cd2d_constant(nx, (10.0, 10.0))
    if nx == ny == nz:
        return P.cd3d_trig(nx)
    return P.convection_diffusion((nx, ny, nz), (np.full(ny, 20.0), np.full(nz, 5.0), np.full(nx, 10.0)))


@pytest.mark.parametrize("dims", [(3, 1, 1), (7, 1, 1), (2, 2, 1), (3, 3, 1), (2, 2, 2), (3, 3, 3), (5, 5, 5),
                                  (9, 9, 1)])
def test_mixed_stencil_tiny_and_ragged_tiles(dims):
    """The staged FP32 sweeps copy tiles of 256 rows rounded up to 16 bytes:
    systems of 3 to 125 rows have a single partial tile, odd tails and x-lines
    of odd length (so row pairs fall back to single rows). Each must reach a
    1e-10 true residual (recomputed by the oracle's SpMV) and agree with the
    oracle's FP64 solution."""
    st = tiny_stencil(*dims)
    A = P.stencil_to_csr(st)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_stencil(st)
    x, info = s.solve_mixed(dev(b), None, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=30, inner_rtol=1e-3,
                            inner_maxit=200)
    assert info["status"] == native.PBCG_OK, info
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - oracle.spmv(A, xg)) <= 1e-10 * np.linalg.norm(b)
    ref = oracle.pbicgstab(A, b, rtol=1e-13, maxit=2000, replace_period=20)
    assert np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    s.close()
