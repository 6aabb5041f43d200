"""Pins of the mixed-precision refinement oracle (CPU only)."""
import numpy as np
import pytest

import oracle
from oracle import mixed
from paper_1612_01395_gb300 import problems as P


def bf16_round(v):
    """Round float32 values to bfloat16 (nearest even), kept in float32."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def cd2d_64():
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    xs = P.splitmix64_uniform(0, A.n)
    return A, xs, oracle.spmv(A, xs)


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625], dtype=np.float32)
    np.testing.assert_array_equal(bf16_round(x), np.array([1.0, 1.0, 1.0 + 2 ** -7, -3.140625], dtype=np.float32))


def test_fp32_inner_solve_reduces_residual_to_inner_tolerance():
    A, xs, b = cd2d_64()
    A32 = __import__("scipy.sparse", fromlist=["csr_matrix"]).csr_matrix(
        (A.val.astype(np.float32), A.col, A.rowptr), shape=(A.n, A.n))
    d, its = mixed.pbicgstab_f32(A32, b.astype(np.float32), 1e-4, 1000)
    rel = np.linalg.norm(b - oracle.spmv(A, d.astype(np.float64))) / np.linalg.norm(b)
    assert its < 200
    assert rel < 1e-3        # FP32 operator and vectors: close to the inner tolerance


def test_refinement_reaches_1e10_and_matches_fp64_solution():
    """Iterative refinement with an FP32 inner solve reaches an FP64 true residual of
    1e-10, and its solution agrees with the FP64 oracle's to kappa-level accuracy."""
    A, xs, b = cd2d_64()
    res = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3)
    assert res["rel_res_true"] <= 1e-10
    assert 2 <= res["outer"] <= 6
    assert np.all(np.diff(res["history"]) < 0)
    ref = oracle.pbicgstab(A, b, rtol=1e-12, maxit=2000, replace_period=20)
    err = np.linalg.norm(res["x"] - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-7
    assert np.linalg.norm(res["x"] - xs) / np.linalg.norm(xs) <= 1e-7


def test_fp32_inner_accuracy_limits_each_step():
    """An inner tolerance below what FP32 can attain (~1e-4 here) does not pay:
    inner solves run to their iteration cap, the outer history loses monotonicity."""
    A, xs, b = cd2d_64()
    tight = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-4, inner_maxit=1000)
    loose = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3, inner_maxit=1000)
    assert loose["inner_iters"] < tight["inner_iters"]


def test_refinement_with_exact_values_equals_one_fp64_like_step_count():
    """Inner tolerance 1e-12 with FP32 arithmetic still needs several steps: FP32
    limits each inner solve to about 1e-6 relative accuracy."""
    A, xs, b = cd2d_64()
    res = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-12, inner_maxit=300)
    assert res["rel_res_true"] <= 1e-10
    assert res["outer"] >= 2


def test_bf16_values_on_a_well_conditioned_system():
    """BF16 matrix values perturb A by ~2^-9; refinement still converges when
    kappa(A) * 2^-9 < 1 (diagonally dominant random system)."""
    A = P.random_sparse(2000, seed=5)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    res = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3, values32=bf16_round(A.val.astype(np.float32)))
    assert res["rel_res_true"] <= 1e-10
    assert res["outer"] <= 10


def test_lowp_algorithm9_in_float64_matches_the_c_oracle():
    """pbicgstab_lowp is generic in the working type. In float64 it is plain
    Algorithm 9 and must follow the C oracle's Algorithm 9 (itself pinned to
    exact rational arithmetic) to rounding over 20 iterations. The two sum
    their dot products in different orders (numpy pairwise, C left to right),
    and BiCGStab amplifies such differences: on the 64^2 system the C oracle's
    own Algorithms 7 and 9 differ by 4e-11 at iteration 20 and by < 1e-12
    through iteration 12. So the bars are 1e-12 through iteration 12 and 1e-9
    to iteration 20 (the random system converges faster, so its relative
    residuals amplify sooner: 1e-12 through 6, 1e-9 through 10). A wrong
    coefficient in any recurrence or in the alpha denominator of eq. (3)
    moves the history by O(1) within two iterations."""
    import scipy.sparse as sp
    for A, k_tight, k_loose in ((cd2d_64()[0], 12, 20), (P.random_sparse(500, seed=3), 6, 10)):
        b = oracle.spmv(A, P.splitmix64_uniform(1, A.n))
        A64 = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
        x, its, hist = mixed.pbicgstab_lowp(A64, b.copy(), 0.0, 20, fixed_iters=20)
        ref = oracle.pbicgstab(A, b, rtol=0.0, maxit=20, fixed_iters=20)
        assert its == 20 and hist.size == 21
        rel = np.abs(hist - ref.hist) / ref.hist
        assert np.all(rel[:k_tight + 1] <= 1e-12), rel
        assert np.all(rel[:k_loose + 1] <= 1e-9), rel
        ref10 = oracle.pbicgstab(A, b, rtol=0.0, maxit=k_tight, fixed_iters=k_tight)
        x10, _, _ = mixed.pbicgstab_lowp(A64, b.copy(), 0.0, k_tight, fixed_iters=k_tight)
        assert np.linalg.norm(x10 - ref10.x) / np.linalg.norm(ref10.x) <= 1e-12


def test_lowp_algorithm9_float32_stays_near_float64_early():
    """The float32 run is the same algorithm: its first iterations agree with
    the float64 run to a few FP32 roundings (the two drift apart later, as any
    two rounding orders of BiCGStab do)."""
    import scipy.sparse as sp
    A, xs, b = cd2d_64()
    A64 = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    A32 = sp.csr_matrix((A.val.astype(np.float32), A.col, A.rowptr), shape=(A.n, A.n))
    _, _, h64 = mixed.pbicgstab_lowp(A64, b.copy(), 0.0, 5, fixed_iters=5)
    _, _, h32 = mixed.pbicgstab_lowp(A32, b.astype(np.float32), 0.0, 5, fixed_iters=5)
    assert np.max(np.abs(h32 - h64) / h64) <= 1e-4


def test_refinement_stops_when_it_does_not_contract():
    """With the low-precision values negated, each inner solve returns about
    -A^{-1} r, so the FP64 residual doubles every step (r + A A^{-1} r = 2 r).
    The refinement stops after `stall_limit` steps without progress, with
    status NOT_CONVERGED, and returns the best iterate: x0 = 0 itself,
    residual ratio 1."""
    A, xs, b = cd2d_64()
    for limit in (2, 6):
        res = mixed.refine(A, b, rtol=1e-10, inner_rtol=1e-3, values32=-A.val.astype(np.float32), stall_limit=limit)
        assert res["status"] == oracle.NOT_CONVERGED
        assert res["outer"] == limit and res["restored"]
        np.testing.assert_allclose(res["history"] / res["history"][0], 2.0 ** np.arange(limit + 1), rtol=1e-3)
        assert np.all(res["x"] == 0.0)
        assert res["rel_res_true"] == 1.0


def test_refinement_with_fixed_inner_iterations():
    """inner_fixed runs every inner solve for exactly that many iterations and
    records the first one's residual history (entry 0 = ||fl32(b)||)."""
    A, xs, b = cd2d_64()
    res = mixed.refine(A, b, rtol=1e-10, max_outer=3, inner_fixed=7)
    assert res["inner_iters"] == 7 * res["outer"]
    h = res["inner_history"]
    assert h.size == 8
    assert h[0] == pytest.approx(np.linalg.norm(b.astype(np.float32).astype(np.float64)), rel=1e-15)
