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
