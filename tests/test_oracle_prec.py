"""Pins of the preconditioned oracle (Algorithms 10 and 11, Jacobi M = diag(A)), CPU only."""
from fractions import Fraction

import numpy as np
import pytest
import sympy

import oracle
from oracle import rational as Q
from paper_1612_01395_gb300 import problems as P
from test_oracle_exact import SYSTEMS, HEALTHY, as_float


def exact_minv(a):
    return [Fraction(1, int(a[i, i])) for i in range(a.shape[0])]


@pytest.mark.parametrize("idx", range(len(SYSTEMS)))
def test_preconditioned_variants_identical_in_exact_arithmetic(idx):
    """Right preconditioning does not change the iterates x_i of Alg. 10 vs Alg. 11
    (with or without replacement), and M = I turns Alg. 10 into Alg. 7."""
    a, b = SYSTEMS[idx]
    if np.any(np.diag(a) == 0):
        pytest.skip("zero diagonal")
    A, bl, n = a.tolist(), b.tolist(), len(b)
    minv = exact_minv(a)
    ref = Q.bicgstab_prec(A, minv, bl, maxit=3 * n)
    if ref["status"] != "converged":
        pytest.skip("breakdown in exact arithmetic")
    for run in (Q.pbicgstab_prec(A, minv, bl, maxit=3 * n),
                Q.pbicgstab_prec(A, minv, bl, maxit=3 * n, replace_period=1),
                Q.pbicgstab_prec(A, minv, bl, maxit=3 * n, replace_period=2)):
        assert run["status"] == ref["status"] and run["half_step"] == ref["half_step"]
        assert run["x"] == ref["x"] and run["r"] == ref["r"]
    # the exact solution of A x = b
    xs = sympy.Matrix(A).LUsolve(sympy.Matrix(bl))
    assert [sympy.Rational(v.numerator, v.denominator) for v in ref["x"][-1]] == list(xs)
    ident = [Fraction(1)] * n
    assert Q.bicgstab_prec(A, ident, bl, maxit=3 * n)["x"] == Q.bicgstab(A, bl, maxit=3 * n)["x"]
    assert Q.pbicgstab_prec(A, ident, bl, maxit=3 * n)["x"] == Q.pbicgstab(A, bl, maxit=3 * n)["x"]


@pytest.mark.parametrize("idx", range(len(HEALTHY)))
@pytest.mark.parametrize("method", ["bicgstab_prec", "pbicgstab_prec"])
def test_fp64_preconditioned_oracle_matches_rational(idx, method):
    a, b = HEALTHY[idx]
    if np.any(np.diag(a) == 0):
        pytest.skip("zero diagonal")
    n = len(b)
    exact = getattr(Q, method)(a.tolist(), exact_minv(a), b.tolist(), maxit=3 * n)
    if exact["status"] != "converged":
        pytest.skip("breakdown")
    steps = len(exact["x"]) - 1 - (1 if exact["half_step"] else 0)
    if steps < 1:
        pytest.skip("terminates immediately")
    A = P.dense_to_csr(a.astype(float))
    res = getattr(oracle, method)(A, oracle.jacobi_minv(A), b.astype(float), fixed_iters=steps, trace=True)
    xq = as_float(exact["x"][: steps + 1])
    np.testing.assert_allclose(res.trace_x, xq, rtol=0, atol=1e-10 * np.max(np.abs(xq)))


def test_identity_preconditioner_reproduces_unpreconditioned_bitwise():
    """With M^{-1} = I every hat vector is a bit-exact copy of its plain twin, so
    Alg. 11 repeats Alg. 9 and Alg. 10 repeats Alg. 7 bit for bit."""
    A = P.stencil_to_csr(P.cd2d_constant(32, (10.0, 10.0)))
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    one = np.ones(A.n)
    for k in (0, 7):
        r9 = oracle.pbicgstab(A, b, rtol=1e-10, maxit=500, replace_period=k)
        r11 = oracle.pbicgstab_prec(A, one, b, rtol=1e-10, maxit=500, replace_period=k)
        assert r9.iters == r11.iters
        np.testing.assert_array_equal(r9.x, r11.x)
    r7 = oracle.bicgstab(A, b, rtol=1e-10, maxit=500)
    r10 = oracle.bicgstab_prec(A, one, b, rtol=1e-10, maxit=500)
    np.testing.assert_array_equal(r7.x, r10.x)


@pytest.mark.parametrize("method", ["bicgstab_prec", "pbicgstab_prec"])
def test_preconditioned_solution_matches_dense_lu(method):
    A = P.random_sparse(300, seed=2)
    b = P.splitmix64_uniform(4, A.n)
    x_lu = np.linalg.solve(A.to_dense(), b)
    res = getattr(oracle, method)(A, oracle.jacobi_minv(A), b, rtol=1e-13, maxit=500)
    assert res.status == oracle.CONVERGED
    assert np.linalg.norm(res.x - x_lu) / np.linalg.norm(x_lu) <= 1e-11


def test_jacobi_helps_on_badly_scaled_rows():
    """Rows scaled by factors spanning 1e4: Jacobi removes the scaling."""
    A = P.random_sparse(500, seed=3)
    scale = 10.0 ** (4 * P.splitmix64_uniform(8, A.n) ** 2)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    A.val = A.val * scale[rows]
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    plain = oracle.pbicgstab(A, b, rtol=1e-10, maxit=2000)
    prec = oracle.pbicgstab_prec(A, oracle.jacobi_minv(A), b, rtol=1e-10, maxit=2000)
    assert prec.status == oracle.CONVERGED
    assert prec.iters < plain.iters


def test_preconditioned_replacement_restores_accuracy():
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    minv = oracle.jacobi_minv(A)
    plain = oracle.bicgstab_prec(A, minv, b, rtol=1e-14, maxit=600)
    pipe = oracle.pbicgstab_prec(A, minv, b, rtol=1e-14, maxit=600)
    rr = oracle.pbicgstab_prec(A, minv, b, rtol=1e-14, maxit=600, replace_period=20)
    assert pipe.rel_res_true > 100 * plain.rel_res_true
    assert rr.status == oracle.CONVERGED and rr.rel_res_true < 10 * max(plain.rel_res_true, 1e-14)
