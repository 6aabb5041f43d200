"""Pins of the oracle in exact arithmetic (CPU only).

In exact arithmetic Algorithm 7 (BiCGStab), Algorithm 8 (CA-BiCGStab) and
Algorithm 9 (p-BiCGStab) produce identical iterates (Section 3.2, Section 3.3),
alpha by eq. (3) equals alpha by eq. (5), and residual replacement
(Section 4.2) changes nothing. BiCGStab on a nonsingular n x n system without
breakdown reaches the exact solution within n iterations. These facts pin the
rational oracle; the FP64 C oracle is then pinned to the rational iterates.
"""
import numpy as np
import pytest
import sympy

import oracle
from oracle import rational as Q
from paper_1612_01395_gb300 import problems as P


def exact_solution(a, b):
    sol = sympy.Matrix(a.tolist()).LUsolve(sympy.Matrix(b.tolist()))
    return [sympy.Rational(v) for v in sol]


def systems(count=12):
    """Small well-conditioned integer systems that run without breakdown."""
    out = []
    seed = 1
    while len(out) < count:
        n = 3 + seed % 5
        a, b = P.random_integer_system(n, seed, diag_boost=5)
        seed += 1
        if np.linalg.matrix_rank(a) < n or np.linalg.cond(a) > 50:
            continue
        ref = Q.bicgstab(a.tolist(), b.tolist(), maxit=3 * n)
        if ref["status"] != "converged":
            continue
        out.append((a, b))
    return out


SYSTEMS = systems()


def healthy(a, b):
    """No near-breakdown: every squared cosine of (r0, s_i) and (q_i, y_i) in the
    exact BiCGStab run is at least 1e-4, so FP64 rounding is not amplified."""
    run = Q.bicgstab(a.tolist(), b.tolist(), maxit=3 * len(b))
    return all(min(c1, c2) >= 1e-4 for c1, c2 in run["angles"])


HEALTHY = [sb for sb in SYSTEMS if healthy(*sb)]


def as_float(vecs):
    return np.array([[float(e) for e in v] for v in vecs])


@pytest.mark.parametrize("idx", range(len(SYSTEMS)))
def test_variants_identical_in_exact_arithmetic(idx):
    a, b = SYSTEMS[idx]
    A, bl = a.tolist(), b.tolist()
    n = len(bl)
    ref = Q.bicgstab(A, bl, maxit=3 * n)
    runs = {
        "alg8": Q.cabicgstab(A, bl, maxit=3 * n),
        "alg9": Q.pbicgstab(A, bl, maxit=3 * n),
        "alg9_eq5": Q.pbicgstab(A, bl, maxit=3 * n, alpha_eq5=True),
    }
    for k in (1, 2, 3):
        runs[f"alg9_rr{k}"] = Q.pbicgstab(A, bl, maxit=3 * n, replace_period=k)
        runs[f"alg9_rr{k}_late"] = Q.pbicgstab(A, bl, maxit=3 * n, replace_period=k, rr_placement=1)
    for name, run in runs.items():
        assert run["status"] == ref["status"], name
        assert run["half_step"] == ref["half_step"], name
        assert len(run["x"]) == len(ref["x"]), name
        for i, (xa, xb) in enumerate(zip(run["x"], ref["x"])):
            assert xa == xb, f"{name}: x_{i} differs"
        for i, (ra, rb) in enumerate(zip(run["r"], ref["r"])):
            assert ra == rb, f"{name}: r_{i} differs"


@pytest.mark.parametrize("idx", range(len(SYSTEMS)))
def test_exact_termination_at_solution(idx):
    a, b = SYSTEMS[idx]
    n = len(b)
    ref = Q.bicgstab(a.tolist(), b.tolist(), maxit=3 * n)
    assert ref["status"] == "converged"
    # BiCG-type termination: at most n iterations (the last may be a half step)
    assert len(ref["x"]) - 1 <= n
    xs = exact_solution(a, b)
    assert [sympy.Rational(v.numerator, v.denominator) for v in ref["x"][-1]] == xs


def test_replacement_counts_exact():
    """A replacement happens after every k-th completed full iteration."""
    for k in (1, 2, 3):
        for a, b in SYSTEMS[:4]:
            n = len(b)
            run = Q.pbicgstab(a.tolist(), b.tolist(), maxit=3 * n, replace_period=k)
            full = len(run["x"]) - 1 - (1 if run["half_step"] else 0)
            assert run["replacements"] == full // k


def test_enough_healthy_systems():
    assert len(HEALTHY) >= 8


@pytest.mark.parametrize("idx", range(len(HEALTHY)))
@pytest.mark.parametrize("method", ["bicgstab", "cabicgstab", "pbicgstab"])
def test_fp64_oracle_matches_rational(idx, method):
    """The C oracle's FP64 iterates track the exact ones to rounding level on
    systems without a near-breakdown (a near-breakdown amplifies rounding,
    which is a property of the method, not of the code)."""
    a, b = HEALTHY[idx]
    n = len(b)
    exact = getattr(Q, method)(a.tolist(), b.tolist(), maxit=3 * n)
    steps = len(exact["x"]) - 1
    if exact["half_step"]:
        steps -= 1                      # compare full iterations only
    if steps < 1:
        pytest.skip("terminates immediately")
    A = P.dense_to_csr(a.astype(float))
    res = getattr(oracle, method)(A, b.astype(float), fixed_iters=steps, trace=True)
    xq, rq = as_float(exact["x"][: steps + 1]), as_float(exact["r"][: steps + 1])
    scale_x = np.max(np.abs(xq)) + 1e-300
    scale_r = np.linalg.norm(rq[0])
    np.testing.assert_allclose(res.trace_x, xq, rtol=0, atol=1e-10 * scale_x)
    # the last exact residual is zero; compare absolute to ||r_0||
    np.testing.assert_allclose(res.trace_r, rq, rtol=0, atol=1e-10 * scale_r)


def test_fp64_oracle_replacement_matches_rational():
    a, b = HEALTHY[3]
    n = len(b)
    exact = Q.pbicgstab(a.tolist(), b.tolist(), maxit=3 * n, replace_period=2)
    steps = len(exact["x"]) - 1 - (1 if exact["half_step"] else 0)
    A = P.dense_to_csr(a.astype(float))
    res = oracle.pbicgstab(A, b.astype(float), fixed_iters=steps, trace=True, replace_period=2)
    xq = as_float(exact["x"][: steps + 1])
    np.testing.assert_allclose(res.trace_x, xq, rtol=0, atol=1e-10 * np.max(np.abs(xq)))
    assert res.n_replacements == steps // 2 == exact["replacements"]
