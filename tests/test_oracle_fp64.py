"""Pins of the FP64 oracle against mathematics, library routines and the paper (CPU only)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_1612_01395_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out[parts[0]] = parts[1:]
    return out


def cd2d_64():
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    xs = P.splitmix64_uniform(0, A.n)
    return A, xs, oracle.spmv(A, xs)


def scipy_csr(A):
    return sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))


def test_spmv_matches_dense_product():
    A = P.stencil_to_csr(P.cd3d_trig(6))
    x = P.splitmix64_uniform(3, A.n)
    np.testing.assert_allclose(oracle.spmv(A, x), A.to_dense() @ x, rtol=1e-14, atol=1e-14)


def test_dot_is_left_to_right_sum():
    a = P.splitmix64_uniform(1, 1000)
    b = P.splitmix64_uniform(2, 1000)
    acc = 0.0
    for u, v in zip(a.tolist(), b.tolist()):
        acc = acc + u * v
    assert oracle.dot(a, b) == acc


@pytest.mark.parametrize("method", ["bicgstab", "cabicgstab", "pbicgstab"])
@pytest.mark.parametrize("grid", [(4, 4), (8, 8), (4, 4, 4)])
def test_solution_matches_dense_lu(method, grid):
    """Dense LU (numpy.linalg.solve) on N <= 64 convection-diffusion systems."""
    if len(grid) == 2:
        st = P.cd2d_constant(grid[0], (10.0, 10.0))
    else:
        st = P.cd3d_trig(grid[0])
    A = P.stencil_to_csr(st)
    b = P.splitmix64_uniform(11, A.n)
    x_lu = np.linalg.solve(A.to_dense(), b)
    res = getattr(oracle, method)(A, b, rtol=1e-13, maxit=500)
    assert res.status == oracle.CONVERGED
    kappa = np.linalg.cond(A.to_dense())
    assert np.linalg.norm(res.x - x_lu) / np.linalg.norm(x_lu) <= 10 * kappa * 1e-13


def test_bicgstab_matches_scipy_iterates():
    """scipy.sparse.linalg.bicgstab implements the same Algorithm 7 (shadow = r_0,
    x0 = 0); only the dot-product summation order differs."""
    A, xs, b = cd2d_64()
    scipy_x = []
    spla.bicgstab(scipy_csr(A), b, rtol=1e-30, atol=0.0, maxiter=25, callback=lambda xk: scipy_x.append(xk.copy()))
    res = oracle.bicgstab(A, b, fixed_iters=25, trace=True)
    assert len(scipy_x) == 25
    for i in range(20):
        xi = res.trace_x[i + 1]
        assert np.linalg.norm(xi - scipy_x[i]) <= 1e-10 * np.linalg.norm(xi), i


def test_pipelined_matches_standard_early_iterations():
    """Exact arithmetic makes Algorithm 7 and Algorithm 9 identical; in FP64 the
    residual norms agree closely in early iterations and drift later (Section 3.3)."""
    A, xs, b = cd2d_64()
    r7 = oracle.bicgstab(A, b, fixed_iters=20)
    r8 = oracle.cabicgstab(A, b, fixed_iters=20)
    r9 = oracle.pbicgstab(A, b, fixed_iters=20)
    r9e = oracle.pbicgstab(A, b, fixed_iters=20, alpha_eq5=True)
    for other in (r8, r9, r9e):
        np.testing.assert_allclose(other.hist, r7.hist, rtol=1e-8)


def test_auxiliary_vectors_satisfy_their_definitions():
    """w = A r, s = A p, z = A s, t = A w, v = A z hold up to rounding (Section 3.3)."""
    A, xs, b = cd2d_64()
    res = oracle.pbicgstab(A, b, fixed_iters=6, keep_work=True)
    W = res.work
    Av = lambda u: oracle.spmv(A, u)
    norm_a = 8.0 + 2.0  # |row sums| of |A| are at most 4 + 2(1 + 10h)
    for lhs, rhs, base in [("w", "r", "r"), ("s", "p", "p"), ("z", "s", "s"), ("t", "w", "w"), ("v", "z", "z")]:
        gap = np.linalg.norm(W[lhs] - Av(W[rhs]))
        assert gap <= 1e-12 * norm_a * np.linalg.norm(W[base]) * 10, (lhs, gap)
    # q = r - alpha s and y = w - alpha z imply y = A q
    assert np.linalg.norm(W["y"] - Av(W["q"])) <= 1e-11 * norm_a * np.linalg.norm(W["q"]) * 10


def test_flop_and_vector_counts_match_table1():
    """AXPY + dot-product flops per iteration (Table 1): 20N vs 38N."""
    g = read_golden("table1_costs.txt")
    A, xs, b = cd2d_64()
    n, its = A.n, 10
    r7 = oracle.bicgstab(A, b, fixed_iters=its)
    r9 = oracle.pbicgstab(A, b, fixed_iters=its)
    assert r7.flops == int(g["bicgstab"][2]) * n * its
    assert r9.flops == int(g["pbicgstab"][2]) * n * its
    # SpMVs per iteration (Table 1, column spmv) after the initialisation
    assert r7.spmvs == 1 + int(g["bicgstab"][1]) * its
    assert r9.spmvs == 3 + int(g["pbicgstab"][1]) * its
    # vectors held: x plus the work vectors of each routine (Table 1, column memory)
    res = oracle.pbicgstab(A, b, fixed_iters=1, keep_work=True)
    assert 1 + len(res.work) == int(g["pbicgstab"][3])


def test_breakdown_permutation_matrix():
    """A = [[0,1],[1,0]], b = (1,0): (r0, A r0) = 0, so alpha's denominator vanishes."""
    A = P.dense_to_csr(np.array([[0.0, 1.0], [1.0, 0.0]]))
    b = np.array([1.0, 0.0])
    for m in ("bicgstab", "cabicgstab", "pbicgstab"):
        res = getattr(oracle, m)(A, b)
        assert res.status == oracle.BREAKDOWN, m
        assert res.iters == 0
        np.testing.assert_array_equal(res.x, [0.0, 0.0])


def test_scaled_identity_converges_in_one_half_step():
    """A = 2I: q_0 = r_0 - alpha_0 A r_0 = 0 exactly, so x = b/2 after a half step."""
    n = 17
    A = P.dense_to_csr(2.0 * np.eye(n))
    b = P.splitmix64_uniform(5, n)
    for m in ("bicgstab", "cabicgstab", "pbicgstab"):
        res = getattr(oracle, m)(A, b)
        assert res.status == oracle.CONVERGED and res.iters == 1 and res.half_step, m
        np.testing.assert_array_equal(res.x, b / 2.0)


def test_zero_rhs_returns_immediately():
    A, xs, b = cd2d_64()
    res = oracle.pbicgstab(A, np.zeros(A.n))
    assert res.status == oracle.CONVERGED and res.iters == 0
    assert np.all(res.x == 0.0)


def test_nonfinite_input_detected():
    A, xs, b = cd2d_64()
    bad = b.copy()
    bad[7] = np.nan
    res = oracle.pbicgstab(A, bad)
    assert res.status in (oracle.NONFINITE, oracle.BREAKDOWN)
    assert res.status == oracle.NONFINITE


def true_gap(A, b, res):
    """||r_i - (b - A x_i)|| / ||r_0|| at exit (recursive vs true residual)."""
    return abs(res.rel_res_true - res.rel_res_rec)


def test_residual_replacement_restores_attainable_accuracy():
    """Section 4.2: without replacement the pipelined method stagnates orders of
    magnitude above BiCGStab; with replacement it reaches BiCGStab's level."""
    A, xs, b = cd2d_64()
    plain = oracle.bicgstab(A, b, rtol=1e-14, maxit=600)
    pipe = oracle.pbicgstab(A, b, rtol=1e-14, maxit=600)
    assert plain.rel_res_true < 1e-13
    assert pipe.rel_res_true > 100 * plain.rel_res_true       # accuracy lost (Table 3)
    for k in (10, 20, 50):
        rr = oracle.pbicgstab(A, b, rtol=1e-14, maxit=600, replace_period=k)
        assert rr.status == oracle.CONVERGED, k
        assert rr.n_replacements == rr.iters // k, k
        assert rr.rel_res_true < 10 * max(plain.rel_res_true, 1e-14), k


def test_replacement_cap():
    A, xs, b = cd2d_64()
    rr = oracle.pbicgstab(A, b, rtol=1e-14, maxit=600, replace_period=10, max_replacements=3)
    assert rr.n_replacements == 3


def test_literal_replacement_placement_is_unstable():
    """Replacing r, w, s, z only after p_i, with t_i, rho_i and alpha_i left from the
    recurrences, breaks the Krylov relations; the split placement does not."""
    A, xs, b = cd2d_64()
    late = oracle.pbicgstab(A, b, rtol=1e-14, maxit=400, replace_period=20, rr_placement=1)
    split = oracle.pbicgstab(A, b, rtol=1e-14, maxit=400, replace_period=20)
    assert not (late.rel_res_true < 1e-6)
    assert split.rel_res_true < 1e-13


def test_ptp2_tolerance_matches_paper():
    """Dirichlet reading of PTP2 gives ||b|| = ||A 1|| with 1e-6 ||b|| = 3.0e-3 (Table 4)."""
    g = read_golden("ptp_reference.txt")
    A = P.stencil_to_csr(P.ptp2(1000))
    nb = np.linalg.norm(oracle.spmv(A, np.ones(A.n)))
    assert round(1e-6 * nb, 4) == float(g["ptp2_true_residual_at_1e-6"][0])


def test_ptp1_norm_of_rhs():
    A = P.stencil_to_csr(P.ptp1(1000))
    nb = np.linalg.norm(oracle.spmv(A, np.ones(A.n)))
    assert abs(nb - 63.4349) < 1e-3


@pytest.mark.slow
def test_ptp1_iteration_count_in_paper_range():
    """PTP1 to 1e-6 takes 205..282 iterations in the paper (Figure 3 caption)."""
    g = read_golden("ptp_reference.txt")
    lo, hi = int(g["ptp1_iters_min"][0]), int(g["ptp1_iters_max"][0])
    A = P.stencil_to_csr(P.ptp1(1000))
    b = oracle.spmv(A, np.ones(A.n))
    res = oracle.pbicgstab(A, b, rtol=1e-6, maxit=2000, replace_period=100)
    assert res.status == oracle.CONVERGED
    assert lo <= res.iters <= hi


@pytest.mark.slow
def test_ptp1_attainable_accuracy_matches_paper():
    """PTP1 accuracy experiment (Section 5, Figure 4): true residual norms the
    paper reports as attained within 2000 iterations -- BiCGStab 5.8e-12,
    p-BiCGStab 1.7e-9, p-BiCGStab-rr (every 100 iterations, at most 10) 2.5e-12.
    Another reduction order (the paper ran on 240 processes) changes these
    levels, so the pin is the order of magnitude (factor 10) and the ordering:
    without replacement the pipelined method stalls two to three orders above
    the other two. p-BiCGStab is sampled at its best region (the true residual
    grows again after it): fixed 500 iterations."""
    g = read_golden("ptp_reference.txt")
    A = P.stencil_to_csr(P.ptp1(1000))
    b = oracle.spmv(A, np.ones(A.n))

    def true_res(x):
        return np.linalg.norm(b - oracle.spmv(A, x))

    std = true_res(oracle.bicgstab(A, b, rtol=1e-17, maxit=2000).x)
    rr = true_res(oracle.pbicgstab(A, b, rtol=1e-17, maxit=2000, replace_period=100, max_replacements=10).x)
    pipe = true_res(oracle.pbicgstab(A, b, rtol=0.0, maxit=500, fixed_iters=500).x)
    for got, key in ((std, "ptp1_attained_bicgstab"), (rr, "ptp1_attained_pbicgstab_rr"),
                     (pipe, "ptp1_attained_pbicgstab")):
        paper = float(g[key][0])
        assert paper / 10 <= got <= paper * 10, (key, got)
    assert pipe > 100 * max(std, rr)


def test_trajectory_sensitivity_to_summation_order():
    """Two equally valid FP64 evaluations of Algorithm 9 -- dot products summed
    left to right (the oracle) or right to left -- agree closely for ~20
    iterations on the 64 x 64 system and then drift apart by orders of
    magnitude more than 1e-9, while both still converge. This is why iterate-
    by-iterate parity is asserted over the first 20 iterations only, and long
    solves are compared through their final solutions."""
    A, xs, b = cd2d_64()

    def rdot(u, v):
        return oracle.dot(u[::-1].copy(), v[::-1].copy())

    def alg9_reversed(iters):
        Av = lambda u: oracle.spmv(A, u)
        x = np.zeros(A.n)
        r = b - Av(x)
        r0 = r.copy()
        w = Av(r)
        t = Av(w)
        p = np.zeros(A.n); s = p.copy(); z = p.copy(); v = p.copy()
        rho = rdot(r0, r)
        alpha, beta, omega = rho / rdot(r0, w), 0.0, 0.0
        for _ in range(iters):
            p = r + beta * (p + (-omega) * s)
            s = w + beta * (s + (-omega) * z)
            z = t + beta * (z + (-omega) * v)
            q = r + (-alpha) * s
            y = w + (-alpha) * z
            qy, yy = rdot(q, y), rdot(y, y)
            v = Av(z)
            omega = qy / yy
            x = (x + alpha * p) + omega * q
            r = q + (-omega) * y
            w = y + (-omega) * (t + (-alpha) * v)
            rn, r0w, r0s, r0z = rdot(r0, r), rdot(r0, w), rdot(r0, s), rdot(r0, z)
            t = Av(w)
            beta = (alpha / omega) * (rn / rho)
            alpha = rn / (r0w + beta * r0s - beta * omega * r0z)
            rho = rn
        return x

    def gap(iters):
        ref = oracle.pbicgstab(A, b, rtol=0.0, maxit=iters, fixed_iters=iters).x
        return np.linalg.norm(alg9_reversed(iters) - ref) / np.linalg.norm(ref)

    assert gap(20) < 1e-10
    assert gap(40) > 1e-7
