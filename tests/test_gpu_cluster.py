"""Single small systems on one thread-block cluster (needs a GB300).

Systems of up to 24576 stored entries (stencil: points x unknowns) are solved
by default by the CTAs of one thread-block cluster, whose reductions go through distributed shared memory
and the hardware cluster barrier instead of a cooperative grid's exchanges
through L2. The solver loops are the same code; only the reduction tree (and
so the rounding of the dot products) differs. It is held against the oracle
as the grid is: residual norms within 1e-8 and x within 1e-9 over the first
20 iterations, for every cluster size and both methods, and final solutions
of tight solves within 1e-9.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu

X_TOL = 1e-9
HIST_TOL = 1e-8
HIST_FLOOR = 1e-13
K = 20


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def problems():
    return {"cd2d_64": P.cd2d_constant(64, (10.0, 10.0)), "cd3d_20": P.cd3d_trig(20), "cd2d_37": P.cd2d_constant(37, (10.0, 4.0))}


@pytest.mark.parametrize("name", ["cd2d_64", "cd3d_20", "cd2d_37"])
@pytest.mark.parametrize("form", ["csr", "stencil"])
@pytest.mark.parametrize("method", ["pipelined", "standard"])
@pytest.mark.parametrize("cluster", [0, 2, 4, 8, 16])
def test_cluster_first_iterations_match_oracle(name, form, method, cluster):
    st = problems()[name]
    A = P.stencil_to_csr(st)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    s = native.Solver.from_stencil(st) if form == "stencil" else native.Solver.from_csr(A)
    ref = (oracle.pbicgstab if method == "pipelined" else oracle.bicgstab)(A, b, rtol=0.0, maxit=K, fixed_iters=K)
    try:
        x, info, hist = s.solve(dev(b), rtol=0.0, maxit=K, fixed_iters=K, method=method, cluster=cluster,
                                history=True)
    except native.PbcgError as e:   # a cluster size this device cannot make resident
        assert cluster == 16 and e.status == native.PBCG_ERR_ARG
        pytest.skip(str(e))
    assert info["status"] == native.PBCG_OK
    if cluster:
        assert info["cluster"] == cluster and info["grid"] == cluster
    else:   # automatic: the cluster for the 2-D systems (<= 24576 entries), the grid for 20^3 (56k)
        assert (info["cluster"] > 0) == (name != "cd3d_20")
    h = hist.cpu().numpy()
    assert np.all(np.abs(h - ref.hist) <= HIST_TOL * ref.hist + HIST_FLOOR * ref.nr0), np.abs(h - ref.hist) / ref.hist
    assert rel(x.cpu().numpy(), ref.x) <= X_TOL
    # deterministic: the same launch gives the same bits
    x2, _ = s.solve(dev(b), rtol=0.0, maxit=K, fixed_iters=K, method=method, cluster=cluster)
    np.testing.assert_array_equal(x.cpu().numpy(), x2.cpu().numpy())
    s.close()


@pytest.mark.parametrize("method,rr", [("pipelined", 20), ("standard", 0)])
def test_cluster_final_solution_matches_oracle(method, rr):
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    b = oracle.spmv(A, P.splitmix64_uniform(2, A.n))
    fn = oracle.pbicgstab if method == "pipelined" else oracle.bicgstab
    kw = {"replace_period": rr} if method == "pipelined" else {}
    ref = fn(A, b, rtol=1e-12, maxit=2000, **kw)
    s = native.Solver.from_csr(A)
    x, info = s.solve(dev(b), rtol=1e-12, maxit=2000, replace_period=rr, method=method)
    assert info["cluster"] > 0 and info["status"] == native.PBCG_OK
    assert rel(x.cpu().numpy(), ref.x) <= X_TOL
    true_rel = np.linalg.norm(b - oracle.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert abs(true_rel - info["rel_res_true"]) <= 1e-3 * true_rel + 1e-15
    assert abs(info["iters"] - ref.iters) <= max(3, ref.iters // 10)
    s.close()


def replaced_history_close(A, h, ref, xg):
    """Residual norms of a window whose last iterate was replaced (r_K := b - A x_K).
    Recursive residuals are compared at the usual bar; the replaced one is the
    true residual of x_K, and two x_K that differ by dx have true residuals
    that differ by up to ||A dx|| (triangle inequality), so that term --
    computed with the oracle's SpMV -- is added to its bar."""
    tol = HIST_TOL * ref.hist + HIST_FLOOR * ref.nr0
    tol[-1] += np.linalg.norm(oracle.spmv(A, xg - ref.x))
    return np.all(np.abs(h - ref.hist) <= tol)


def test_cluster_replacement_window_matches_oracle():
    """Residual replacement every 5 iterations inside the 20-iteration window."""
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    ref = oracle.pbicgstab(A, b, rtol=0.0, maxit=K, fixed_iters=K, replace_period=5)
    s = native.Solver.from_csr(A)
    x, info, hist = s.solve(dev(b), rtol=0.0, maxit=K, fixed_iters=K, replace_period=5, history=True)
    assert info["cluster"] > 0 and info["n_replacements"] == ref.n_replacements == 4
    xg = x.cpu().numpy()
    assert replaced_history_close(A, hist.cpu().numpy(), ref, xg)
    assert rel(xg, ref.x) <= X_TOL
    s.close()


def test_path_selection():
    """Automatic: a cluster up to 24576 stored entries, the cooperative grid above;
    cluster=-1 or a forced grid always take the grid; Jacobi handles always
    take the grid."""
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    b = dev(oracle.spmv(A, P.splitmix64_uniform(0, A.n)))
    s = native.Solver.from_csr(A)
    assert s.solve(b, rtol=1e-8, maxit=500)[1]["cluster"] > 0
    assert s.solve(b, rtol=1e-8, maxit=500, cluster=-1)[1]["cluster"] == 0
    assert s.solve(b, rtol=1e-8, maxit=500, grid=32)[1]["cluster"] == 0
    with pytest.raises(native.PbcgError):
        s.solve(b, rtol=1e-8, maxit=500, cluster=3)
    s.close()
    big = P.cd3d_trig(16)   # 4096 unknowns, 7 points: 28672 entries
    sb = native.Solver.from_stencil(big)
    bb = sb.spmv(dev(P.splitmix64_uniform(0, big.n)))
    assert sb.solve(bb, rtol=1e-8, maxit=500)[1]["cluster"] == 0
    sb.close()
    sj = native.Solver.from_csr(A, prec=native.PBCG_PREC_JACOBI)
    assert sj.solve(b, rtol=1e-8, maxit=500)[1]["cluster"] == 0
    sj.close()


def test_cluster_degenerate_systems():
    """Fewer rows than CTAs (empty row ranges), A = 2I, a zero right-hand side."""
    for n in (1, 2, 5, 300):
        s = native.Solver.from_csr(P.dense_to_csr(2.0 * np.eye(n)))
        b = P.splitmix64_uniform(5, n)
        x, info = s.solve(dev(b), rtol=1e-10, maxit=10, cluster=2)
        assert info["cluster"] == 2 and info["half_step"] == 1 and info["iters"] == 1
        np.testing.assert_array_equal(x.cpu().numpy(), b / 2.0)
        x, info = s.solve(dev(np.zeros(n)), rtol=1e-10, maxit=10)
        assert info["status"] == native.PBCG_OK and info["iters"] == 0
        s.close()


def test_cluster_breakdown_is_reported():
    """The 2x2 permutation with b = e1 breaks down at (r0, s_0) = 0 on both paths."""
    A = P.dense_to_csr(np.array([[0.0, 1.0], [1.0, 0.0]]))
    s = native.Solver.from_csr(A)
    for method in ("pipelined", "standard"):
        _, info = s.solve(dev(np.array([1.0, 0.0])), rtol=1e-10, maxit=10, method=method)
        assert info["cluster"] > 0 and info["status"] == native.PBCG_BREAKDOWN
    s.close()
