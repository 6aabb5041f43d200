"""Batched solves on the GPU: many independent systems in one launch (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def small_batch():
    return P.random_batch(nsys=24, seed=3, nmin=50, nmax=4000)


# (cluster_size, cluster_min_rows): every system on one CTA; every system on a
# whole cluster of 8 or 16 CTAs (min rows 1); large systems on clusters of 4,
# small ones alone; the library defaults.
SHAPES = [(1, 0), (8, 1), (16, 1), (4, 1000), (0, 0)]
SHAPE_IDS = ["alone", "cluster8", "cluster16", "mixed4", "default"]


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_batched_final_solutions_match_oracle(shape):
    """Each system solved to rtol 1e-12 (replacement every 20) matches the oracle's
    solution of that system to 1e-9, and iteration counts agree within 10 %,
    whether a system is solved by one CTA or by a cluster."""
    import torch
    B = small_batch()
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    bs.launch(b, x, rtol=1e-12, maxit=3000, replace_period=20, cluster_size=shape[0], cluster_min_rows=shape[1])
    res = bs.fetch_results()
    xg = x.cpu().numpy()
    for s in range(B.nsys):
        A = B.system(s)
        r0, r1 = B.row_offset[s], B.row_offset[s + 1]
        ref = oracle.pbicgstab(A, B.b[r0:r1], rtol=1e-12, maxit=3000, replace_period=20)
        assert res["status"][s] == native.PBCG_OK, s
        assert abs(res["iters"][s] - ref.iters) <= max(3, 0.1 * ref.iters), s
        xs = xg[r0:r1]
        assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-9, s
        true_rel = np.linalg.norm(B.b[r0:r1] - oracle.spmv(A, xs)) / ref.nr0
        assert abs(true_rel - res["rel_res_true"][s]) <= 1e-3 * true_rel + 1e-15


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_batched_iteration_count_matches_oracle(shape):
    """A batch of one system takes the oracle's number of iterations (within 2)."""
    import torch
    B = P.random_batch(nsys=1, seed=9, nmin=3000, nmax=3000)
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    bs.launch(b, x, rtol=1e-8, maxit=1000, cluster_size=shape[0], cluster_min_rows=shape[1])
    res = bs.fetch_results()
    ref = oracle.pbicgstab(B.system(0), B.b, rtol=1e-8, maxit=1000)
    assert res["status"][0] == native.PBCG_OK
    assert abs(res["iters"][0] - ref.iters) <= 2


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_invalid_system_is_isolated(shape):
    import torch
    B = small_batch()
    col = B.col.copy()
    e0 = int(B.rowptr[B.row_offset[5]])
    col[e0] = int(B.sizes[5]) + 7          # out of range for system 5
    B.col = col
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    bs.launch(b, x, rtol=1e-8, maxit=1000, cluster_size=shape[0], cluster_min_rows=shape[1])
    res = bs.fetch_results()
    assert res["status"][5] == native.PBCG_ERR_ARG
    others = np.delete(res["status"], 5)
    assert np.all(others == native.PBCG_OK)


@pytest.mark.parametrize("shape", [(1, 0), (8, 1000)], ids=["alone", "mixed8"])
def test_batched_launch_replays_in_a_cuda_graph(shape):
    """A captured launch replays to the bits of a direct launch (the result of a
    system does not depend on which CTA or cluster took it)."""
    import torch
    B = small_batch()
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    kw = dict(rtol=1e-8, maxit=1000, cluster_size=shape[0], cluster_min_rows=shape[1])
    bs.launch(b, x, **kw)
    torch.cuda.synchronize()
    direct = x.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x.zero_()
    with torch.cuda.graph(g, stream=s):
        x.zero_()
        bs.launch(b, x, stream=s, **kw)
    x.fill_(123.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, direct)
    assert np.all(bs.fetch_results()["status"] == native.PBCG_OK)


def test_unsupported_cluster_size_is_rejected():
    import torch
    B = small_batch()
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(native.PbcgError):
        bs.launch(b, x, cluster_size=3)


def test_autotuner_picks_a_launchable_shape_and_leaves_its_solution():
    """The library autotuner times the candidate shapes; on return x holds the
    solve of the chosen shape, bitwise equal to a direct launch with it."""
    import torch
    B = small_batch()
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    cs, cm, ms = bs.autotune(b, x, rtol=1e-8, maxit=1000)
    assert cs in (1, 2, 4, 8, 16) and cm > 0 and ms > 0
    assert np.all(bs.fetch_results()["status"] == native.PBCG_OK)
    tuned = x.clone()
    x.zero_()
    bs.launch(b, x, rtol=1e-8, maxit=1000, cluster_size=cs, cluster_min_rows=cm)
    torch.cuda.synchronize()
    assert torch.equal(x, tuned)


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_degenerate_systems_in_a_batch(shape):
    """An empty system, a 1x1 system and a 2x2 system among ordinary ones:
    the empty one converges in 0 iterations, the others to the exact solution."""
    import torch
    base = P.random_batch(nsys=3, seed=5, nmin=200, nmax=900)
    # systems: [base0, empty, 1x1 (a = 4), 2x2 diagonally dominant, base1, base2]
    sys_csr = [base.system(0), None, P.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0])),
               P.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
                     np.array([3.0, 1.0, -1.0, 2.0])), base.system(1), base.system(2)]
    sizes, rowptr, col, val, bs_ = [], [0], [], [], []
    for k, A in enumerate(sys_csr):
        if A is None:
            sizes.append(0)
            continue
        sizes.append(A.n)
        off = rowptr[-1]
        rowptr.extend((A.rowptr[1:].astype(np.int64) + off).tolist())
        col.extend(A.col.tolist())
        val.extend(A.val.tolist())
        bs_.append(P.splitmix64_uniform(40 + k, A.n))
    sizes = np.array(sizes, dtype=np.int64)
    B = P.Batch(sizes=sizes, row_offset=np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64),
                rowptr=np.array(rowptr, dtype=np.int32), col=np.array(col, dtype=np.int32),
                val=np.array(val, dtype=np.float64), b=np.concatenate(bs_))
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    bs.launch(b, x, rtol=1e-12, maxit=500, replace_period=20, cluster_size=shape[0], cluster_min_rows=shape[1])
    res = bs.fetch_results()
    assert np.all(res["status"] == native.PBCG_OK), res
    assert res["iters"][1] == 0
    xg = x.cpu().numpy()
    for k, A in enumerate(sys_csr):
        if A is None:
            continue
        r0, r1 = int(B.row_offset[k]), int(B.row_offset[k + 1])
        exact = np.linalg.solve(A.to_dense(), B.b[r0:r1])
        assert np.linalg.norm(xg[r0:r1] - exact) <= 1e-9 * np.linalg.norm(exact), k


@pytest.mark.parametrize("shape", [(1, 0), (8, 1), (4, 1000)], ids=["alone", "cluster8", "mixed4"])
def test_batched_first_iterations_match_oracle(shape):
    """Every system of a batch, step by step against the oracle's Algorithm 9
    on that system: residual norms within 1e-8 and x within 1e-9, whether the
    system is solved by one CTA or by a cluster, without replacement (12
    iterations) and with replacement every 5 (10 iterations, so the window
    ends on a replaced entry, whose bar adds ||A (x_gpu - x_oracle)||: the
    true residuals of two x that differ by dx differ by up to that).

    The horizon is the one these systems allow any correct FP64
    implementation: they converge by about 8 orders in 20 iterations, and two
    correct summation orders (the C oracle's Algorithms 7 and 9, and a numpy
    Algorithm 9) differ in ||r_i|| by 1e-9 at iteration 12, 2e-8 at 14 and
    1e-5 at 19 on them."""
    import torch
    B = P.random_batch(nsys=10, seed=4, nmin=300, nmax=3000)
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    for rr, K in ((0, 12), (5, 10)):
        x = torch.zeros_like(b)
        hist = torch.full((B.nsys, K + 1), float("nan"), dtype=torch.float64, device="cuda")
        bs.launch(b, x, rtol=0.0, maxit=K, replace_period=rr, cluster_size=shape[0], cluster_min_rows=shape[1],
                  fixed_iters=K, history=hist)
        res = bs.fetch_results()
        xg, hg = x.cpu().numpy(), hist.cpu().numpy()
        for s in range(B.nsys):
            A = B.system(s)
            r0, r1 = B.row_offset[s], B.row_offset[s + 1]
            ref = oracle.pbicgstab(A, B.b[r0:r1], rtol=0.0, maxit=K, fixed_iters=K, replace_period=rr)
            assert res["status"][s] == native.PBCG_OK and res["iters"][s] == K, (s, res[s])
            assert res["n_replacements"][s] == ref.n_replacements
            xs = xg[r0:r1]
            tol = 1e-8 * ref.hist + 1e-13 * ref.nr0
            if rr:
                tol[-1] += np.linalg.norm(oracle.spmv(A, xs - ref.x))
            assert np.all(np.abs(hg[s] - ref.hist) <= tol), (s, np.abs(hg[s] - ref.hist) / ref.hist)
            assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-9, s


def test_batched_history_arguments_are_checked():
    import torch
    B = P.random_batch(nsys=2, seed=4, nmin=300, nmax=400)
    bs = native.BatchSolver(B)
    b = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(b)
    short = torch.zeros((B.nsys, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(native.PbcgError):
        bs.launch(b, x, rtol=0.0, maxit=20, fixed_iters=20, history=short)
    with pytest.raises(native.PbcgError):
        bs.launch(b, x, rtol=1e-8, maxit=100, fixed_iters=-1)
