"""Adjoint (reverse-mode) solves on the GPU, checked against the oracle's adjoint
and central finite differences (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P
from test_oracle_adjoint import oracle_gradients, transpose

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def test_transpose_matches_scipy_bitwise():
    import torch
    from paper_1612_01395_gb300.adjoint import CSRStructure
    A = P.random_sparse(2000, seed=4)
    st = CSRStructure(A.rowptr, A.col)
    val = torch.from_numpy(A.val).cuda()
    rc = native.pbicgstab_csr_transpose(st.n, st.nnz, st.rowptr.data_ptr(), st.col.data_ptr(), val.data_ptr(),
                                        st.trowptr.data_ptr(), st.tcol.data_ptr(), st.tval.data_ptr(),
                                        st.work.data_ptr(), st.work_bytes, torch.cuda.current_stream().cuda_stream)
    assert rc == native.PBCG_OK
    T = transpose(A)
    np.testing.assert_array_equal(st.trowptr.cpu().numpy(), T.rowptr)
    np.testing.assert_array_equal(st.tcol.cpu().numpy(), T.col)
    np.testing.assert_array_equal(st.tval.cpu().numpy(), T.val)


def setup(n=48, seed=1):
    import torch
    from paper_1612_01395_gb300.adjoint import CSRStructure
    A = P.stencil_to_csr(P.cd2d_field(n, seed=seed))
    b = P.splitmix64_uniform(2, A.n)
    xt = P.splitmix64_uniform(3, A.n)
    return A, b, xt, CSRStructure(A.rowptr, A.col)


def gpu_loss_and_grads(A, b, xt, st):
    import torch
    from paper_1612_01395_gb300.adjoint import sparse_solve
    vals = torch.from_numpy(A.val).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = sparse_solve(vals, bt, st, rtol=1e-13)
    L = 0.5 * ((x - torch.from_numpy(xt).cuda()) ** 2).sum()
    L.backward()
    return float(L), x.detach().cpu().numpy(), bt.grad.cpu().numpy(), vals.grad.cpu().numpy()


def test_adjoint_gradients_match_oracle_adjoint():
    A, b, xt, st = setup()
    L, x, gb, gv = gpu_loss_and_grads(A, b, xt, st)
    xo, gbo, gvo = oracle_gradients(A, b, xt)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-9
    assert np.linalg.norm(gb - gbo) / np.linalg.norm(gbo) <= 1e-8
    assert np.linalg.norm(gv - gvo) / np.linalg.norm(gvo) <= 1e-8


def test_adjoint_gradients_match_central_differences():
    """32 random coordinates of dL/db and dL/dvalues by central differences.

    A difference quotient carries the solves' noise divided by 2h (about
    L * 1e-13 / h here), so the steps are as large as truncation allows. L is a
    quadratic function of b, so the central difference in b has no truncation
    error at any step: h = 1e-2. In a stored value, x is a rational function
    (Sherman-Morrison) and the central difference errs by O(h^2); one
    Richardson step over h and 2h (h = 5e-3) removes that term. Errors are
    measured against |g| + 1e-3 max|g|."""
    import torch
    from paper_1612_01395_gb300.adjoint import sparse_solve
    A, b, xt, st = setup()
    L, x, gb, gv = gpu_loss_and_grads(A, b, xt, st)
    xt_d = torch.from_numpy(xt).cuda()
    vals0 = torch.from_numpy(A.val).cuda()
    b0 = torch.from_numpy(b).cuda()

    def f(vals, bb):
        xx = sparse_solve(vals, bb, st, rtol=1e-13)
        return float(0.5 * ((xx - xt_d) ** 2).sum())

    def central_b(i, h):
        e = torch.zeros_like(b0)
        e[i] = h
        return (f(vals0, b0 + e) - f(vals0, b0 - e)) / (2 * h)

    def central_v(k, h):
        e = torch.zeros_like(vals0)
        e[k] = h
        return (f(vals0 + e, b0) - f(vals0 - e, b0)) / (2 * h)

    sb = 1e-3 * np.abs(gb).max()
    for i in (P.splitmix64(11, 16) % np.uint64(A.n)).astype(int):
        fd = central_b(i, 1e-2)
        assert abs(fd - gb[i]) <= 1e-6 * (abs(gb[i]) + sb), i
    sv = 1e-3 * np.abs(gv).max()
    for k in (P.splitmix64(12, 16) % np.uint64(A.nnz)).astype(int):
        fd = (4 * central_v(k, 5e-3) - central_v(k, 1e-2)) / 3
        assert abs(fd - gv[k]) <= 1e-6 * (abs(gv[k]) + sv), k


def test_adjoint_gradients_match_oracle_adjoint_at_256():
    """The GPU adjoint against the oracle's adjoint on the largest grid the
    oracle solves in test time (256^2 = 65536 unknowns, both solves to 1e-13)."""
    A, b, xt, st = setup(n=256, seed=3)
    L, x, gb, gv = gpu_loss_and_grads(A, b, xt, st)
    xo, gbo, gvo = oracle_gradients(A, b, xt)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-9
    assert np.linalg.norm(gb - gbo) / np.linalg.norm(gbo) <= 1e-8
    assert np.linalg.norm(gv - gvo) / np.linalg.norm(gvo) <= 1e-8


def test_adjoint_central_differences_with_step_1e6():
    """The configured check: central differences with h = 1e-6 on 32 random
    coordinates (16 of b, 16 of the values), per-coordinate relative error, no
    floor. A perturbed solution is x* + d with A' d = b' - A' x* solved to rtol
    1e-10 of its own right-hand side (so d's error scales with h), and
    L(+) - L(-) is evaluated as (x* - x_t).(d+ - d-) + (|d+|^2 - |d-|^2)/2,
    which is exact algebra for this quadratic loss and avoids cancelling two
    nearly equal losses. Truncation is O(h^2) ~ 1e-12 relative and the
    corrections carry ~1e-10 relative error, so 1e-6 per coordinate leaves
    room only for coordinates whose gradient is far below the terms of the
    dot product."""
    import torch
    from paper_1612_01395_gb300.adjoint import sparse_solve
    A, b, xt, st = setup()
    L, x, gb, gv = gpu_loss_and_grads(A, b, xt, st)
    vals0 = torch.from_numpy(A.val).cuda()
    b0 = torch.from_numpy(b).cuda()
    xt_d = torch.from_numpy(xt).cuda()
    xstar = sparse_solve(vals0, b0, st, rtol=1e-13).detach()

    def correction(v, bvec):
        s = native.Solver()
        ws, nb = s._workspace(A.n, None)
        s.h = native.pbicgstab_create_csr(A.n, A.nnz, st.rowptr.data_ptr(), st.col.data_ptr(), v.data_ptr(),
                                          native.PBCG_PREC_NONE, ws, nb, torch.cuda.current_stream().cuda_stream)
        d, info = s.solve(bvec - s.spmv(xstar), rtol=1e-10, maxit=20000, replace_period=50)
        s.close()
        assert info["status"] == native.PBCG_OK
        return d

    def numerator(vp, bp, vm, bm):
        dp, dm = correction(vp, bp), correction(vm, bm)
        return float(torch.dot(xstar - xt_d, dp - dm) + 0.5 * (torch.dot(dp, dp) - torch.dot(dm, dm)))

    h = 1e-6
    errs = []
    for i in (P.splitmix64(21, 16) % np.uint64(A.n)).astype(int):
        e = torch.zeros_like(b0)
        e[i] = h
        fd = numerator(vals0, b0 + e, vals0, b0 - e) / (2 * h)
        errs.append(abs(fd - gb[i]) / abs(gb[i]))
    for k in (P.splitmix64(22, 16) % np.uint64(A.nnz)).astype(int):
        e = torch.zeros_like(vals0)
        e[k] = h
        fd = numerator(vals0 + e, b0, vals0 - e, b0) / (2 * h)
        errs.append(abs(fd - gv[k]) / abs(gv[k]))
    assert max(errs) <= 1e-6, errs
