"""The bounds-checked build (-DPBCG_CHECK) on the GPU (needs a GB300).

Every solver path runs under the checked library: stencil and CSR forms (both
CSR operator forms), both methods, the Jacobi-preconditioned methods
(Algorithms 10 and 11), the mixed-precision solve (stencil with even and odd
nx, CSR with FP32 and BF16 values), the SpMV entry point, the
allocation-free entry point, the adjoint transpose and value gradient, and a
small batch. No index may be reported out of range, and
the results must equal the default build's bit for bit: the checks only guard
indices, they change no arithmetic.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    default = native.build()
    checked = native.build(check=True)
    yield default, checked
    native.LIB_PATH, native._lib = default, None


def use(path):
    native.LIB_PATH, native._lib = path, None


def run_all():
    import torch
    out = {}
    for name, st in (("cd3d_20", P.cd3d_trig(20)), ("cd2d_37", P.cd2d_constant(37, (10.0, 4.0)))):
        A = P.stencil_to_csr(st)
        b = torch.from_numpy(oracle.spmv(A, P.splitmix64_uniform(0, A.n))).cuda()
        for form in ("stencil", "csr"):
            s = native.Solver.from_stencil(st) if form == "stencil" else native.Solver.from_csr(A)
            for method in ("pipelined", "standard"):
                x, _ = s.solve(b, rtol=1e-10, maxit=2000, replace_period=20, method=method)
                out[(name, form, method)] = x.cpu().numpy()
            v32 = None if form == "stencil" else torch.from_numpy(A.val).cuda().to(torch.float32)
            x, _ = s.solve_mixed(b, v32, native.PBCG_VALUES_F32, rtol=1e-10, max_outer=30, inner_rtol=1e-3,
                                 inner_maxit=500)
            out[(name, form, "mixed")] = x.cpu().numpy()
            if form == "csr":
                v16 = torch.from_numpy(A.val).cuda().to(torch.bfloat16)
                x, _ = s.solve_mixed(b, v16, native.PBCG_VALUES_BF16, rtol=1e-10, max_outer=30, inner_rtol=1e-2,
                                     inner_maxit=150)
                out[(name, form, "mixed_bf16")] = x.cpu().numpy()
            out[(name, form, "spmv")] = s.spmv(b).cpu().numpy()
            s.close()
            s = native.Solver.from_stencil(st, prec=native.PBCG_PREC_JACOBI) if form == "stencil" else \
                native.Solver.from_csr(A, prec=native.PBCG_PREC_JACOBI)
            for method in ("pipelined", "standard"):
                x, _ = s.solve(b, rtol=1e-10, maxit=2000, replace_period=20, method=method)
                out[(name, form, method + "_jacobi")] = x.cpu().numpy()
            s.close()
        # the allocation-free entry point
        rowptr, col, val = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val))
        x = torch.zeros_like(b)
        st_, _ = native.pbicgstab_solve_csr_noalloc(A.n, A.nnz, rowptr.data_ptr(), col.data_ptr(), val.data_ptr(),
                                                    b.data_ptr(), x.data_ptr(), 1e-10, 2000, 20,
                                                    torch.cuda.current_stream().cuda_stream)
        assert st_ == native.PBCG_OK
        out[(name, "csr", "noalloc")] = x.cpu().numpy()
        # the adjoint building blocks: A^T and the value gradient
        from paper_1612_01395_gb300.adjoint import CSRStructure
        cs = CSRStructure(A.rowptr, A.col)
        stream = torch.cuda.current_stream().cuda_stream
        assert native.pbicgstab_csr_transpose(cs.n, cs.nnz, cs.rowptr.data_ptr(), cs.col.data_ptr(), val.data_ptr(),
                                              cs.trowptr.data_ptr(), cs.tcol.data_ptr(), cs.tval.data_ptr(),
                                              cs.work.data_ptr(), cs.work_bytes, stream) == native.PBCG_OK
        out[(name, "csr", "transpose")] = cs.tval.cpu().numpy()
        g = torch.empty_like(val)
        assert native.pbicgstab_csr_value_grad(cs.n, cs.rowptr.data_ptr(), cs.col.data_ptr(), b.data_ptr(),
                                               x.data_ptr(), g.data_ptr(), stream) == native.PBCG_OK
        out[(name, "csr", "value_grad")] = g.cpu().numpy()
    R = P.random_sparse(3001, seed=5)
    s = native.Solver.from_csr(R)
    b = torch.from_numpy(oracle.spmv(R, P.splitmix64_uniform(1, R.n))).cuda()
    out[("rand_3001", "csr", "pipelined")] = s.solve(b, rtol=1e-10, maxit=2000)[0].cpu().numpy()
    s.close()
    B = P.random_batch(nsys=6, seed=2, nmin=500, nmax=3000)
    bs = native.BatchSolver(B)
    bd = torch.from_numpy(B.b).cuda()
    x = torch.zeros_like(bd)
    bs.launch(bd, x, rtol=1e-10, maxit=500)
    torch.cuda.synchronize()
    out[("batch", "csr", "pipelined")] = x.cpu().numpy()
    del bs
    return out


def test_checked_build_reports_no_fault_and_matches_default(libs):
    default, checked = libs
    use(default)
    assert native.pbicgstab_check_faults() == -1
    ref = run_all()
    use(checked)
    assert native.pbicgstab_check_faults() == 0
    got = run_all()
    assert native.pbicgstab_check_faults() == 0
    use(default)
    for key, x in ref.items():
        assert np.all(np.isfinite(x)), key
        np.testing.assert_array_equal(got[key], x, err_msg=str(key))
