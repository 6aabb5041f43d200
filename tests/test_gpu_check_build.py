"""The bounds-checked build (-DPBCG_CHECK) on the GPU (needs a GB300).

Every solver path runs under the checked library: stencil and CSR forms (both
CSR operator forms), both methods, the mixed-precision solve (stencil with even
and odd nx, CSR) and a small batch. No index may be reported out of range, and
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
            s.close()
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
