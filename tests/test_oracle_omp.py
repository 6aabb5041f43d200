"""The OpenMP build of the oracle (used only to time the oracle on all host
cores) computes the same algorithm: only its dot products are summed in
another order, so its residual histories agree with the single-threaded
parity build to rounding over the first iterations and its solves converge
alike (CPU only)."""
import numpy as np

import oracle
from paper_1612_01395_gb300 import problems as P


def test_openmp_build_agrees_with_parity_build():
    A = P.stencil_to_csr(P.cd3d_trig(24))
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    assert oracle.num_threads(omp=False) == 1
    assert oracle.num_threads(omp=True) >= 1
    for fn, kw in ((oracle.pbicgstab, {"replace_period": 5}), (oracle.bicgstab, {})):
        ref = fn(A, b, rtol=0.0, maxit=12, fixed_iters=12, **kw)
        got = fn(A, b, rtol=0.0, maxit=12, fixed_iters=12, omp=True, **kw)
        np.testing.assert_allclose(got.hist, ref.hist, rtol=1e-10)
        assert np.linalg.norm(got.x - ref.x) / np.linalg.norm(ref.x) <= 1e-10
        full = fn(A, b, rtol=1e-8, maxit=2000, omp=True, **kw)
        assert full.status == oracle.CONVERGED and full.rel_res_true <= 1e-8
