"""The allocation-free entry point pbicgstab_solve_csr_noalloc (needs a GB300).

Some callers cannot allocate device memory or pass a workspace (an application
that owns all device memory and forbids allocation after start-up, a real-time
loop, a plug-in that only receives input and output pointers). This entry
point serves them from a fixed array inside the library. The test calls it
twice in a row through the C ABI, with different right-hand sides so the
second call starts from the first call's leftovers, and checks each result
against the handle-based pbicgstab_solve within the parity tolerance. Around
the second call, with the device idle on both sides, the device's free memory
must not change: the call allocates nothing.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu

X_TOL = 1e-9


def test_noalloc_solve_matches_handle_solve_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()
    A = P.stencil_to_csr(P.cd2d_constant(64, (10.0, 10.0)))
    rowptr = torch.as_tensor(A.rowptr).cuda()
    col = torch.as_tensor(A.col).cuda()
    val = torch.as_tensor(A.val).cuda()
    ref = native.Solver.from_csr(A)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (0, 1):
        b = ref.spmv(torch.from_numpy(P.splitmix64_uniform(seed, A.n)).cuda())
        x_ref, info_ref = ref.solve(b, rtol=1e-10, maxit=1000, replace_period=20)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st, info = native.pbicgstab_solve_csr_noalloc(A.n, A.nnz, rowptr.data_ptr(), col.data_ptr(),
                                                      val.data_ptr(), b.data_ptr(), x.data_ptr(), 1e-10, 1000,
                                                      20, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert st == native.PBCG_OK, native.pbicgstab_last_error()
        if seed == 1:   # the first call may load the module; the second must leave free memory unchanged
            assert free_after == free_before, (free_before, free_after)
        assert info.iters == info_ref["iters"]
        xr = x_ref.cpu().numpy()
        assert np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr) <= X_TOL
    ref.close()


def test_noalloc_rejects_oversized_systems():
    n = native.PBCG_NOALLOC_MAX_N + 1
    st, info = native.pbicgstab_solve_csr_noalloc(n, 0, 1, None, None, 1, 1, 1e-8, 10, 0, None)
    assert st == native.PBCG_ERR_ARG
    assert "no-allocation limit" in native.pbicgstab_last_error()
