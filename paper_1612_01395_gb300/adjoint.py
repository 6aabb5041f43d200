"""Differentiable sparse solve: x = A(values)^{-1} b with gradients by an
adjoint pipelined BiCGStab solve with A^T (an extension of the method).

Forward: Algorithm 9 on the CUDA library with A's CSR values. Backward: for an
incoming gradient g = dL/dx, solve A^T lambda = g with the same solver on the
transpose built by the library (deterministic CSR transpose), then
dL/db = lambda and dL/dvalues[k] = -lambda_i x_j for stored entry k = (i, j)
(library kernel). This module only marshals arguments between torch and the
C ABI; every step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import native


class CSRStructure:
    """Row pointers and column indices of A on the device (int32), plus the
    buffers for A^T."""

    def __init__(self, rowptr, col):
        self.rowptr = torch.as_tensor(rowptr, dtype=torch.int32).cuda()
        self.col = torch.as_tensor(col, dtype=torch.int32).cuda()
        self.n = self.rowptr.numel() - 1
        self.nnz = self.col.numel()
        self.trowptr = torch.empty_like(self.rowptr)
        self.tcol = torch.empty_like(self.col)
        self.tval = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        wb = native.pbicgstab_transpose_work_bytes(self.n)
        self.work = torch.empty(wb // 4 + 64, dtype=torch.int32, device="cuda")
        self.work_bytes = wb


def _solve(structure, rowptr, col, values, rhs, rtol, maxit, replace_period):
    from .problems import CSR
    solver = native.Solver()
    torch_ = torch
    # a handle on the caller's device arrays (no copies of the matrix)
    ws, nb = solver._workspace(structure.n, None)
    solver.h = native.pbicgstab_create_csr(structure.n, structure.nnz, rowptr.data_ptr(), col.data_ptr(),
                                           values.data_ptr(), native.PBCG_PREC_NONE, ws, nb,
                                           torch_.cuda.current_stream().cuda_stream)
    x, info = solver.solve(rhs, rtol=rtol, maxit=maxit, replace_period=replace_period)
    solver.close()
    if info["status"] != native.PBCG_OK:
        raise native.PbcgError(info["status"], "solve did not converge")
    return x, info


class SparseSolve(torch.autograd.Function):
    """x = SparseSolve.apply(values, b, structure, rtol, maxit, replace_period)."""

    @staticmethod
    def forward(ctx, values, b, structure, rtol=1e-12, maxit=20000, replace_period=50):
        values = values.detach().contiguous()
        b = b.detach().contiguous()
        x, info = _solve(structure, structure.rowptr, structure.col, values, b, rtol, maxit, replace_period)
        ctx.structure = structure
        ctx.params = (rtol, maxit, replace_period)
        ctx.info = info
        ctx.save_for_backward(values, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        values, x = ctx.saved_tensors
        st = ctx.structure
        rtol, maxit, rp = ctx.params
        stream = torch.cuda.current_stream().cuda_stream
        rc = native.pbicgstab_csr_transpose(st.n, st.nnz, st.rowptr.data_ptr(), st.col.data_ptr(),
                                            values.data_ptr(), st.trowptr.data_ptr(), st.tcol.data_ptr(),
                                            st.tval.data_ptr(), st.work.data_ptr(), st.work_bytes, stream)
        if rc != native.PBCG_OK:
            raise native.PbcgError(rc, native.pbicgstab_last_error())
        lam, _ = _solve(st, st.trowptr, st.tcol, st.tval, gx.contiguous(), rtol, maxit, rp)
        grad_values = torch.empty_like(values)
        rc = native.pbicgstab_csr_value_grad(st.n, st.rowptr.data_ptr(), st.col.data_ptr(), lam.data_ptr(),
                                             x.data_ptr(), grad_values.data_ptr(), stream)
        if rc != native.PBCG_OK:
            raise native.PbcgError(rc, native.pbicgstab_last_error())
        return grad_values, lam, None, None, None, None


def sparse_solve(values, b, structure, rtol=1e-12, maxit=20000, replace_period=50):
    return SparseSolve.apply(values, b, structure, rtol, maxit, replace_period)
