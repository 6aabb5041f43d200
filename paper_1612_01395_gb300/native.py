"""Python binding of the C ABI in include/pbicgstab.h (argument marshalling only).

Every function here has the name of the C entry point it calls and takes raw
pointers (Python ints) and sizes, exactly like the C ABI; ``Solver`` is a thin
convenience layer that keeps device buffers in PyTorch tensors. All solver
arithmetic runs in the CUDA library; if the library is not built this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_INCLUDE = os.path.join(_ROOT, "include")
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libpbicgstab.so")
CHECK_LIB_PATH = os.path.join(_BUILD, "libpbicgstab_check.so")   # -DPBCG_CHECK build
NVCC_ARCH = "-gencode=arch=compute_103a,code=sm_103a"

PBCG_OK, PBCG_NOT_CONVERGED, PBCG_BREAKDOWN, PBCG_NONFINITE = 0, 1, 2, 3
PBCG_ERR_ARG, PBCG_ERR_CUDA, PBCG_ERR_OOM, PBCG_ERR_TIMEOUT = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", 3: "NONFINITE", 4: "ERR_ARG",
                5: "ERR_CUDA", 6: "ERR_OOM", 7: "ERR_TIMEOUT"}
PBCG_PREC_NONE, PBCG_PREC_JACOBI = 0, 1

# Exported symbols, as declared in include/pbicgstab.h.
EXPORTS = ["pbicgstab_workspace_bytes", "pbicgstab_workspace_bytes_prec", "pbicgstab_create_csr", "pbicgstab_create_stencil",
           "pbicgstab_solve", "bicgstab_solve", "pbicgstab_solve_host", "pbicgstab_spmv",
           "pbicgstab_size", "pbicgstab_destroy", "pbicgstab_last_error", "pbicgstab_solve_csr_noalloc",
           "pbicgstab_solve_mixed", "pbicgstab_batched_workspace_bytes", "pbicgstab_solve_batched",
           "pbicgstab_transpose_work_bytes", "pbicgstab_csr_transpose", "pbicgstab_csr_value_grad",
           "pbicgstab_probe_sync_timeout", "pbicgstab_batched_autotune", "pbicgstab_check_faults"]
PBCG_VALUES_F32, PBCG_VALUES_BF16 = 0, 1
# Largest system the allocation-free entry point accepts (PBCG_NOALLOC_MAX_N).
PBCG_NOALLOC_MAX_N = 32768


class PbcgCoef(ctypes.Structure):
    _fields_ = [("value", ctypes.c_double), ("data", ctypes.c_void_p), ("stride", ctypes.c_int64 * 3),
                ("len", ctypes.c_int64), ("data2", ctypes.c_void_p), ("stride2", ctypes.c_int64 * 3),
                ("len2", ctypes.c_int64)]


class PbcgStencil(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("coef", PbcgCoef * 7)]


class PbcgOpts(ctypes.Structure):
    _fields_ = [("max_replacements", ctypes.c_int32), ("fixed_iters", ctypes.c_int32),
                ("d_history", ctypes.c_void_p), ("plain_variant", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("d_inner_history", ctypes.c_void_p), ("cluster", ctypes.c_int32), ("stall_steps", ctypes.c_int32)]


class PbcgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("half_step", ctypes.c_int32),
                ("n_replacements", ctypes.c_int32), ("nr0", ctypes.c_double),
                ("rel_res_recursive", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32), ("grid_syncs", ctypes.c_int32),
                ("spmvs", ctypes.c_int32), ("kernel_ms", ctypes.c_float), ("cluster", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PbcgMixedInfo(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("inner_iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("nr0", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("grid_syncs", ctypes.c_int32), ("spmvs", ctypes.c_int32), ("kernel_ms", ctypes.c_float),
                ("restored", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PbcgBatch(ctypes.Structure):
    _fields_ = [("nsys", ctypes.c_int32), ("nnz", ctypes.c_int32), ("d_row_offset", ctypes.c_void_p),
                ("d_rowptr", ctypes.c_void_p), ("d_col", ctypes.c_void_p), ("d_val", ctypes.c_void_p)]


class PbcgBatchOpts(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int32), ("fixed_iters", ctypes.c_int32),
                ("cluster_min_rows", ctypes.c_int64), ("d_history", ctypes.c_void_p),
                ("history_stride", ctypes.c_int64)]


class PbcgBatchResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("half_step", ctypes.c_int32),
                ("n_replacements", ctypes.c_int32), ("rel_res_recursive", ctypes.c_double),
                ("rel_res_true", ctypes.c_double)]


def sources():
    return [os.path.join(_CSRC, f) for f in sorted(os.listdir(_CSRC)) if f.endswith((".cu", ".cuh"))] + \
        [os.path.join(_INCLUDE, "pbicgstab.h")]


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile the CUDA library for sm_103a with nvcc (in-tree, under _build/).
    check=True builds the bounds-checked variant (-DPBCG_CHECK) at CHECK_LIB_PATH."""
    os.makedirs(_BUILD, exist_ok=True)
    out = CHECK_LIB_PATH if check else LIB_PATH
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(p) for p in sources())
        if os.path.getmtime(out) >= newest:
            return out
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["nvcc", NVCC_ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", _INCLUDE, "-o", tmp, os.path.join(_CSRC, "pbicgstab.cu")]
    if check:
        cmd.insert(1, "-DPBCG_CHECK")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


_lib = None


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run paper_1612_01395_gb300.native.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, f64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
        L.pbicgstab_workspace_bytes.argtypes = [i32]
        L.pbicgstab_workspace_bytes.restype = sz
        L.pbicgstab_workspace_bytes_prec.argtypes = [i32]
        L.pbicgstab_workspace_bytes_prec.restype = sz
        L.pbicgstab_create_csr.argtypes = [i32, i32, vp, vp, vp, ctypes.c_int, vp, sz, vp, ctypes.POINTER(vp)]
        L.pbicgstab_create_stencil.argtypes = [ctypes.POINTER(PbcgStencil), ctypes.c_int, vp, sz, vp,
                                               ctypes.POINTER(vp)]
        L.pbicgstab_solve.argtypes = [vp, vp, vp, f64, i32, i32, ctypes.POINTER(PbcgOpts), ctypes.POINTER(PbcgInfo)]
        L.bicgstab_solve.argtypes = [vp, vp, vp, f64, i32, ctypes.POINTER(PbcgOpts), ctypes.POINTER(PbcgInfo)]
        L.pbicgstab_solve_host.argtypes = [vp, i32, vp, vp, f64, i32, i32, ctypes.POINTER(PbcgOpts),
                                           ctypes.POINTER(PbcgInfo)]
        L.pbicgstab_spmv.argtypes = [vp, vp, vp]
        L.pbicgstab_solve_mixed.argtypes = [vp, vp, i32, vp, vp, f64, i32, f64, i32, ctypes.POINTER(PbcgOpts),
                                            ctypes.POINTER(PbcgMixedInfo)]
        L.pbicgstab_batched_workspace_bytes.argtypes = [ctypes.c_int64]
        L.pbicgstab_batched_workspace_bytes.restype = sz
        L.pbicgstab_solve_batched.argtypes = [ctypes.POINTER(PbcgBatch), ctypes.c_int64, vp, vp, f64, i32, i32,
                                              ctypes.POINTER(PbcgBatchOpts), vp, sz, vp, vp]
        L.pbicgstab_solve_batched.restype = ctypes.c_int
        L.pbicgstab_transpose_work_bytes.argtypes = [i32]
        L.pbicgstab_transpose_work_bytes.restype = sz
        L.pbicgstab_csr_transpose.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.pbicgstab_csr_transpose.restype = ctypes.c_int
        L.pbicgstab_csr_value_grad.argtypes = [i32, vp, vp, vp, vp, vp, vp]
        L.pbicgstab_probe_sync_timeout.argtypes = [vp, i32, ctypes.POINTER(i32)]
        L.pbicgstab_check_faults.argtypes = []
        L.pbicgstab_check_faults.restype = i32
        L.pbicgstab_batched_autotune.argtypes = [ctypes.POINTER(PbcgBatch), ctypes.c_int64, vp, vp, f64, i32, i32,
                                                 vp, sz, vp, vp, ctypes.POINTER(PbcgBatchOpts),
                                                 ctypes.POINTER(ctypes.c_float)]
        L.pbicgstab_batched_autotune.restype = ctypes.c_int
        L.pbicgstab_probe_sync_timeout.restype = ctypes.c_int
        L.pbicgstab_csr_value_grad.restype = ctypes.c_int
        L.pbicgstab_solve_csr_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, f64, i32, i32,
                                                  ctypes.POINTER(PbcgOpts), vp, ctypes.POINTER(PbcgInfo)]
        L.pbicgstab_size.argtypes = [vp]
        L.pbicgstab_size.restype = i32
        L.pbicgstab_destroy.argtypes = [vp]
        L.pbicgstab_destroy.restype = None
        L.pbicgstab_last_error.argtypes = []
        L.pbicgstab_last_error.restype = ctypes.c_char_p
        for name in ("pbicgstab_create_csr", "pbicgstab_create_stencil", "pbicgstab_solve", "bicgstab_solve",
                     "pbicgstab_solve_host", "pbicgstab_spmv", "pbicgstab_solve_csr_noalloc",
                     "pbicgstab_solve_mixed"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class PbcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _opts(max_replacements=-1, fixed_iters=0, d_history=None, plain_variant=0, grid=0, d_inner_history=None,
          cluster=0, stall_steps=0):
    return PbcgOpts(int(max_replacements), int(fixed_iters), d_history or None, int(plain_variant), int(grid),
                    d_inner_history or None, int(cluster), int(stall_steps))


# ---- thin wrappers with the C names ---------------------------------------------------------

def pbicgstab_workspace_bytes(n: int) -> int:
    return int(lib().pbicgstab_workspace_bytes(int(n)))


def pbicgstab_workspace_bytes_prec(n: int) -> int:
    return int(lib().pbicgstab_workspace_bytes_prec(int(n)))


def pbicgstab_last_error() -> str:
    return lib().pbicgstab_last_error().decode()


def _check_create(st):
    if st != PBCG_OK:
        raise PbcgError(st, pbicgstab_last_error())


def pbicgstab_create_csr(n, nnz, d_rowptr, d_col, d_val, prec, d_ws, ws_bytes, stream) -> int:
    out = ctypes.c_void_p()
    _check_create(lib().pbicgstab_create_csr(int(n), int(nnz), d_rowptr, d_col, d_val, int(prec), d_ws,
                                             int(ws_bytes), stream, ctypes.byref(out)))
    return out.value


def pbicgstab_create_stencil(desc: PbcgStencil, prec, d_ws, ws_bytes, stream) -> int:
    out = ctypes.c_void_p()
    _check_create(lib().pbicgstab_create_stencil(ctypes.byref(desc), int(prec), d_ws, int(ws_bytes), stream,
                                                 ctypes.byref(out)))
    return out.value


def pbicgstab_solve(h, d_b, d_x, rtol, maxit, replace_period=0, **opts):
    info = PbcgInfo()
    o = _opts(**opts)
    st = lib().pbicgstab_solve(h, d_b, d_x, float(rtol), int(maxit), int(replace_period), ctypes.byref(o),
                               ctypes.byref(info))
    return st, info


def bicgstab_solve(h, d_b, d_x, rtol, maxit, **opts):
    info = PbcgInfo()
    o = _opts(**opts)
    st = lib().bicgstab_solve(h, d_b, d_x, float(rtol), int(maxit), ctypes.byref(o), ctypes.byref(info))
    return st, info


def pbicgstab_solve_host(h, method, h_b, h_x, rtol, maxit, replace_period=0, **opts):
    info = PbcgInfo()
    o = _opts(**opts)
    st = lib().pbicgstab_solve_host(h, int(method), h_b, h_x, float(rtol), int(maxit), int(replace_period),
                                    ctypes.byref(o), ctypes.byref(info))
    return st, info


def pbicgstab_solve_csr_noalloc(n, nnz, d_rowptr, d_col, d_val, d_b, d_x, rtol, maxit, replace_period, stream,
                                **opts):
    """Solve with a CSR matrix without any device allocation, for callers that
    may not allocate (see include/pbicgstab.h); n <= PBCG_NOALLOC_MAX_N."""
    info = PbcgInfo()
    o = _opts(**opts)
    st = lib().pbicgstab_solve_csr_noalloc(int(n), int(nnz), d_rowptr, d_col, d_val, d_b, d_x, float(rtol),
                                           int(maxit), int(replace_period), ctypes.byref(o), stream,
                                           ctypes.byref(info))
    return st, info


def pbicgstab_solve_mixed(h, d_val_lowp, lowp_type, d_b, d_x, rtol, max_outer, inner_rtol, inner_maxit, **opts):
    info = PbcgMixedInfo()
    o = _opts(**opts)
    st = lib().pbicgstab_solve_mixed(h, d_val_lowp, int(lowp_type), d_b, d_x, float(rtol), int(max_outer),
                                     float(inner_rtol), int(inner_maxit), ctypes.byref(o), ctypes.byref(info))
    return st, info


def pbicgstab_batched_workspace_bytes(total_rows: int) -> int:
    return int(lib().pbicgstab_batched_workspace_bytes(int(total_rows)))


def pbicgstab_solve_batched(batch: PbcgBatch, total_rows, d_b, d_x, rtol, maxit, replace_period, opts, d_ws,
                            ws_bytes, d_results, stream) -> int:
    """opts: a PbcgBatchOpts or None (defaults)."""
    return lib().pbicgstab_solve_batched(ctypes.byref(batch), int(total_rows), d_b, d_x, float(rtol), int(maxit),
                                         int(replace_period), ctypes.byref(opts) if opts is not None else None,
                                         d_ws, int(ws_bytes), d_results, stream)


class BatchSolver:
    """Device copies of a problems.Batch plus workspace and per-system results."""

    RESULT_DTYPE = None

    def __init__(self, batch):
        import torch
        import numpy as np
        self.torch = torch
        self.total = batch.total_rows
        self.nsys = batch.nsys
        self.row_offset = torch.as_tensor(batch.row_offset, dtype=torch.int64).cuda()
        self.rowptr = torch.as_tensor(batch.rowptr, dtype=torch.int32).cuda()
        self.col = torch.as_tensor(batch.col, dtype=torch.int32).cuda()
        self.val = torch.as_tensor(batch.val, dtype=torch.float64).cuda()
        nb = pbicgstab_batched_workspace_bytes(self.total)
        self.ws = torch.empty(nb // 8 + 64, dtype=torch.float64, device="cuda")
        self.ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.ws_bytes = nb
        self.results = torch.zeros(self.nsys * ctypes.sizeof(PbcgBatchResult) // 8, dtype=torch.float64,
                                   device="cuda")
        self.desc = PbcgBatch(self.nsys, int(batch.rowptr[-1]), self.row_offset.data_ptr(), self.rowptr.data_ptr(),
                              self.col.data_ptr(), self.val.data_ptr())
        self._np = np

    def launch(self, b, x, rtol=1e-8, maxit=1000, replace_period=0, stream=None, cluster_size=0,
               cluster_min_rows=0, fixed_iters=0, history=None):
        """Enqueue the batched solve (asynchronous). cluster_size / cluster_min_rows:
        the launch shape (0 = library defaults). fixed_iters > 0 runs every system
        exactly that many iterations; history: a float64 CUDA tensor of shape
        (nsys, stride) receiving each system's residual norms."""
        torch = self.torch
        st = (stream or torch.cuda.current_stream()).cuda_stream
        hp, hs = (history.data_ptr(), history.shape[1]) if history is not None else (None, 0)
        opts = PbcgBatchOpts(int(cluster_size), int(fixed_iters), int(cluster_min_rows), hp, int(hs))
        rc = pbicgstab_solve_batched(self.desc, self.total, b.data_ptr(), x.data_ptr(), rtol, maxit, replace_period,
                                     opts, self.ws_ptr, self.ws_bytes, self.results.data_ptr(), st)
        if rc != PBCG_OK:
            raise PbcgError(rc, pbicgstab_last_error())

    def autotune(self, b, x, rtol=1e-8, maxit=1000, replace_period=0, stream=None):
        """Time the candidate launch shapes (library autotuner; x is overwritten
        with the best shape's solution). Returns (cluster_size, cluster_min_rows, ms)."""
        torch = self.torch
        st = (stream or torch.cuda.current_stream()).cuda_stream
        best = PbcgBatchOpts()
        ms = ctypes.c_float(0.0)
        rc = lib().pbicgstab_batched_autotune(ctypes.byref(self.desc), int(self.total), b.data_ptr(), x.data_ptr(),
                                              float(rtol), int(maxit), int(replace_period), self.ws_ptr,
                                              int(self.ws_bytes), self.results.data_ptr(), st, ctypes.byref(best),
                                              ctypes.byref(ms))
        if rc != PBCG_OK:
            raise PbcgError(rc, pbicgstab_last_error())
        return best.cluster_size, best.cluster_min_rows, ms.value

    def fetch_results(self):
        """Per-system results as a numpy structured array (synchronises)."""
        np = self._np
        raw = self.results.cpu().numpy().tobytes()
        dt = np.dtype([("iters", np.int32), ("status", np.int32), ("half_step", np.int32),
                       ("n_replacements", np.int32), ("rel_res_recursive", np.float64),
                       ("rel_res_true", np.float64)])
        return np.frombuffer(raw, dtype=dt, count=self.nsys)


def pbicgstab_transpose_work_bytes(n: int) -> int:
    return int(lib().pbicgstab_transpose_work_bytes(int(n)))


def pbicgstab_csr_transpose(n, nnz, d_rowptr, d_col, d_val, d_trowptr, d_tcol, d_tval, d_work, work_bytes,
                            stream) -> int:
    return lib().pbicgstab_csr_transpose(int(n), int(nnz), d_rowptr, d_col, d_val, d_trowptr, d_tcol, d_tval,
                                         d_work, int(work_bytes), stream)


def pbicgstab_csr_value_grad(n, d_rowptr, d_col, d_lambda, d_x, d_grad, stream) -> int:
    return lib().pbicgstab_csr_value_grad(int(n), d_rowptr, d_col, d_lambda, d_x, d_grad, stream)


def pbicgstab_check_faults() -> int:
    """Bounds-checked build: source line of the first out-of-range index since
    the last call (0: none); -1 from the default build."""
    return int(lib().pbicgstab_check_faults())


def pbicgstab_probe_sync_timeout(h, limit_ms):
    """Returns (call status, status the device recorded)."""
    st = ctypes.c_int32(-1)
    rc = lib().pbicgstab_probe_sync_timeout(h, int(limit_ms), ctypes.byref(st))
    return rc, st.value


def pbicgstab_spmv(h, d_x, d_y) -> int:
    return lib().pbicgstab_spmv(h, d_x, d_y)


def pbicgstab_size(h) -> int:
    return lib().pbicgstab_size(h)


def pbicgstab_destroy(h) -> None:
    lib().pbicgstab_destroy(h)


# ---- convenience layer over torch tensors ----------------------------------------------------

class Solver:
    """A handle plus the device buffers it refers to, kept alive in torch tensors.

    ``Solver.from_csr(csr)`` / ``Solver.from_stencil(stencil)`` take the host
    structures of ``problems`` (numpy arrays) and copy them to the device.
    """

    def __init__(self):
        self.h = None
        self._keep = []

    @staticmethod
    def _torch():
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        return torch

    def _workspace(self, n, stream, prec=PBCG_PREC_NONE):
        torch = self._torch()
        nbytes = pbicgstab_workspace_bytes_prec(n) if prec == PBCG_PREC_JACOBI else pbicgstab_workspace_bytes(n)
        ws = torch.empty(nbytes // 8 + 64, dtype=torch.float64, device="cuda")
        base = ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        self._keep.append(ws)
        self.ws_bytes = nbytes
        self.n = n
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        return aligned, nbytes

    @classmethod
    def from_csr(cls, A, stream=None, prec=PBCG_PREC_NONE) -> "Solver":
        self = cls()
        torch = self._torch()
        rowptr = torch.as_tensor(A.rowptr, dtype=torch.int32).cuda()
        col = torch.as_tensor(A.col, dtype=torch.int32).cuda()
        val = torch.as_tensor(A.val, dtype=torch.float64).cuda()
        self._keep += [rowptr, col, val]
        ws, nb = self._workspace(A.n, stream, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.h = pbicgstab_create_csr(A.n, A.nnz, rowptr.data_ptr(), col.data_ptr() if A.nnz else None,
                                      val.data_ptr() if A.nnz else None, prec, ws, nb, self.stream.cuda_stream)
        torch.cuda.synchronize()
        self.create_s = time.perf_counter() - t0   # the C create call alone (arrays already on the device)
        return self

    @classmethod
    def from_stencil(cls, st, stream=None, prec=PBCG_PREC_NONE) -> "Solver":
        self = cls()
        torch = self._torch()
        desc = PbcgStencil()
        desc.nx, desc.ny, desc.nz = st.nx, st.ny, st.nz
        for d, c in enumerate(st.coefs):
            cd = desc.coef[d]
            cd.value = float(c.value)
            if c.table is not None:
                t = torch.as_tensor(c.table, dtype=torch.float64).cuda()
                self._keep.append(t)
                cd.data = t.data_ptr()
                cd.len = t.numel()
                cd.stride[:] = [int(v) for v in c.stride]
            if c.table2 is not None:
                t2 = torch.as_tensor(c.table2, dtype=torch.float64).cuda()
                self._keep.append(t2)
                cd.data2 = t2.data_ptr()
                cd.len2 = t2.numel()
                cd.stride2[:] = [int(v) for v in c.stride2]
        ws, nb = self._workspace(st.n, stream, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.h = pbicgstab_create_stencil(desc, prec, ws, nb, self.stream.cuda_stream)
        torch.cuda.synchronize()
        self.create_s = time.perf_counter() - t0   # the C create call alone (tables already on the device)
        return self

    def spmv(self, x):
        torch = self._torch()
        y = torch.empty_like(x)
        st = pbicgstab_spmv(self.h, x.data_ptr(), y.data_ptr())
        if st != PBCG_OK:
            raise PbcgError(st, pbicgstab_last_error())
        return y

    def solve(self, b, x0=None, rtol=1e-8, maxit=1000, replace_period=0, method="pipelined",
              history=False, **opts):
        """Solve A x = b on the device; returns (x, info dict[, history tensor])."""
        torch = self._torch()
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        hist = None
        if history:
            steps = opts.get("fixed_iters", 0) or maxit
            hist = torch.full((steps + 1,), float("nan"), dtype=torch.float64, device=b.device)
            opts["d_history"] = hist.data_ptr()
        if method == "pipelined":
            st, info = pbicgstab_solve(self.h, b.data_ptr(), x.data_ptr(), rtol, maxit, replace_period, **opts)
        elif method == "standard":
            st, info = bicgstab_solve(self.h, b.data_ptr(), x.data_ptr(), rtol, maxit, **opts)
        else:
            raise ValueError(method)
        if st in (PBCG_ERR_ARG, PBCG_ERR_CUDA, PBCG_ERR_OOM, PBCG_ERR_TIMEOUT):
            raise PbcgError(st, pbicgstab_last_error())
        d = info.as_dict()
        if hist is not None:
            return x, d, hist[: d["iters"] + 1]
        return x, d

    def solve_mixed(self, b, values_lowp, lowp_type=PBCG_VALUES_F32, x0=None, rtol=1e-10, max_outer=30,
                    inner_rtol=1e-4, inner_maxit=2000, history=False, inner_history=False, **opts):
        """FP64 refinement around FP32 Algorithm 9. CSR handles: values_lowp is a
        float32 or bfloat16 tensor with the CSR values; stencil handles: None
        (the library rounds the coefficient tables). Returns (x, info[, history]
        [, inner_history]): the FP64 residual norm before each step, and the
        recursive residual norms of the first step's inner solve."""
        torch = self._torch()
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        hist = ihist = None
        if history:
            hist = torch.full((max_outer + 1,), float("nan"), dtype=torch.float64, device=b.device)
            opts["d_history"] = hist.data_ptr()
        if inner_history:
            steps = opts.get("fixed_iters", 0) or inner_maxit
            ihist = torch.full((steps + 1,), float("nan"), dtype=torch.float64, device=b.device)
            opts["d_inner_history"] = ihist.data_ptr()
        vp = values_lowp.data_ptr() if values_lowp is not None else None
        st, info = pbicgstab_solve_mixed(self.h, vp, lowp_type, b.data_ptr(), x.data_ptr(),
                                         rtol, max_outer, inner_rtol, inner_maxit, **opts)
        if st in (PBCG_ERR_ARG, PBCG_ERR_CUDA, PBCG_ERR_OOM, PBCG_ERR_TIMEOUT):
            raise PbcgError(st, pbicgstab_last_error())
        d = info.as_dict()
        out = (x, d)
        if hist is not None:
            out += (hist[: d["outer"] + 1],)
        if ihist is not None:
            out += (ihist,)
        return out

    def close(self):
        if self.h:
            pbicgstab_destroy(self.h)
            self.h = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
