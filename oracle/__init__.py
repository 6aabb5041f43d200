"""CPU oracle for (pipelined) BiCGStab -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never loads it and shares no code with it.

* ``oracle.c``     plain FP64 C: Algorithm 7, Algorithm 8 and Algorithm 9 with
                   residual replacement (Section 4.2), built with gcc here.
* ``rational.py``  the same three algorithms in exact rational arithmetic for
                   tiny systems (Python ``fractions``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
# OpenMP build of the same source, for timing the oracle on all host cores
# (bench.py's CPU legs); the tests use the single-threaded build above.
_OMP_LIB_PATH = os.path.join(_BUILD, "liboracle_omp.so")

CONVERGED, NOT_CONVERGED, BREAKDOWN, NONFINITE, ERR_ARG, ERR_OOM = range(6)


class OInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("half_step", ctypes.c_int32),
                ("n_replacements", ctypes.c_int32), ("nr0", ctypes.c_double),
                ("rel_res_rec", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("flops", ctypes.c_double), ("spmvs", ctypes.c_int32), ("pad", ctypes.c_int32)]


def build(force: bool = False, omp: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -ffp-contract=off);
    omp=True: the OpenMP build (-fopenmp) used only to time the oracle."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _OMP_LIB_PATH if omp else _LIB_PATH
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.check_call(cmd)
        os.replace(tmp, path)
    return path


_libs = {}


def lib(omp: bool = False):
    """The single-threaded oracle library, or (omp=True) its OpenMP build."""
    if omp not in _libs:
        L = ctypes.CDLL(build(omp=omp))
        _libs[omp] = L
        _lib = L
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i32, f64 = ctypes.c_int32, ctypes.c_double
        _lib.o_spmv.argtypes = [i32, ip, ip, dp, dp, dp]
        _lib.o_dot.argtypes = [i32, dp, dp]
        _lib.o_dot.restype = f64
        common = [i32, ip, ip, dp, dp, dp, f64, i32, i32]
        _lib.o_bicgstab.argtypes = common + [dp, dp, dp, ctypes.POINTER(OInfo)]
        _lib.o_cabicgstab.argtypes = common + [dp, dp, dp, ctypes.POINTER(OInfo)]
        _lib.o_pbicgstab.argtypes = common + [i32, i32, i32, i32, dp, dp, dp, dp, ctypes.POINTER(OInfo)]
        pcommon = [i32, ip, ip, dp, dp, dp, dp, f64, i32, i32]
        _lib.o_bicgstab_prec.argtypes = pcommon + [dp, dp, dp, ctypes.POINTER(OInfo)]
        _lib.o_pbicgstab_prec.argtypes = pcommon + [i32, i32, dp, dp, dp, ctypes.POINTER(OInfo)]
        _lib.o_num_threads.restype = ctypes.c_int
    return _libs[omp]


def num_threads(omp: bool = False) -> int:
    """Threads the oracle build runs on (1 for the parity build)."""
    return int(lib(omp).o_num_threads())


def _p(a: Optional[np.ndarray], ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _csr_args(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    return rowptr, col, val


def spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x with each row summed in CSR order (FP64)."""
    rowptr, col, val = _csr_args(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n)
    lib().o_spmv(A.n, _p(rowptr, ctypes.c_int32), _p(col, ctypes.c_int32), _p(val), _p(x), _p(y))
    return y


def dot(a: np.ndarray, b: np.ndarray) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().o_dot(a.size, _p(a), _p(b))


@dataclass
class Result:
    x: np.ndarray
    iters: int
    status: int
    half_step: bool
    n_replacements: int
    nr0: float
    rel_res_rec: float
    rel_res_true: float
    flops: float
    spmvs: int
    hist: np.ndarray                 # ||r_i||, i = 0..iters
    trace_x: Optional[np.ndarray] = None
    trace_r: Optional[np.ndarray] = None
    work: Optional[dict] = None


def _run(method: str, A, b, x0, rtol, maxit, fixed_iters, trace, replace_period=0,
         max_replacements=-1, alpha_eq5=False, keep_work=False, rr_placement=0, omp=False) -> Result:
    rowptr, col, val = _csr_args(A)
    n = A.n
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    steps = fixed_iters if fixed_iters > 0 else maxit
    hist = np.full(steps + 1, np.nan)
    tx = np.full((steps + 1, n), np.nan) if trace else None
    trr = np.full((steps + 1, n), np.nan) if trace else None
    work = np.zeros(10 * max(n, 1)) if keep_work else None
    info = OInfo()
    L = lib(omp)
    args = [n, _p(rowptr, ctypes.c_int32), _p(col, ctypes.c_int32), _p(val), _p(b), _p(x),
            float(rtol), int(maxit), int(fixed_iters)]
    if method == "bicgstab":
        L.o_bicgstab(*args, _p(hist), _p(tx), _p(trr), ctypes.byref(info))
    elif method == "cabicgstab":
        L.o_cabicgstab(*args, _p(hist), _p(tx), _p(trr), ctypes.byref(info))
    elif method == "pbicgstab":
        L.o_pbicgstab(*args, int(replace_period), int(max_replacements), int(bool(alpha_eq5)),
                      int(rr_placement), _p(hist), _p(tx), _p(trr), _p(work), ctypes.byref(info))
    else:
        raise ValueError(method)
    k = info.iters
    wd = None
    if keep_work:
        names = ["r", "r0", "p", "s", "z", "q", "y", "w", "t", "v"]
        wd = {nm: work[i * n:(i + 1) * n].copy() for i, nm in enumerate(names)}
    return Result(x=x, iters=k, status=info.status, half_step=bool(info.half_step),
                  n_replacements=info.n_replacements, nr0=info.nr0, rel_res_rec=info.rel_res_rec,
                  rel_res_true=info.rel_res_true, flops=info.flops, spmvs=info.spmvs,
                  hist=hist[:k + 1].copy(),
                  trace_x=None if tx is None else tx[:k + 1].copy(),
                  trace_r=None if trr is None else trr[:k + 1].copy(), work=wd)


def jacobi_minv(A) -> np.ndarray:
    """1 / diag(A) for the Jacobi preconditioner (M = diag(A))."""
    d = np.zeros(A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    on = A.col == rows
    d[rows[on]] = A.val[on]
    return 1.0 / d


def _run_prec(method, A, minv, b, x0, rtol, maxit, fixed_iters, trace, replace_period=0, max_replacements=-1):
    rowptr, col, val = _csr_args(A)
    n = A.n
    minv = np.ascontiguousarray(minv, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    steps = fixed_iters if fixed_iters > 0 else maxit
    hist = np.full(steps + 1, np.nan)
    tx = np.full((steps + 1, n), np.nan) if trace else None
    trr = np.full((steps + 1, n), np.nan) if trace else None
    info = OInfo()
    L = lib()
    args = [n, _p(rowptr, ctypes.c_int32), _p(col, ctypes.c_int32), _p(val), _p(minv), _p(b), _p(x),
            float(rtol), int(maxit), int(fixed_iters)]
    if method == "bicgstab":
        L.o_bicgstab_prec(*args, _p(hist), _p(tx), _p(trr), ctypes.byref(info))
    else:
        L.o_pbicgstab_prec(*args, int(replace_period), int(max_replacements), _p(hist), _p(tx), _p(trr),
                           ctypes.byref(info))
    k = info.iters
    return Result(x=x, iters=k, status=info.status, half_step=bool(info.half_step),
                  n_replacements=info.n_replacements, nr0=info.nr0, rel_res_rec=info.rel_res_rec,
                  rel_res_true=info.rel_res_true, flops=info.flops, spmvs=info.spmvs, hist=hist[:k + 1].copy(),
                  trace_x=None if tx is None else tx[:k + 1].copy(),
                  trace_r=None if trr is None else trr[:k + 1].copy())


def bicgstab_prec(A, minv, b, x0=None, rtol=1e-8, maxit=1000, fixed_iters=0, trace=False) -> Result:
    """Algorithm 10 (preconditioned BiCGStab) with M^{-1} u = minv * u, plain FP64."""
    return _run_prec("bicgstab", A, minv, b, x0, rtol, maxit, fixed_iters, trace)


def pbicgstab_prec(A, minv, b, x0=None, rtol=1e-8, maxit=1000, fixed_iters=0, trace=False, replace_period=0,
                   max_replacements=-1) -> Result:
    """Algorithm 11 (preconditioned pipelined BiCGStab) with M^{-1} u = minv * u and residual
    replacement every ``replace_period`` iterations, plain FP64."""
    return _run_prec("pbicgstab", A, minv, b, x0, rtol, maxit, fixed_iters, trace, replace_period,
                     max_replacements)


def bicgstab(A, b, x0=None, rtol=1e-8, maxit=1000, fixed_iters=0, trace=False, omp=False) -> Result:
    """Algorithm 7 (standard BiCGStab) in plain FP64 (omp=True: the OpenMP build)."""
    return _run("bicgstab", A, b, x0, rtol, maxit, fixed_iters, trace, omp=omp)


def cabicgstab(A, b, x0=None, rtol=1e-8, maxit=1000, fixed_iters=0, trace=False) -> Result:
    """Algorithm 8 (communication-avoiding BiCGStab) in plain FP64."""
    return _run("cabicgstab", A, b, x0, rtol, maxit, fixed_iters, trace)


def pbicgstab(A, b, x0=None, rtol=1e-8, maxit=1000, fixed_iters=0, trace=False,
              replace_period=0, max_replacements=-1, alpha_eq5=False, keep_work=False,
              rr_placement=0, omp=False) -> Result:
    """Algorithm 9 (pipelined BiCGStab) with residual replacement every
    ``replace_period`` iterations (0 = off), in plain FP64. ``rr_placement`` 0 is
    the default (split) placement, 1 the literal late placement (see oracle.c).
    omp=True runs the OpenMP build (timing only)."""
    return _run("pbicgstab", A, b, x0, rtol, maxit, fixed_iters, trace, replace_period,
                max_replacements, alpha_eq5, keep_work, rr_placement, omp)
