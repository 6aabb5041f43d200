"""The C-ABI library builds, loads and exports every symbol include/*.h declares (CPU, no compute)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1612_01395_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text):
            name = m.group(1)
            if name not in ("sizeof",):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    native.build()
    return native.lib()


def test_header_declares_the_binding_exports():
    assert declared_functions() == set(native.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_workspace_query_without_gpu(lib):
    n = 1000
    nb = native.pbicgstab_workspace_bytes(n)
    stride = (n + 31) // 32 * 32
    assert nb >= 12 * stride * 8
    assert native.pbicgstab_workspace_bytes(-1) == 0


def test_argument_errors_need_no_gpu(lib):
    out = ctypes.c_void_p()
    st = lib.pbicgstab_create_csr(-1, 0, None, None, None, 0, None, 0, None, ctypes.byref(out))
    assert st == native.PBCG_ERR_ARG
    assert "n and nnz" in native.pbicgstab_last_error()
    info = native.PbcgInfo()
    assert lib.pbicgstab_solve(None, None, None, 1e-8, 10, 0, None, ctypes.byref(info)) == native.PBCG_ERR_ARG
    assert lib.pbicgstab_spmv(None, None, None) == native.PBCG_ERR_ARG
    lib.pbicgstab_destroy(None)


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    import subprocess
    src = tmp_path / "layout.c"
    fields = {
        "pbcg_coef": native.PbcgCoef, "pbcg_stencil": native.PbcgStencil,
        "pbcg_opts": native.PbcgOpts, "pbcg_info": native.PbcgInfo, "pbcg_mixed_info": native.PbcgMixedInfo,
        "pbcg_batch": native.PbcgBatch, "pbcg_batch_result": native.PbcgBatchResult,
        "pbcg_batch_opts": native.PbcgBatchOpts,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pbicgstab.h"', "int main(void){"]
    for cname, py in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, py in fields.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_bounds_checked_build_compiles_and_exports():
    """-DPBCG_CHECK build (nvcc cross-compiles without a GPU): same exports."""
    import ctypes
    path = native.build(check=True)
    L = ctypes.CDLL(path)
    for name in native.EXPORTS:
        assert hasattr(L, name), name


def test_batched_option_errors_need_no_gpu(lib):
    """Host-side checks of the batched options run before any CUDA call."""
    batch = native.PbcgBatch(1, 4, 256, 512, 768, 1024)   # fake device addresses, never dereferenced
    ws_bytes = native.pbicgstab_batched_workspace_bytes(4)
    res = native.PbcgBatchResult()
    for opts, msg in ((native.PbcgBatchOpts(1, -1, 0, None, 0), "fixed_iters"),
                      (native.PbcgBatchOpts(1, 20, 0, 4096, 10), "history_stride"),
                      (native.PbcgBatchOpts(3, 0, 0, None, 0), "cluster_size")):
        st = lib.pbicgstab_solve_batched(ctypes.byref(batch), 4, 256, 512, 1e-8, 100, 0, ctypes.byref(opts), 4096,
                                         ws_bytes, ctypes.addressof(res), None)
        assert st == native.PBCG_ERR_ARG, msg
        assert msg in native.pbicgstab_last_error()
