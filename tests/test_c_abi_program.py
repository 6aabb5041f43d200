"""The C ABI used from a C program alone (tests/c_abi_solve.c): compiled and
linked against the library on CPU; run on a GB300."""
import json
import os
import subprocess

import pytest

from paper_1612_01395_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def compile_program(tmp_path):
    native.build()
    exe = tmp_path / "c_abi_solve"
    build_dir = os.path.dirname(native.LIB_PATH)
    cmd = ["gcc", "-O2", "-std=c11", os.path.join(ROOT, "tests", "c_abi_solve.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", build_dir, "-lpbicgstab", "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm",
           f"-Wl,-rpath,{build_dir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-o", str(exe)]
    subprocess.check_call(cmd)
    return exe


def test_c_program_compiles_and_links_against_the_library(tmp_path):
    exe = compile_program(tmp_path)
    assert exe.exists()


@pytest.mark.gpu
def test_c_program_solves_through_the_abi(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = compile_program(tmp_path)
    out = subprocess.run([str(exe), "64"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr + out.stdout
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["pbicgstab"]["status"] == native.PBCG_OK and r["bicgstab"]["status"] == native.PBCG_OK
    assert r["pbicgstab"]["true_rel"] < 1e-9 and r["bicgstab"]["true_rel"] < 1e-9
