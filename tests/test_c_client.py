"""The C ABI from plain C: tests/c_abi_client.c compiles against
include/hba.h and links the library (CPU), and runs the first worked example
on the GPU with exit status 0."""
from __future__ import annotations

import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_client.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp_path):
    from paper_2405_07079_gb300.build import BUILD, build_library

    build_library()
    exe = str(tmp_path / "c_abi_client")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), SRC, "-o", exe,
           "-L", BUILD, "-lhba", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{BUILD}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    subprocess.check_call(cmd)
    return exe


def test_c_client_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_client_runs_worked_example(tmp_path, gpu_lib):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c client: ok" in r.stdout
