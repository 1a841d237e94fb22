"""The C ABI on its own: a plain C program (tests/c_abi_example.c) compiled
against include/lbvh.h and linked with the library, with no Python in the
loop, builds, queries, checks against brute force and round-trips a
checkpoint."""
from __future__ import annotations

import os
import subprocess

import pytest

from paper_2402_00665_gb300 import _build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_program(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    so = _build.build()
    lib_dir = os.path.dirname(so)
    libname = os.path.basename(so)[3:-3]  # lib<name>.so
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = tmp_path / "c_abi_example"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", os.path.join(ROOT, "tests", "c_abi_example.c"),
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    "-L", lib_dir, "-l" + libname, "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-lm", "-Wl,-rpath," + lib_dir, "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", str(exe)],
                   check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    assert "c abi ok" in res.stdout
