"""Host tables of a fused-block pass (tile boxes, output staging swizzle, store
walk), checked on the CPU by tests/block_tables_check.cpp built against the
library: every element reaches the slot its consumer reads, and every staging
access pattern is free of shared-memory bank conflicts."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib_path():
    from paper_2008_13490_gb300 import _build
    return _build.build()


def test_block_pass_tables(lib_path, tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    libdir = os.path.dirname(lib_path)
    exe = tmp_path / "block_tables_check"
    subprocess.run(["g++", "-O1", "-std=c++17", os.path.join(ROOT, "tests", "block_tables_check.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "failures 0" in r.stdout
