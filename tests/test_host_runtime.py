"""Host runtime without a GPU: exceptions stop at the C ABI as status codes, and the
planners' parallel loop runs every item once, passes an item's exception to the
caller and honours QS_HOST_THREADS (tests/host_runtime_check.cpp)."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def check_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2008_13490_gb300 import _build
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path_factory.mktemp("hostrt") / "host_runtime_check"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["g++", "-O1", "-std=c++17", "-pthread", os.path.join(ROOT, "tests", "host_runtime_check.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_guard_and_parallel_loop(check_exe, threads):
    env = dict(os.environ, QS_HOST_THREADS=str(threads))
    r = subprocess.run([str(check_exe), str(threads)], env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
