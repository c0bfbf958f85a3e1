"""The host block planner on the CPU: the 5-qubit blocks it makes of a circuit,
applied in order to a random state (each block's 32x32 matrix on its qubits,
numpy), give the oracle's state; every block of a unitary circuit is reported
unitary.  Covers dense one- and two-qubit gates, diagonals (which the planner
applies by scaling rows), SWAPs, and layered and QFT circuits."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from conftest import ROOT
from oracle import statevector as SV


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2008_13490_gb300 import _build
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path_factory.mktemp("planner") / "block_plan_dump"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["g++", "-O1", "-std=c++17", os.path.join(ROOT, "tests", "block_plan_dump.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    return exe


def _blocks(exe, tmp_path, n, ops):
    import paper_2008_13490_gb300 as qs
    gin, bout = tmp_path / "g.bin", tmp_path / "b.bin"
    qs.gates_array(ops).tofile(gin)
    subprocess.run([str(exe), str(gin), str(n), str(bout)], check=True)
    raw = np.fromfile(bout, dtype=np.uint8)
    rec = 24 + 1024 * 16
    assert raw.size % rec == 0
    out = []
    for k in range(raw.size // rec):
        r = raw[k * rec:(k + 1) * rec]
        q = r[:20].view(np.int32).tolist()
        unitary = int(r[20:24].view(np.int32)[0])
        U = r[24:].view(np.complex128).reshape(32, 32)
        out.append((q, unitary, U))
    return out


def _apply_block(psi, n, q, U):
    # amplitude index bit b = qubit b; local index bit i = qubit q[i]
    t = psi.reshape([2] * n)                 # axis a <-> bit n-1-a
    axes = [n - 1 - q[i] for i in reversed(range(5))]   # local bit 4 first (most significant)
    t = np.moveaxis(t, axes, range(5)).reshape(32, -1)
    t = U @ t
    t = np.moveaxis(t.reshape([2] * n), range(5), axes)
    return t.reshape(-1)


@pytest.mark.parametrize("name", ["gate_mix", "diagonals", "layered", "qft"])
def test_blocks_reproduce_the_circuit(dump_exe, tmp_path, name):
    n = 10
    ops = {
        "gate_mix": lambda: W.random_gate_mix(n, 300, seed=91),
        "diagonals": lambda: W.random_gate_mix(n, 300, seed=92, two_q_fraction=0.6,
                                               names1=["RZ", "S", "T", "Z", "H", "U1"],
                                               names2=["CZ", "CP", "CNOT", "SWAP"]),
        "layered": lambda: W.layered_haar_cz(n, 12, seed=93),
        "qft": lambda: W.qft_circuit(n),
    }[name]()
    blocks = _blocks(dump_exe, tmp_path, n, ops)
    assert blocks
    psi0 = W.random_state(n, W.rng(94))
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    psi = psi0.copy()
    for q, unitary, U in blocks:
        assert sorted(q) == q and len(set(q)) == 5 and max(q) < n
        assert unitary == 1
        np.testing.assert_allclose(U.conj().T @ U, np.eye(32), atol=1e-12)
        psi = _apply_block(psi, n, q, U)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_block_plan_does_not_depend_on_host_threads(dump_exe, tmp_path):
    # the blocks' products run on host threads (QS_HOST_THREADS caps them): the plan of
    # the 30-qubit layered circuit (100 blocks) is byte for byte the same on one
    # thread as on eight
    import paper_2008_13490_gb300 as qs
    gin = tmp_path / "g.bin"
    qs.gates_array(W.layered_haar_cz(30, 40, seed=2001)).tofile(gin)
    outs = []
    for threads in ("1", "8"):
        bout = tmp_path / f"b{threads}.bin"
        env = dict(os.environ, QS_HOST_THREADS=threads)
        subprocess.run([str(dump_exe), str(gin), "30", str(bout)], check=True, env=env)
        outs.append(bout.read_bytes())
    assert len(outs[0]) == 100 * (24 + 1024 * 16)
    assert outs[0] == outs[1]


@pytest.mark.parametrize("case", range(8))
def test_random_circuits_blocks_reproduce_the_circuit(dump_exe, tmp_path, case):
    # seed sweep over widths 6..12 and gate mixes (dense, diagonal-heavy, permutations
    # and user matrices): the blocks applied in order give the oracle's state
    n = 6 + (case * 5) % 7
    mix = case % 3
    if mix == 0:
        ops = W.random_gate_mix(n, 250, seed=960 + case)
    elif mix == 1:
        ops = W.random_gate_mix(n, 250, seed=960 + case, two_q_fraction=0.7,
                                names1=["RZ", "T", "S", "H", "U3"], names2=["CP", "CZ", "CNOT"])
    else:
        ops = W.random_gate_mix(n, 200, seed=960 + case, two_q_fraction=0.5,
                                names2=["SWAP", "MAT2", "CNOT"])
    blocks = _blocks(dump_exe, tmp_path, n, ops)
    psi0 = W.random_state(n, W.rng(980 + case))
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    psi = psi0.copy()
    for q, unitary, U in blocks:
        assert sorted(q) == q and len(set(q)) == 5 and max(q) < n
        assert unitary == 1
        psi = _apply_block(psi, n, q, U)
    assert np.max(np.abs(psi - ref)) < 1e-12


@pytest.fixture(scope="module")
def auto_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2008_13490_gb300 import _build
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path_factory.mktemp("autoplan") / "auto_plan_check"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["g++", "-O1", "-std=c++17", os.path.join(ROOT, "tests", "auto_plan_check.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("name,n,expect", [
    ("qft", 30, 1),        # one dense block; the whole QFT takes the same 3 tile passes and 3 remaps
    ("qft", 13, 0),        # its whole-circuit plan would add a tile pass
    ("qft", 17, 0),
    ("layered", 30, 0),    # 93 dense blocks
    ("mixed", 16, 0),      # dense layers around a QFT: 14 dense blocks
    ("phases", 14, 0),     # no dense block at all
])
def test_default_method_runs_lone_dense_blocks_on_tiles_when_free(auto_exe, tmp_path, name, n, expect):
    import paper_2008_13490_gb300 as qs
    ops = {
        "qft": lambda: W.qft_circuit(n),
        "layered": lambda: W.layered_haar_cz(n, 40, seed=2001),
        "mixed": lambda: W.layered_haar_cz(n, 6, seed=1) + W.qft_circuit(n) + W.layered_haar_cz(n, 6, seed=2),
        "phases": lambda: W.random_gate_mix(n, 300, seed=3, two_q_fraction=0.9, names1=["RZ", "T"],
                                            names2=["CP", "CZ"]),
    }[name]()
    gin = tmp_path / "g.bin"
    qs.gates_array(ops).tofile(gin)
    r = subprocess.run([str(auto_exe), str(gin), str(n)], check=True, capture_output=True, text=True)
    tiles, dense = (int(x) for x in r.stdout.split())
    assert tiles == expect, (name, n, dense)
