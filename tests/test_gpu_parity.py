"""Parity that index work must meet exactly, and full-state parity at larger sizes.

* Permutations (SWAP networks, the QFT's bit reversal, X / CNOT / SWAP mixes) move
  amplitudes without arithmetic that could round (SWAPs are relabelings restored
  by the remap kernel; X and CNOT are matrices of 0 and 1), so the library must
  reproduce the oracle's permutation bit for bit: ``np.array_equal``, both
  precisions, at 13, 17 and 20 qubits, and on sampled indices of a 30-qubit state.
* The 30-qubit benchmark family (layered Haar SU(2) + brickwork CZ) at 24 qubits,
  every amplitude against the FP64 C oracle, through the tile passes (complex64:
  relative L2 <= 1e-5; complex128: max |da| <= 1e-12) and the tensor-core blocks
  (BF16 and TF32 splits, relative L2 <= 1e-5).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cstate as C
from oracle import statevector as SV

pytestmark = pytest.mark.gpu


def _run(qs, n, prec, psi0, ops, method=0):
    st = qs.State(n, prec)
    qs.sv_copy_in(st, psi0)
    stats = qs.sv_apply_circuit(st, ops, method)
    out = qs.sv_copy_out(st)
    st.close()
    return out, stats


def _state(n, prec, seed):
    psi = W.random_state(n, W.rng(seed))
    return psi.astype(np.complex64 if prec == 0 else np.complex128)


def _random_swaps(n, count, seed):
    g = W.rng(seed)
    return [tuple(int(x) for x in g.choice(n, size=2, replace=False)) for _ in range(count)]


def _swap_cases(n):
    rev = [(i, n - 1 - i) for i in range(n // 2)]                   # the QFT's bit reversal
    chain = [(i, i + 1) for i in range(n - 1)] * 3                   # qubits cycled three times
    return {"random": _random_swaps(n, 40, 100 + n), "bit_reversal": rev, "chain": chain,
            "mixed": _random_swaps(n, 10, 200 + n) + rev + chain[: n - 1]}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [13, 17, 20])
def test_swap_networks_bit_exact(qs, n, prec):
    psi0 = _state(n, prec, 300 + n)
    for name, swaps in _swap_cases(n).items():
        ops = [("SWAP", s, (), None) for s in swaps]
        out, _ = _run(qs, n, prec, psi0, ops)
        ref = C.permute_qubits(psi0, n, C.swap_network_dest(n, swaps))
        assert np.array_equal(out, ref), name


def _perm_circuit(n, count, seed):
    g = W.rng(seed)
    ops = []
    for _ in range(count):
        k = int(g.integers(0, 3))
        if k == 0:
            ops.append(("X", (int(g.integers(0, n)),), (), None))
        else:
            a, b = (int(x) for x in g.choice(n, size=2, replace=False))
            ops.append(("CNOT" if k == 1 else "SWAP", (a, b), (), None))
    return ops


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [5, 13, 17, 20])
@pytest.mark.parametrize("method", [0, 1])
def test_permutation_circuits_bit_exact(qs, n, prec, method):
    # X / CNOT / SWAP mixes through the fused tile passes (method 0; the small-state
    # kernel for n = 5) and one launch per gate (method 1)
    psi0 = _state(n, prec, 400 + n)
    ops = _perm_circuit(n, 150, 500 + n)
    out, _ = _run(qs, n, prec, psi0, ops, method)
    assert np.array_equal(out, C.permutation_gates(psi0, n, ops))


@pytest.mark.parametrize("method", [2, 3])
def test_permutation_circuits_through_blocks(qs, method):
    # the tensor-core blocks apply a permutation as a 32x32 product in split
    # precision: within the block path's tolerance (exactness is not claimed)
    n = 17
    psi0 = _state(n, 0, 600)
    ops = _perm_circuit(n, 150, 601)
    out, _ = _run(qs, n, 0, psi0, ops, method)
    ref = C.permutation_gates(psi0, n, ops)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-6


def _structured_values(J):
    # exact complex64 values (12-bit numerators over 2^12) that differ between indices
    re = (((J * 2654435761) >> 7) & 4095) - 2048
    im = (((J * 40503) >> 3) & 4095) - 2048
    return re, im


def test_permutations_30_qubits_sampled_bit_exact(qs):
    n = 30
    N = 1 << n
    buf = torch.empty(N, dtype=torch.complex64, device="cuda")
    view = torch.view_as_real(buf)
    chunk = 1 << 26
    for c0 in range(0, N, chunk):
        J = torch.arange(c0, c0 + chunk, dtype=torch.int64, device="cuda")
        re, im = _structured_values(J)
        view[c0:c0 + chunk, 0] = re.to(torch.float32) / 4096
        view[c0:c0 + chunk, 1] = im.to(torch.float32) / 4096
    del J, re, im
    ops = ([("SWAP", (i, n - 1 - i), (), None) for i in range(n // 2)]
           + _perm_circuit(n, 60, 700))
    st = qs.State(n, 0)
    qs.sv_copy_in(st, buf)
    qs.sv_apply_circuit(st, ops, qs.METHOD_TILED)
    qs.sv_copy_out(st, buf)
    st.close()
    K = np.sort(W.rng(701).integers(0, N, size=1 << 16))
    K = np.concatenate([K, [0, 1, N - 2, N - 1]])
    got = torch.view_as_real(buf[torch.tensor(K, device="cuda")]).cpu().numpy()
    src = C.permutation_source(K, n, ops)
    re, im = _structured_values(src)
    assert np.array_equal(got[:, 0], (re / 4096).astype(np.float32))
    assert np.array_equal(got[:, 1], (im / 4096).astype(np.float32))
    del buf
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- 24 qubits, full state
N24 = 24


@pytest.fixture(scope="module")
def layered24():
    ops = W.layered_haar_cz(N24, 40, seed=2001 + N24)
    ref = C.apply_circuit(SV.basis(N24), N24, ops)
    return ops, ref


@pytest.mark.parametrize("method,prec", [(0, 0), (0, 1), (2, 0), (3, 0)])
def test_layered_24_qubits_full_state(qs, layered24, method, prec):
    ops, ref = layered24
    st = qs.State(N24, prec)
    stats = qs.sv_apply_circuit(st, ops, method)
    out = qs.sv_copy_out(st)
    st.close()
    if prec == 1:
        assert np.max(np.abs(out - ref)) <= 1e-12
    else:
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, err
    assert stats["passes"] >= 1
