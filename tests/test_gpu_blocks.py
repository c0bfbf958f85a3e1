"""Fused 5-qubit blocks on the tensor cores (tcgen05) vs the FP64 oracle.

Error budget (stated as numbers, relative L2 of the final state):
* TF32 split: each operand in two TF32 parts (~22 significant bits); three
  correction products; FP32 accumulation in tensor memory;
* BF16 split: each operand in three BF16 parts (~24 bits); five correction
  products;
* both: every block is unitary, so each 32-amplitude row keeps its norm; the
  epilogue rescales each output row to its input row's norm (this removes the
  magnitude the FP32 accumulation loses on every pass, which otherwise grows
  linearly: 1.3e-5 after 151 blocks without it).
Measured: 2e-7 .. 5e-7 for 8-13 blocks, 1.2e-6 (TF32) and 7.5e-7 (BF16) for the
151 blocks of a depth-60 20-qubit circuit.  Asserted: <= 2e-6 for <= 13 blocks
and <= 1e-5 (the FP32 bar) for 151 blocks.  The measured errors are printed
(pytest -s) for the record.
"""
import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV

pytestmark = pytest.mark.gpu

TOL = {2: 2e-6, 3: 2e-6}
TOL_DEEP = {2: 1e-5, 3: 1e-5}


def _run(qs, n, ops, method, psi0=None):
    st = qs.State(n, qs.QS_C64)
    if psi0 is not None:
        qs.sv_copy_in(st, psi0.astype(np.complex64))
    stats = qs.sv_apply_circuit(st, ops, method)
    out = qs.sv_copy_out(st)
    st.close()
    return out, stats


@pytest.mark.parametrize("method", [2, 3])
@pytest.mark.parametrize("n", [12, 13, 16])
def test_blocks_random_gate_mix(qs, n, method):
    ops = W.random_gate_mix(n, 120, seed=700 + n)
    psi0 = W.random_state(n, W.rng(n)).astype(np.complex64).astype(np.complex128)
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out, stats = _run(qs, n, ops, method, psi0)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    print(f"n={n} method={method} blocks={stats['passes']} rel_l2={err:.2e}")
    assert err <= TOL[method], err


# one dense block on chosen positions of an 18-qubit random state: the tile's five
# positions above bit 6 hold runs of every length (the tile loads as 2^(5-g)
# tensor boxes of 2^g runs), at bit 7, in the middle and at the top of the index
PLACEMENTS = [
    [0, 1, 2, 3, 4],          # tile = bits 0..11: one box of 32 runs
    [7, 8, 9, 10, 11],        # the same tile through block positions
    [13, 14, 15, 16, 17],     # box at the top of the index
    [0, 7, 14, 15, 17],       # runs {7,8} {14,15} {17}: four boxes
    [2, 9, 12, 15, 17],       # no two adjacent: sixteen boxes of 2 KiB
    [8, 10, 11, 12, 16],      # the run {10,11,12} with one position below it, one above
    [9, 10, 13, 14, 15],      # the run {13,14,15} above the run {9,10}
]


@pytest.mark.parametrize("method", [2, 3])
@pytest.mark.parametrize("q", PLACEMENTS, ids=lambda q: "-".join(map(str, q)))
def test_blocks_tile_boxes(qs, q, method):
    n = 18
    g = W.rng(1800 + sum(q))
    ops = []
    for layer in range(3):
        for b in q:
            ops.append(("MAT1", (b,), (), W.haar_su2(g)))
        for a in range(layer % 2, 4, 2):
            ops.append(("CZ", (q[a], q[a + 1]), (), None))
    psi0 = W.random_state(n, g).astype(np.complex64).astype(np.complex128)
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out, stats = _run(qs, n, ops, method, psi0)
    assert stats["passes"] == 1
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err <= TOL[method], err


@pytest.mark.parametrize("method", [2, 3])
def test_blocks_depth60_n20(qs, method):
    # the 32-qubit workload's circuit family at 20 qubits (seed 3002), checked in full
    n = 20
    ops = W.layered_haar_cz(n, 60, seed=3002)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, stats = _run(qs, n, ops, method)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    print(f"depth-60 n=20 method={method} blocks={stats['passes']} rel_l2={err:.2e}")
    assert err <= TOL_DEEP[method], err


def test_blocks_qft_closed_form(qs):
    n = 14
    J = W.random_basis_index(n, 77)
    st = qs.State(n, qs.QS_C64)
    qs.sv_set_basis(st, J)
    qs.sv_apply_circuit(st, W.qft_circuit(n), 2)
    out = qs.sv_copy_out(st)
    st.close()
    ref = SV.qft_amplitudes(n, J)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("method", [2, 3])
def test_blocks_non_unitary_matrix(qs, method):
    # a non-unitary MAT1 makes its block non-unitary: rows do not keep their
    # norm, so the epilogue must leave that block's rows unscaled
    n = 14
    ops = W.random_gate_mix(n, 40, seed=901)
    ops.insert(20, ("MAT1", (3,), (), np.array([[1.0, 0.3], [0.0, 0.8]], dtype=np.complex128)))
    psi0 = W.random_state(n, W.rng(n + 1)).astype(np.complex64).astype(np.complex128)
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out, stats = _run(qs, n, ops, method, psi0)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    print(f"non-unitary n={n} method={method} blocks={stats['passes']} rel_l2={err:.2e}")
    assert err <= TOL[method], err


def test_blocks_reject_unsupported(qs):
    st = qs.State(8, qs.QS_C64)
    with pytest.raises(qs.QsimError) as e:
        qs.sv_apply_circuit(st, [("H", (0,), (), None)], 2)
    assert e.value.status == qs.QS_EUNSUPPORTED
    st.close()


# ---------------------------------------------------------------- the default method
def test_auto_dense_circuit_uses_blocks(qs):
    # layered Haar + CZ: every block is dense, so the default equals the BF16 blocks
    n = 18
    ops = W.layered_haar_cz(n, 20, seed=77)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, st = _run(qs, n, ops, qs.METHOD_AUTO)
    outb, stb = _run(qs, n, ops, 3)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
    assert np.linalg.norm(out - outb) / np.linalg.norm(ref) <= 2e-6
    assert st["passes"] <= stb["passes"] + 2 and st["tile_launches"] <= 2


@pytest.mark.parametrize("n", [13, 17])
def test_auto_sparse_circuit_uses_tiles(qs, n):
    # the QFT's blocks are nearly diagonal (one or two Hadamards among phases):
    # tile passes only, as the tiled method
    J = W.random_basis_index(n, 2002 + n)
    ops = W.qft_circuit(n)
    st = qs.State(n, qs.QS_C64)
    qs.sv_set_basis(st, J)
    stats = qs.sv_apply_circuit(st, ops, qs.METHOD_AUTO)
    out = qs.sv_copy_out(st)
    st.close()
    ref = SV.qft_amplitudes(n, J)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
    assert stats["tile_launches"] >= 1 and stats["passes"] <= 8


def test_auto_mixed_circuit(qs):
    # dense layers, then a QFT, then dense layers again: both segment kinds in one
    # call, composed in the canonical layout; against the oracle
    n = 16
    g = W.rng(5)
    psi0 = W.random_state(n, g)
    ops = W.layered_haar_cz(n, 6, seed=1) + W.qft_circuit(n) + W.layered_haar_cz(n, 6, seed=2)
    ref = SV.apply_circuit(psi0.astype(np.complex64).astype(np.complex128), n, ops)
    out, stats = _run(qs, n, ops, qs.METHOD_AUTO, psi0=psi0)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
    assert stats["tile_launches"] >= 1 and stats["passes"] > stats["tile_launches"]
    # complex128 states take the tile path
    st = qs.State(n, qs.QS_C128)
    qs.sv_copy_in(st, psi0)
    s128 = qs.sv_apply_circuit(st, ops, qs.METHOD_AUTO)
    out128 = qs.sv_copy_out(st)
    st.close()
    assert np.max(np.abs(out128 - SV.apply_circuit(psi0, n, ops))) <= 1e-12
