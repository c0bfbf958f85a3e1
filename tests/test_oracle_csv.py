"""Pins of the plain-C FP64 state-vector oracle and of the exact qubit permutation.

Each check is fixed by something other than the C code itself: closed forms
(GHZ amplitudes, the QFT of Eq. (multiqubitqft)), the brute-force product of
entry-by-entry embedded 2^n x 2^n matrices for n <= 6 (random non-symmetric
matrices and both qubit orders, so a transposed operand or a swapped index
fails), U.U^dagger returning |0...0>, and, for the permutation, basis states
relabelled bit by bit as strings and the gate table's SWAP matrix.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import cstate as C
from oracle import statevector as SV


def test_ghz_closed_form():
    for n in (3, 12):
        psi = C.apply_circuit(SV.basis(n), n, W.ghz_circuit(n))
        ref = np.zeros(1 << n, dtype=complex)
        ref[0] = ref[-1] = 1 / math.sqrt(2)
        assert np.max(np.abs(psi - ref)) < 1e-15


@pytest.mark.parametrize("n", [3, 10])
def test_qft_closed_form(n):
    J = W.random_basis_index(n, 2002 + n)
    psi = C.apply_circuit(SV.basis(n, J), n, W.qft_circuit(n))
    assert np.max(np.abs(psi - SV.qft_amplitudes(n, J))) < 1e-13


@pytest.mark.parametrize("n", [2, 4, 6])
def test_brute_force_full_unitary(n):
    g = W.rng(50 + n)
    ops = W.random_gate_mix(n, 60, seed=60 + n)
    # explicit non-symmetric matrices on both qubit orders
    for _ in range(6):
        a, b = (int(x) for x in g.choice(n, size=2, replace=False))
        z = g.normal(size=(4, 4)) + 1j * g.normal(size=(4, 4))
        ops.append(("MAT2", (a, b), (), z))
        ops.append(("MAT1", (a,), (), g.normal(size=(2, 2)) + 1j * g.normal(size=(2, 2))))
    psi0 = W.random_state(n, g)
    ref = SV.circuit_unitary(ops, n) @ psi0
    out = C.apply_circuit(psi0, n, ops)
    assert np.max(np.abs(out - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_circuit_then_inverse_returns_to_zero():
    n = 14
    ops = W.random_gate_mix(n, 200, seed=7, names1=["H", "X", "S", "T", "RX", "RY", "RZ", "U1", "U3",
                                                   "MAT1"])
    psi = C.apply_circuit(SV.basis(n), n, ops + W.inverse_circuit(ops))
    assert abs(psi[0] - 1) < 1e-12 and np.max(np.abs(psi[1:])) < 1e-12


def test_probabilities_and_norm():
    n = 12
    psi = C.apply_circuit(SV.basis(n), n, W.layered_haar_cz(n, 5, seed=3))
    p, s = C.probabilities(psi, n)
    assert abs(s - 1) < 1e-12
    assert np.max(np.abs(p - np.abs(psi) ** 2)) < 1e-15


def _permute_by_strings(n, dest, J):
    # bit string of J, most significant first; the character of bit b moves to bit dest[b]
    s = format(J, f"0{n}b")
    out = ["0"] * n
    for b in range(n):
        out[n - 1 - dest[b]] = s[n - 1 - b]
    return int("".join(out), 2)


def test_permute_qubits_moves_basis_states_bit_by_bit():
    n = 5
    g = W.rng(11)
    for _ in range(5):
        dest = [int(x) for x in g.permutation(n)]
        for J in range(1 << n):
            out = C.permute_qubits(SV.basis(n, J), n, dest)
            assert out[_permute_by_strings(n, dest, J)] == 1 and np.count_nonzero(out) == 1
        K = np.arange(1 << n)
        assert all(_permute_by_strings(n, dest, int(j)) == k
                   for j, k in zip(C.source_index(K, n, dest), K))


def test_swap_network_equals_gate_table_swaps_exactly():
    # the SWAP matrix of the gate table, applied by the numpy oracle, moves every
    # value unchanged: the same array, bit for bit
    n = 6
    g = W.rng(12)
    psi = W.random_state(n, g)
    swaps = [tuple(int(x) for x in g.choice(n, size=2, replace=False)) for _ in range(15)]
    ops = [("SWAP", s, (), None) for s in swaps]
    by_gates = SV.apply_circuit(psi.copy(), n, ops)
    by_index = C.permute_qubits(psi, n, C.swap_network_dest(n, swaps))
    assert np.array_equal(by_gates, by_index)
    # the QFT's final bit reversal
    rev = [(i, n - 1 - i) for i in range(n // 2)]
    assert C.swap_network_dest(n, rev) == list(range(n - 1, -1, -1))


def test_permutation_gates_equal_gate_table_exactly():
    # X, CNOT, SWAP from the gate table (numpy oracle, complex products with 0 and 1)
    # move every value unchanged; so does the index map, bit for bit
    n = 7
    g = W.rng(13)
    psi = W.random_state(n, g)
    ops = []
    for _ in range(60):
        k = int(g.integers(0, 3))
        if k == 0:
            ops.append(("X", (int(g.integers(0, n)),), (), None))
        else:
            a, b = (int(x) for x in g.choice(n, size=2, replace=False))
            ops.append(("CNOT" if k == 1 else "SWAP", (a, b), (), None))
    assert np.array_equal(SV.apply_circuit(psi.copy(), n, ops), C.permutation_gates(psi, n, ops))
    K = np.arange(1 << n)
    assert np.array_equal(C.permutation_gates(psi, n, ops)[K], psi[C.permutation_source(K, n, ops)])
    # a wrong control/target order is caught
    bad = [("CNOT", (1, 0), (), None)]
    assert not np.array_equal(SV.apply_circuit(psi.copy(), n, bad),
                              C.permutation_gates(psi, n, [("CNOT", (0, 1), (), None)]))
