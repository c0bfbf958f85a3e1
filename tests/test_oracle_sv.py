"""Pins of the state-vector oracle.

* tensordot gate application vs the entry-by-entry 2^n x 2^n products
  (two independent methods, every gate of the set, n <= 6);
* GHZ amplitudes, Bell / singlet states (Eqs. (bellstatephi), (bellstatepsi)
  and the singlet preparation CNOT_01 H_0 X_0 X_1 |00>);
* QFT of a basis state vs the closed form of Eq. (multiqubitqft);
* U U^dagger returns to |0...0>, norm preservation;
* the singlet measurement distribution of Eq. (singletProgramGatesResult) and
  its correlators (Eqs. (singletProgramExpectationCorrelation)-(...1)).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_tensordot_matches_full_unitary(n):
    ops = W.random_gate_mix(n, 40, seed=100 + n)
    U = SV.circuit_unitary(ops, n)
    g = W.rng(900 + n)
    psi0 = W.random_state(n, g)
    np.testing.assert_allclose(SV.apply_circuit(psi0.copy(), n, ops), U @ psi0, atol=1e-13)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(1 << n), atol=1e-12)


@pytest.mark.parametrize("n", [2, 5, 9, 13])
def test_ghz(n):
    psi = SV.apply_circuit(SV.basis(n), n, W.ghz_circuit(n))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15)


def test_bell_and_singlet_states():
    # thesis qubit 0 = bit 1
    phi = SV.apply_circuit(SV.basis(2), 2, [("H", (1,), (), None), ("CNOT", (1, 0), (), None)])
    np.testing.assert_allclose(phi, np.array([1, 0, 0, 1]) / math.sqrt(2), atol=1e-15)
    ops = [("X", (1,), (), None), ("X", (0,), (), None), ("H", (1,), (), None),
           ("CNOT", (1, 0), (), None)]
    psi = SV.apply_circuit(SV.basis(2), 2, ops)
    # |Psi^-> = (|01> - |10>)/sqrt 2
    np.testing.assert_allclose(psi, np.array([0, 1, -1, 0]) / math.sqrt(2), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_qft_closed_form(n):
    ops = W.qft_circuit(n)
    for J in sorted({0, 1, (1 << n) - 1, W.random_basis_index(n, 2002 + n)}):
        psi = SV.apply_circuit(SV.basis(n, J), n, ops)
        np.testing.assert_allclose(psi, SV.qft_amplitudes(n, J), atol=1e-13)


def test_u_udagger_returns_to_zero():
    n = 10
    ops = W.layered_haar_cz(n, 8, seed=2001)
    psi = SV.apply_circuit(SV.basis(n), n, ops + W.inverse_circuit(ops))
    np.testing.assert_allclose(psi, SV.basis(n), atol=1e-13)
    ops = W.random_gate_mix(n, 120, seed=11, names1=["H", "S", "T", "RX", "RY", "RZ", "U1", "U3",
                                                      "MAT1", "X", "PX", "MY"])
    psi = SV.apply_circuit(SV.basis(n), n, ops + W.inverse_circuit(ops))
    np.testing.assert_allclose(psi, SV.basis(n), atol=1e-13)


def test_norm_preserved():
    n = 12
    psi = SV.apply_circuit(SV.basis(n), n, W.layered_haar_cnot(n, 6, seed=1001))
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    assert abs(SV.probabilities(psi).sum() - 1) < 1e-13


@pytest.mark.parametrize("t0,t1", [(0.0, 0.0), (0.3, 1.9), (-2.0, 0.5), (math.pi / 2, 0.0)])
def test_singlet_distribution(t0, t1):
    psi = SV.apply_circuit(SV.basis(2), 2, W.singlet_circuit(t0, t1))
    p = SV.probabilities(psi)
    for J in range(4):
        j0, j1 = J >> 1, J & 1          # j0 = thesis qubit 0 = bit 1
        ref = (1 - (-1) ** (j0 + j1) * math.cos(t1 - t0)) / 4
        assert abs(p[J] - ref) < 1e-14
    E01 = sum((-1) ** (J >> 1) * (-1) ** (J & 1) * p[J] for J in range(4))
    E0 = sum((-1) ** (J >> 1) * p[J] for J in range(4))
    E1 = sum((-1) ** (J & 1) * p[J] for J in range(4))
    assert abs(E01 + math.cos(t1 - t0)) < 1e-14 and abs(E0) < 1e-14 and abs(E1) < 1e-14


def test_marginal_brute_force():
    n = 7
    g = W.rng(5)
    p = SV.probabilities(W.random_state(n, g))
    mask = 0b1010010
    m = SV.marginal(p, n, mask)
    bits = [1, 4, 6]
    ref = np.zeros(8)
    for J in range(1 << n):
        K = sum(((J >> b) & 1) << i for i, b in enumerate(bits))
        ref[K] += p[J]
    np.testing.assert_allclose(m, ref, atol=1e-15)


def test_metrics():
    g = W.rng(3)
    psi = W.random_state(4, g)
    assert abs(SV.overlap(psi, np.exp(0.7j) * psi) - 1) < 1e-14
    U = W.haar_su2(g)
    assert SV.matrix_distance(np.exp(-1.1j) * U, U) < 1e-28
    assert abs(SV.statistical_distance([1, 0], [0, 1]) - 1) < 1e-15
