"""Pins of the density-matrix / PTM oracle.

* Kraus completeness of the depolarizing and amplitude-damping channels
  (trace preservation criterion under Eq. (krausrepresentation));
* PTM structure (section "Quantum operations"): first row (1,0,..,0) iff
  trace preserving, unital iff first column (1,0,..,0)^T, Clifford gates are
  signed permutations, composition = matrix product;
* the symmetric depolarizing channel of Eq. (singletDepolarizingChannel)
  equals the mixture form of Eq.
  (singletDepolarizingChannelSymmetricMixture) with F = 1 - 4p/3;
* pure states under unitaries reproduce the state-vector oracle;
* Pauli-vector propagation with PTMs (Eq. (GSTBornRuleVectorized)) equals the
  density-matrix (Kraus) propagation on noisy circuits;
* amplitude damping's closed-form action on the Bloch vector.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import density as D
from oracle import gates as G
from oracle import noisy as NZ
from oracle import statevector as SV


@pytest.mark.parametrize("p", [0.0, 1e-3, 0.05, 0.3])
def test_depolarizing_kraus_complete_and_mixture_form(p):
    K = D.depolarizing_kraus(p / 3, p / 3, p / 3)
    np.testing.assert_allclose(D.kraus_sum(K), np.eye(2), atol=1e-15)
    F = 1 - 4 * p / 3
    mix = D.ptm_of_map(lambda P: F * P + (1 - F) * np.trace(P) * np.eye(2) / 2, 1)
    np.testing.assert_allclose(D.ptm_kraus(K), mix, atol=1e-15)


@pytest.mark.parametrize("pa,gamma", [(1.0, 0.01), (1.0, 0.4), (0.7, 0.2), (0.0, 0.3)])
def test_amplitude_damping(pa, gamma):
    K = D.amplitude_damping_kraus(pa, gamma)
    np.testing.assert_allclose(D.kraus_sum(K), np.eye(2), atol=1e-15)
    Gm = D.ptm_kraus(K)
    np.testing.assert_allclose(Gm[0], [1, 0, 0, 0], atol=1e-15)          # TP
    # Bloch vector: x,y scale by sqrt(1-gamma); z -> (1-gamma) z + gamma (2 pa - 1)
    s = math.sqrt(1 - gamma)
    np.testing.assert_allclose(Gm[1:, 1:], np.diag([s, s, 1 - gamma]), atol=1e-15)
    np.testing.assert_allclose(Gm[1:, 0], [0, 0, gamma * (2 * pa - 1)], atol=1e-15)
    # fixed point of pure decay is |0><0|
    if pa == 1.0:
        rho = np.array([[0.3, 0.2 + 0.1j], [0.2 - 0.1j, 0.7]])
        # coherences decay as (1-gamma)^(k/2): iterate until below 1e-14
        for _ in range(int(2 * math.log(1e-14) / math.log(1 - gamma)) + 1):
            rho = D.apply_kraus(rho, 1, K, (0,))
        np.testing.assert_allclose(rho, np.diag([1, 0]), atol=1e-12)


def _is_signed_perm(M):
    A = np.abs(np.round(M, 12))
    return (np.all((A == 0) | (A == 1)) and np.all(A.sum(0) == 1) and np.all(A.sum(1) == 1))


def test_ptm_structure():
    for name in ("X", "Y", "Z", "H", "S", "PX", "MY"):
        Gm = D.ptm_unitary(G.matrix(name))
        assert _is_signed_perm(Gm), name
        assert Gm[0, 0] == pytest.approx(1) and np.allclose(Gm[0, 1:], 0) and np.allclose(Gm[1:, 0], 0)
    for name in ("CNOT", "CZ", "SWAP"):
        assert _is_signed_perm(D.ptm_unitary(G.matrix(name))), name
    assert not _is_signed_perm(D.ptm_unitary(G.rx(0.3)))
    assert not _is_signed_perm(D.ptm_unitary(G.matrix("T")))
    # depolarizing is unital, amplitude damping (gamma > 0) is not
    dep = D.ptm_kraus(D.depolarizing_kraus(0.01, 0.01, 0.01))
    ad = D.ptm_kraus(D.amplitude_damping_kraus(1.0, 0.05))
    assert np.allclose(dep[:, 0], [1, 0, 0, 0]) and not np.allclose(ad[:, 0], [1, 0, 0, 0])
    # a trace-decreasing map (leakage-like projection) breaks the first-row rule
    proj = D.ptm_kraus([np.diag([1.0, 0.9]).astype(complex)])
    assert not np.allclose(proj[0], [1, 0, 0, 0])


def test_ptm_composition_is_product():
    U = W.haar_su2(W.rng(1))
    K = D.amplitude_damping_kraus(0.8, 0.2)
    comp = D.ptm_of_map(lambda P: sum(M @ (U @ P @ U.conj().T) @ M.conj().T for M in K), 1)
    np.testing.assert_allclose(comp, D.ptm_kraus(K) @ D.ptm_unitary(U), atol=1e-14)
    # two-qubit: CZ then Haar on one qubit
    U2 = np.kron(U, np.eye(2))
    comp2 = D.ptm_of_map(lambda P: (U2 @ G.CZ) @ P @ (U2 @ G.CZ).conj().T, 2)
    np.testing.assert_allclose(comp2, D.ptm_unitary(U2) @ D.ptm_unitary(G.CZ), atol=1e-14)


def test_rotation_ptms_rotate_bloch_vector():
    # right-hand rule (section "Elementary quantum gates"): R^x rotates y -> z
    t = 0.37
    c, s = math.cos(t), math.sin(t)
    np.testing.assert_allclose(D.ptm_unitary(G.rx(t))[1:, 1:], [[1, 0, 0], [0, c, -s], [0, s, c]],
                               atol=1e-15)
    np.testing.assert_allclose(D.ptm_unitary(G.ry(t))[1:, 1:], [[c, 0, s], [0, 1, 0], [-s, 0, c]],
                               atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_pure_state_dm_matches_sv(n):
    ops = W.random_gate_mix(n, 25, seed=40 + n)
    psi = SV.apply_circuit(SV.basis(n), n, ops)
    rho = D.pure(SV.basis(n))
    for name, qs, ps, m in ops:
        rho = D.apply_unitary(rho, n, G.matrix(name, ps, m), qs)
    np.testing.assert_allclose(rho, D.pure(psi), atol=1e-13)
    np.testing.assert_allclose(D.probabilities(rho), SV.probabilities(psi), atol=1e-14)


@pytest.mark.parametrize("n", [1, 2])
def test_pauli_vector_round_trip_and_born_rule(n):
    g = W.rng(9)
    psi = W.random_state(n, g)
    rho = D.pure(psi)
    r = D.pauli_vector(rho, n)
    np.testing.assert_allclose(D.rho_from_pauli_vector(r, n), rho, atol=1e-14)
    for J in range(1 << n):
        assert abs(D.effect_vector(J, n) @ r - rho[J, J].real) < 1e-14


def test_noisy_dm_matches_ptm_propagation():
    batch = W.noisy_batch(count=24, seed=77, n_range=(1, 3), len_range=(1, 30),
                          p_range=(0.01, 0.1), gamma_range=(0.01, 0.1))
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        tx, ty, p, gam = params
        C = D.ptm_kraus(D.amplitude_damping_kraus(1.0, gam)) @ D.ptm_kraus(
            D.depolarizing_kraus(p / 3, p / 3, p / 3))
        GX = C @ D.ptm_unitary(G.rx(tx))
        GY = C @ D.ptm_unitary(G.ry(ty))
        GCZ = D.ptm_unitary(G.CZ)
        rho0 = np.zeros((1 << n, 1 << n))
        rho0[0, 0] = 1
        r = D.pauli_vector(rho0, n)
        for code, a, b in ops:
            if code == NZ.OP_X90:
                r = D.apply_ptm_digits(r, n, GX, (a,))
            elif code == NZ.OP_Y90:
                r = D.apply_ptm_digits(r, n, GY, (a,))
            elif code == NZ.OP_CZ:
                r = D.apply_ptm_digits(r, n, GCZ, (a, b))
                r = D.apply_ptm_digits(r, n, C, (a,))
                r = D.apply_ptm_digits(r, n, C, (b,))
            else:
                for q in range(n):
                    r = D.apply_ptm_digits(r, n, C, (q,))
        pv = np.array([D.effect_vector(J, n) @ r for J in range(1 << n)])
        pd = NZ.circuit_probabilities(n, ops, params)
        np.testing.assert_allclose(pv, pd, atol=1e-14)
        assert abs(pd.sum() - 1) < 1e-13 and np.all(pd > -1e-15)


def test_singlet_no_channels_via_dm():
    t0, t1 = 0.4, -1.3
    rho = D.pure(SV.basis(2))
    for name, qs, ps, m in W.singlet_circuit(t0, t1):
        rho = D.apply_unitary(rho, 2, G.matrix(name, ps, m), qs)
    p = D.probabilities(rho)
    for J in range(4):
        assert abs(p[J] - (1 - (-1) ** ((J >> 1) + (J & 1)) * math.cos(t1 - t0)) / 4) < 1e-14


def test_single_qubit_depolarizing_bloch_scaling():
    # one X90 then channels: the Bloch vector of R^x|0> scaled by 1-4p/3 before damping
    p = 0.03
    ops = np.array([[NZ.OP_X90, 0, -1]])
    rho = NZ.final_density(1, ops, (math.pi / 2, 0.0, p, 1e-12))
    r = D.pauli_vector(rho, 1) * math.sqrt(2)
    np.testing.assert_allclose(r[1:], [0, -(1 - 4 * p / 3), 0], atol=1e-9)
