"""Pins of the GST-prediction oracle (Eq. (GSTPrediction)) against closed forms:
the thesis's four preparations with ideal gates, the period of repeated X90,
the depolarizing decay, power = series, and the statistical distance."""
import math

import numpy as np
import pytest

from oracle import density as D
from oracle import gates as G
from oracle import gst as GS

I2 = np.eye(2)


def ideal_table():
    """PTMs of the thesis's GST gates on 2 qubits (qubit 0 = first tensor factor):
    XI, YI, IX, IY, II, CNOT (X90 = R^x(pi/2), Y90 = R^y(pi/2))."""
    x90, y90 = G.rx(math.pi / 2), G.ry(math.pi / 2)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    Us = [np.kron(x90, I2), np.kron(y90, I2), np.kron(I2, x90), np.kron(I2, y90), np.eye(4), cnot]
    return [D.ptm_unitary(U) for U in Us]


XI, YI, IX, IY, II, CNOT = range(6)
PREPS = {"00": [], "10": [XI, XI], "++": [IY, YI], "psi-": [IX, IX, XI, XI, YI, CNOT]}


def rho00():
    rho = np.zeros((4, 4), dtype=complex)
    rho[0, 0] = 1
    return D.pauli_vector(rho, 2)


def effects(n):
    return np.array([D.effect_vector(J, n) for J in range(1 << n)])


@pytest.mark.parametrize("name,ref", [("00", [1, 0, 0, 0]), ("10", [0, 0, 1, 0]),
                                      ("++", [0.25] * 4), ("psi-", [0, 0.5, 0.5, 0])])
def test_thesis_preparations(name, ref):
    # J = 2 j0 + j1 (qubit 0 the most significant): the thesis's |00>, |10>, |++>, |Psi^->
    T = ideal_table()
    p = effects(2) @ GS.prepared(T, rho00(), PREPS[name])
    np.testing.assert_allclose(p, ref, atol=1e-14)


def test_repeated_x90_period():
    # X90 on qubit 0 from |00>: p(10) = sin^2(pi r / 4), p(00) = cos^2(pi r / 4)
    T = ideal_table()
    s = GS.series(T, rho00(), effects(2), XI, [], 12)
    r = np.arange(1, 13)
    np.testing.assert_allclose(s[:, 2], np.sin(math.pi * r / 4) ** 2, atol=1e-13)
    np.testing.assert_allclose(s[:, 0], np.cos(math.pi * r / 4) ** 2, atol=1e-13)
    np.testing.assert_allclose(s[:, [1, 3]], 0, atol=1e-13)


def test_cnot_period_two():
    T = ideal_table()
    s = GS.series(T, rho00(), effects(2), CNOT, [XI, XI], 6)   # |10> <-> |11>
    np.testing.assert_allclose(s[0::2], [[0, 0, 0, 1]] * 3, atol=1e-14)
    np.testing.assert_allclose(s[1::2], [[0, 0, 1, 0]] * 3, atol=1e-14)


@pytest.mark.parametrize("p", [0.01, 0.2])
def test_depolarizing_decay(p):
    # Eq. (singletDepolarizingChannel) with p_x = p_y = p_z = p/3 shrinks the Bloch
    # vector by 1 - 4p/3: p_0(r) = 1/2 + (1 - 4p/3)^r / 2 from |0>
    Gd = D.ptm_kraus(D.depolarizing_kraus(p / 3, p / 3, p / 3))
    rho = D.pauli_vector(np.array([[1, 0], [0, 0]], dtype=complex), 1)
    s = GS.series([Gd], rho, effects(1), 0, [], 300)
    r = np.arange(1, 301)
    np.testing.assert_allclose(s[:, 0], 0.5 + 0.5 * (1 - 4 * p / 3) ** r, atol=1e-13)


def test_power_equals_series():
    # noisy gates: the same one-qubit depolarizing channel on both qubits after each gate
    # (the PTM of a product channel is the Kronecker product of the PTMs)
    Gd = D.ptm_kraus(D.depolarizing_kraus(0.01, 0.02, 0.005))
    T = [np.kron(Gd, Gd) @ Tg for Tg in ideal_table()]
    E = effects(2)
    for gate, prep in ((XI, PREPS["psi-"]), (CNOT, PREPS["++"]), (IY, [])):
        s = GS.series(T, rho00(), E, gate, prep, 1000)
        for r in (1, 7, 100, 1000):
            np.testing.assert_allclose(GS.power(T, rho00(), E, gate, prep, r), s[r - 1], atol=1e-12)


def test_statistical_distance():
    p = np.array([0.1, 0.2, 0.3, 0.4])
    assert GS.statistical_distance(p, p) == 0.0
    assert GS.statistical_distance([1, 0, 0, 0], [0, 0, 0.5, 0.5]) == pytest.approx(1.0)
    assert GS.statistical_distance([0.5, 0.5], [0.25, 0.75]) == pytest.approx(0.25)
