"""Pins of the readout oracle (measurement-error model, Bloch vectors) against
closed forms, the thesis's statements and a second method."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import density as D
from oracle import gates as G
from oracle import readout as RO
from oracle import statevector as SV


def _rand_p(n, seed):
    g = W.rng(seed)
    p = g.random(1 << n)
    return p / p.sum()


# ---------------------------------------------------------------- measurement error
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_meas_error_zero_rate_is_identity(n):
    p = _rand_p(n, 10 + n)
    np.testing.assert_allclose(RO.measurement_error(p, n, 0.0), p, atol=0, rtol=0)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_meas_error_half_rate_gives_uniform(n):
    p = _rand_p(n, 20 + n)
    np.testing.assert_allclose(RO.measurement_error(p, n, 0.5), np.full(1 << n, 1.0 / (1 << n)),
                               atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_meas_error_unit_rate_complements_every_bit(n):
    p = _rand_p(n, 30 + n)
    N = 1 << n
    out = RO.measurement_error(p, n, 1.0)
    np.testing.assert_allclose(out, p[(N - 1) ^ np.arange(N)], atol=0, rtol=0)


@pytest.mark.parametrize("n,eps", [(2, 0.08), (5, 0.08), (4, 0.3)])
def test_meas_error_basis_state_hamming_form(n, eps):
    # the thesis's form: a true string J0 is read as J with eps^D (1-eps)^(n-D)
    g = W.rng(40 + n)
    J0 = int(g.integers(0, 1 << n))
    p = np.zeros(1 << n)
    p[J0] = 1.0
    out = RO.measurement_error(p, n, eps)
    ref = [eps ** RO.hamming(J, J0) * (1 - eps) ** (n - RO.hamming(J, J0)) for J in range(1 << n)]
    np.testing.assert_allclose(out, ref, rtol=1e-14, atol=0)


def test_meas_error_asymmetric_rates_direction():
    # all-0 true string: each bit read as 1 with e01; all-1: each read as 0 with e10
    n, e01, e10 = 3, 0.1, 0.25
    for true, rate_flip in ((0, e01), ((1 << n) - 1, e10)):
        p = np.zeros(1 << n)
        p[true] = 1.0
        out = RO.measurement_error(p, n, e01, e10)
        for J in range(1 << n):
            k = RO.hamming(J, true)
            assert out[J] == pytest.approx(rate_flip ** k * (1 - rate_flip) ** (n - k), rel=1e-14)


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_meas_error_kron_equals_sum(n):
    g = W.rng(50 + n)
    p = _rand_p(n, 60 + n)
    e01 = g.uniform(0, 0.2, size=n)
    e10 = g.uniform(0, 0.2, size=n)
    a = RO.measurement_error(p, n, e01, e10)
    b = RO.measurement_error_kron(p, n, e01, e10)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-16)
    assert a.sum() == pytest.approx(1.0, abs=1e-13)
    assert np.all(a >= 0)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_meas_error_is_depolarizing_before_measurement(n):
    # the thesis: the model is a depolarizing channel right before the
    # measurement; with p_x = p_y = p_z = p/3 a Z outcome flips with p_x + p_y, so
    # eps = 2p/3 per qubit
    eps = 0.08
    g = W.rng(70 + n)
    psi = W.random_state(n, g)
    rho = D.pure(psi)
    p = D.probabilities(rho)
    kr = D.depolarizing_kraus(eps / 2, eps / 2, eps / 2)
    for q in range(n):
        rho = D.apply_kraus(rho, n, kr, [q])
    np.testing.assert_allclose(D.probabilities(rho), RO.measurement_error(p, n, eps), atol=1e-14)


# ---------------------------------------------------------------- Bloch vectors
def _single(theta, phi):
    # Eq. (singlequbitblochangles)
    return np.array([math.cos(theta / 2), np.exp(1j * phi) * math.sin(theta / 2)])


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_bloch_product_state_closed_form(n):
    g = W.rng(80 + n)
    th = g.uniform(0, math.pi, size=n)
    ph = g.uniform(0, 2 * math.pi, size=n)
    psi = np.array([1.0 + 0j])
    for q in range(n - 1, -1, -1):        # most significant bit = first tensor factor
        psi = np.kron(psi, _single(th[q], ph[q]))
    r = RO.bloch_vectors(psi, n)
    ref = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    np.testing.assert_allclose(r, ref, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-14)


def test_bloch_pauli_eigenstates():
    s = 1 / math.sqrt(2)
    cases = {(1, 0): (0, 0, 1), (0, 1): (0, 0, -1), (s, s): (1, 0, 0), (s, -s): (-1, 0, 0),
             (s, 1j * s): (0, 1, 0), (s, -1j * s): (0, -1, 0)}
    for amps, ref in cases.items():
        np.testing.assert_allclose(RO.bloch_vectors(np.array(amps, dtype=complex), 1)[0], ref,
                                   atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 6])
def test_bloch_entangled_states_are_centred(n):
    ghz = np.zeros(1 << n, dtype=complex)
    ghz[0] = ghz[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(RO.bloch_vectors(ghz, n), 0.0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_bloch_pair_sums_equal_expectation_values(n):
    psi = W.random_state(n, W.rng(90 + n))
    r = RO.bloch_vectors(psi, n)
    np.testing.assert_allclose(r, RO.bloch_vectors_expectation(psi, n), atol=1e-14)
    assert np.all(np.linalg.norm(r, axis=1) <= 1 + 1e-12)


def test_bloch_rotates_with_rz():
    # R^z(alpha) multiplies a0* a1 by e^{i alpha}: the (x, y) part turns by +alpha
    n, q, alpha = 3, 1, 0.7
    psi = W.random_state(n, W.rng(99))
    r0 = RO.bloch_vectors(psi, n)
    r1 = RO.bloch_vectors(SV.apply_matrix(psi, n, G.rz(alpha), [q]), n)
    c, s = math.cos(alpha), math.sin(alpha)
    np.testing.assert_allclose(r1[q], [c * r0[q, 0] - s * r0[q, 1], s * r0[q, 0] + c * r0[q, 1],
                                       r0[q, 2]], atol=1e-14)
    np.testing.assert_allclose(np.delete(r1, q, axis=0), np.delete(r0, q, axis=0), atol=1e-14)
