"""GPU parity of the readout transforms (measurement-error model, Bloch vectors)
against the oracle, through the C ABI.

Tolerances.  The measurement-error map multiplies and adds non-negative terms
only, so each output keeps a relative error below about 2 n u (u = 6e-8 in
FP32, 1.1e-16 in FP64): rtol 3e-6 (FP32, n <= 20), 1e-13 (FP64).  Rates 0 and 1
make every 2x2 map a copy or a swap: bit-exact.  Bloch vectors are sums of 2^(n-1)
pair terms whose absolute values add up to at most 1: absolute 5e-6 (complex64,
FP32 sums within a tile, FP64 across tiles), 1e-12 (complex128).
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import readout as RO

pytestmark = pytest.mark.gpu


def _rand_p(n, seed):
    g = W.rng(seed)
    p = g.random(1 << n)
    return p / p.sum()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 5, 11, 12, 13, 16, 20])
def test_meas_error_matches_oracle(qs, n, fp64):
    g = W.rng(500 + n)
    p = _rand_p(n, 510 + n)
    e01 = g.uniform(0, 0.2, size=n)
    e10 = g.uniform(0, 0.2, size=n)
    dt = torch.float64 if fp64 else torch.float32
    dev = torch.tensor(p, dtype=dt, device="cuda")
    qs.meas_error(dev, e01, e10)
    got = dev.cpu().numpy()
    ref = RO.measurement_error_kron(p.astype(np.float64 if fp64 else np.float32), n, e01, e10)
    np.testing.assert_allclose(got, ref, rtol=1e-13 if fp64 else 3e-6, atol=0)


@pytest.mark.parametrize("n", [2, 5])
def test_meas_error_thesis_cases(qs, n):
    # the thesis applies eps = 0.08 to the bare (n = 2) and encoded (n = 5) distributions
    p = _rand_p(n, 520 + n)
    dev = torch.tensor(p, dtype=torch.float64, device="cuda")
    qs.meas_error(dev, 0.08)
    np.testing.assert_allclose(dev.cpu().numpy(), RO.measurement_error(p, n, 0.08), rtol=1e-14)


@pytest.mark.parametrize("n", [3, 12, 14])
def test_meas_error_rates_zero_and_one_are_exact(qs, n):
    p = _rand_p(n, 530 + n).astype(np.float32)
    dev = torch.tensor(p, device="cuda")
    qs.meas_error(dev, 0.0)
    assert np.array_equal(dev.cpu().numpy(), p)
    qs.meas_error(dev, 1.0)
    N = 1 << n
    assert np.array_equal(dev.cpu().numpy(), p[(N - 1) ^ np.arange(N)])


def test_meas_error_30_qubits_basis_state(qs):
    # full size: a true outcome J0 is read as J with prod_q P(j_q | j0_q)
    n = 30
    g = W.rng(540)
    J0 = int(g.integers(0, 1 << n))
    e01 = g.uniform(0.01, 0.1, size=n)
    e10 = g.uniform(0.01, 0.1, size=n)
    p = torch.zeros(1 << n, dtype=torch.float32, device="cuda")
    p[J0] = 1.0
    qs.meas_error(p, e01, e10)
    assert float(p.double().sum()) == pytest.approx(1.0, abs=1e-5)
    Js = np.concatenate([[J0, J0 ^ 1, J0 ^ (1 << 29), (1 << n) - 1 - J0],
                         g.integers(0, 1 << n, size=60)])
    got = p[torch.tensor(Js, device="cuda")].cpu().numpy()
    for J, v in zip(Js, got):
        ref = 1.0
        for q in range(n):
            t, r = (J0 >> q) & 1, (int(J) >> q) & 1
            P = RO.flip_matrix(e01[q], e10[q])
            ref *= P[r, t]
        assert v == pytest.approx(ref, rel=4e-6, abs=1e-30), (J, v, ref)


def test_meas_error_after_probabilities(qs):
    # sv_probs writes the distribution, the model transforms it in place
    n = 14
    ops = W.layered_haar_cz(n, 8, seed=550)
    st = qs.State(n, qs.QS_C128)
    qs.sv_apply_circuit(st, ops)
    p, _ = qs.sv_probs(st, fp64=True)
    amps = qs.sv_copy_out(st)
    st.close()
    qs.meas_error(p, 0.03)
    ref = RO.measurement_error_kron(np.abs(amps) ** 2, n, 0.03)
    np.testing.assert_allclose(p.cpu().numpy(), ref, rtol=1e-12, atol=1e-18)


def test_meas_error_invalid_arguments(qs):
    lib = qs.load()
    p = torch.zeros(16, dtype=torch.float32, device="cuda")
    rates = (ctypes.c_double * 4)(0.1, 0.1, 0.1, 0.1)
    bad = (ctypes.c_double * 4)(0.1, 1.5, 0.1, 0.1)
    nan = (ctypes.c_double * 4)(0.1, float("nan"), 0.1, 0.1)
    assert lib.qs_meas_error(None, 4, 0, rates, None, None) == qs.QS_EINVAL
    assert lib.qs_meas_error(p.data_ptr(), 0, 0, rates, None, None) == qs.QS_EINVAL
    assert lib.qs_meas_error(p.data_ptr(), 41, 0, rates, None, None) == qs.QS_EINVAL
    assert lib.qs_meas_error(p.data_ptr() + 4, 2, 0, rates, None, None) == qs.QS_EINVAL
    assert lib.qs_meas_error(p.data_ptr(), 4, 0, bad, None, None) == qs.QS_EINVAL
    assert lib.qs_meas_error(p.data_ptr(), 4, 0, nan, None, None) == qs.QS_EINVAL
    assert lib.qs_meas_error(p.data_ptr(), 4, 0, None, None, None) == qs.QS_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [1, 3, 11, 12, 13, 17, 20])
def test_bloch_matches_oracle(qs, n, prec):
    psi = W.random_state(n, W.rng(600 + n))
    if prec == 0:
        psi = psi.astype(np.complex64)
    st = qs.State(n, prec)
    qs.sv_copy_in(st, psi)
    r = qs.sv_bloch(st)
    st.close()
    np.testing.assert_allclose(r, RO.bloch_vectors(psi.astype(np.complex128), n),
                               atol=1e-12 if prec else 5e-6, rtol=0)


def test_bloch_30_qubits_product_and_ghz(qs):
    # full size: R^y(theta_q) then R^z(phi_q) on every qubit of |0..0> gives the
    # single-qubit form of Eq. (singlequbitblochvector) on each qubit
    n = 30
    g = W.rng(610)
    th = g.uniform(0, math.pi, size=n)
    ph = g.uniform(-math.pi, math.pi, size=n)
    ops = [("RY", (q,), (float(th[q]),), None) for q in range(n)]
    ops += [("RZ", (q,), (float(ph[q]),), None) for q in range(n)]
    st = qs.State(n, qs.QS_C64)
    qs.sv_apply_circuit(st, ops)
    r = qs.sv_bloch(st)
    ref = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    np.testing.assert_allclose(r, ref, atol=2e-5, rtol=0)
    qs.sv_set_basis(st, 0)
    qs.sv_apply_circuit(st, W.ghz_circuit(n))
    np.testing.assert_allclose(qs.sv_bloch(st), 0.0, atol=1e-6)
    st.close()
