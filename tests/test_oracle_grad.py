"""Pins of the oracle's gradients and log-likelihood.

* state-vector adjoint vs central finite differences (both objectives);
* noisy-circuit adjoint (density matrices, Heisenberg picture) vs central
  finite differences (h = 1e-6), agreement to 1e-7 relative;
* log-likelihood vs an explicit loop over outcomes (0 log 0 = 0).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import gradient as GR
from oracle import noisy as NZ
from oracle import statevector as SV


def _param_circuit(n, count, seed):
    return W.random_gate_mix(n, count, seed, names1=["RX", "RY", "RZ", "U1", "U2", "U3", "H", "MAT1"],
                             names2=["CNOT", "CZ", "CP"])


@pytest.mark.parametrize("n", [1, 3, 5])
def test_sv_adjoint_vs_fd_weights(n):
    ops = _param_circuit(n, 30, 300 + n)
    w = W.rng(n).normal(size=1 << n)
    L, g = GR.grad_adjoint(ops, n, weights=w)
    fd = GR.grad_fd(ops, n, weights=w)
    np.testing.assert_allclose(g, fd, atol=1e-8)
    assert abs(L - GR.objective(SV.apply_circuit(SV.basis(n), n, ops), weights=w)) < 1e-13


@pytest.mark.parametrize("n", [2, 4])
def test_sv_adjoint_vs_fd_loglik(n):
    ops = _param_circuit(n, 24, 400 + n)
    p = SV.probabilities(SV.apply_circuit(SV.basis(n), n, ops))
    counts = W.multinomial_counts([p], 1000, seed=5)
    L, g = GR.grad_adjoint(ops, n, counts=counts)
    fd = GR.grad_fd(ops, n, counts=counts)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6)


def test_loglik_explicit_loop():
    p = np.array([0.5, 0.25, 0.0, 0.25])
    n = np.array([3, 0, 0, 7])
    ref = 0.0
    for J in range(4):
        if n[J] > 0:
            ref += n[J] * math.log(p[J])
    assert NZ.loglik(p, n) == pytest.approx(ref, rel=1e-15)


def test_noisy_adjoint_vs_fd():
    batch = W.noisy_batch(count=10, seed=4101, n_range=(1, 3), len_range=(1, 20))
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        p = NZ.circuit_probabilities(n, ops, params)
        counts = W.multinomial_counts([p], 1000, seed=c)
        L, p2, g = NZ.grad_adjoint(n, ops, params, counts)
        fd = NZ.grad_fd(n, ops, params, counts)
        np.testing.assert_allclose(p2, p, atol=1e-15)
        assert L == pytest.approx(NZ.loglik(p, counts), rel=1e-14)
        scale = np.maximum(np.abs(fd), 1.0)
        assert np.all(np.abs(g - fd) / scale < 1e-6), (c, g, fd)
