"""Oracle for batches of small noisy circuits (the GST-shaped forward model).

Model of one circuit (readings of the thesis, each stated where used):

* initial state rho_0 = |0...0><0...0| and projective measurement
  E_J = |J><J| -- the ideal version of the GST preparation/measurement
  (Sec. "Gate set tomography", Eq. (GSTBornRule));
* ops X90(theta_x) = R^x(theta_x) and Y90(theta_y) = R^y(theta_y) on one qubit
  (Eqs. (singlequbitrotationx), (singlequbitrotationy)), CZ on a pair, and
  IDLE (identity on the whole register);
* after every op, on each qubit the op touches (IDLE: all qubits), the
  symmetric depolarizing channel with p_x = p_y = p_z = p/3
  (Eq. (singletDepolarizingChannel)) and then amplitude damping with
  decay parameter 1 and rate gamma (Eqs. (singletAmplitudeDampingChannel1-2))
  -- the channel placement of Fig. (singletcircuitwitherrorchannels) applied
  after every gate;
* p_J = Tr(E_J rho_L) and the multinomial log-likelihood
  l = sum_J n_J log p_J (terms with n_J = 0 contribute 0).

Everything is computed on 2^n x 2^n density matrices (no PTMs), fp64.
Gradients of l with respect to (theta_x, theta_y, p, gamma): central finite
differences, and an adjoint sweep in the Heisenberg picture
(lambda <- E^dagger(lambda) = sum_a M_a^dagger lambda M_a).
"""
from __future__ import annotations

import math

import numpy as np

from . import gates as G
from .density import (amplitude_damping_kraus, apply_kraus, apply_unitary, depolarizing_kraus,
                      probabilities)

OP_X90, OP_Y90, OP_CZ, OP_IDLE = 0, 1, 2, 3
N_GRAD = 4   # d/d(theta_x, theta_y, p, gamma)


def _elementary_maps(n: int, ops, params):
    """Flatten a circuit into elementary maps.

    Each map is (kind, qubits, operators, dparam) where kind is 'U' (unitary
    sandwich) or 'K' (Kraus sum), operators the matrices, and dparam the index
    of the parameter the map depends on (or -1).
    """
    tx, ty, p, gam = (float(x) for x in params)
    dep = depolarizing_kraus(p / 3, p / 3, p / 3)
    ad = amplitude_damping_kraus(1.0, gam)
    maps = []

    def channels(q):
        maps.append(("K", (q,), dep, 2))
        maps.append(("K", (q,), ad, 3))

    for code, a, b in ops:
        code, a, b = int(code), int(a), int(b)
        if code == OP_X90:
            maps.append(("U", (a,), [G.rx(tx)], 0))
            channels(a)
        elif code == OP_Y90:
            maps.append(("U", (a,), [G.ry(ty)], 1))
            channels(a)
        elif code == OP_CZ:
            maps.append(("U", (a, b), [G.CZ], -1))
            channels(a)
            channels(b)
        elif code == OP_IDLE:
            for q in range(n):
                channels(q)
        else:
            raise ValueError(f"bad op code {code}")
    return maps


def _dops(kind, dparam, params):
    """Derivatives of the map's operators with respect to its parameter."""
    tx, ty, p, gam = (float(x) for x in params)
    if dparam == 0:
        return [-0.5j * G.SX @ G.rx(tx)]
    if dparam == 1:
        return [-0.5j * G.SY @ G.ry(ty)]
    if dparam == 2:   # d/dp of sqrt(1-p) I, sqrt(p/3) sigma
        a = -0.5 / math.sqrt(1 - p)
        b = 0.5 / math.sqrt(3 * p)
        return [a * G.I2, b * G.SX, b * G.SY, b * G.SZ]
    if dparam == 3:   # d/dgamma of the four amplitude-damping operators (decay parameter 1)
        ds = -0.5 / math.sqrt(1 - gam)
        dg = 0.5 / math.sqrt(gam)
        return [np.array([[0, 0], [0, ds]], dtype=np.complex128),
                np.array([[0, dg], [0, 0]], dtype=np.complex128),
                np.zeros((2, 2), dtype=np.complex128),
                np.zeros((2, 2), dtype=np.complex128)]
    raise ValueError


def _sandwich(rho, n, A, B, qubits):
    """A rho B^dagger with A, B acting on `qubits` (A, B need not be equal)."""
    v = rho.reshape(-1)
    from .statevector import apply_matrix
    v = apply_matrix(v, 2 * n, A, [q + n for q in qubits])
    v = apply_matrix(v, 2 * n, B.conj(), list(qubits))
    return v.reshape(rho.shape)


def _apply(rho, n, m):
    kind, qubits, opsl, _ = m
    if kind == "U":
        return apply_unitary(rho, n, opsl[0], qubits)
    return apply_kraus(rho, n, opsl, qubits)


def _apply_adjoint(lam, n, m):
    """Heisenberg-picture adjoint E^dagger(lam) = sum_a M_a^dagger lam M_a."""
    kind, qubits, opsl, _ = m
    out = np.zeros_like(lam)
    for M in opsl:
        out += _sandwich(lam, n, M.conj().T, M.conj().T, qubits)
    return out


def final_density(n: int, ops, params) -> np.ndarray:
    N = 1 << n
    rho = np.zeros((N, N), dtype=np.complex128)
    rho[0, 0] = 1.0
    for m in _elementary_maps(n, ops, params):
        rho = _apply(rho, n, m)
    return rho


def circuit_probabilities(n: int, ops, params) -> np.ndarray:
    return probabilities(final_density(n, ops, params))


def loglik(probs: np.ndarray, counts: np.ndarray) -> float:
    """sum_J n_J log p_J with 0 log(.) = 0."""
    counts = np.asarray(counts, dtype=np.float64)
    m = counts > 0
    return float(np.sum(counts[m] * np.log(probs[m])))


def circuit_loglik(n, ops, params, counts) -> float:
    return loglik(circuit_probabilities(n, ops, params), counts)


def grad_fd(n, ops, params, counts, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of the log-likelihood, step h."""
    g = np.zeros(N_GRAD)
    for k in range(N_GRAD):
        pp = np.array(params, dtype=np.float64)
        pm = pp.copy()
        pp[k] += h
        pm[k] -= h
        g[k] = (circuit_loglik(n, ops, pp, counts) - circuit_loglik(n, ops, pm, counts)) / (2 * h)
    return g


def grad_adjoint(n, ops, params, counts) -> tuple[float, np.ndarray, np.ndarray]:
    """(loglik, probabilities, gradient) by an adjoint sweep on density matrices.

    Lambda_L = sum_J (n_J / p_J) |J><J|; going backwards each map contributes
    Tr(Lambda_k dE_k(rho_{k-1})) and Lambda_{k-1} = E_k^dagger(Lambda_k).
    """
    maps = _elementary_maps(n, ops, params)
    N = 1 << n
    rho = np.zeros((N, N), dtype=np.complex128)
    rho[0, 0] = 1.0
    states = [rho]
    for m in maps:
        rho = _apply(rho, n, m)
        states.append(rho)
    p = probabilities(rho)
    counts = np.asarray(counts, dtype=np.float64)
    w = np.where(counts > 0, counts / np.where(p > 0, p, 1.0), 0.0)
    lam = np.diag(w).astype(np.complex128)
    g = np.zeros(N_GRAD)
    for k in range(len(maps) - 1, -1, -1):
        kind, qubits, opsl, dparam = maps[k]
        if dparam >= 0:
            prev = states[k]
            dl = _dops(kind, dparam, params)
            drho = np.zeros_like(prev)
            for M, dM in zip(opsl, dl):
                drho += _sandwich(prev, n, dM, M, qubits) + _sandwich(prev, n, M, dM, qubits)
            g[dparam] += float(np.real(np.trace(lam @ drho)))
        lam = _apply_adjoint(lam, n, maps[k])
    return loglik(p, counts), p, g


def batch_forward(batch, idx=None):
    """Probabilities (concatenated), per-circuit log-likelihood for a NoisyBatch."""
    idx = range(batch.size) if idx is None else idx
    probs, ll = [], []
    for c in idx:
        n, ops, params = batch.circuit(c)
        p = circuit_probabilities(n, ops, params)
        probs.append(p)
        if batch.counts is not None:
            ll.append(loglik(p, batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]))
    return probs, np.array(ll)
