"""State-vector parameter gradients, fp64.

Objective: a function of the outcome probabilities p_J = |a_J|^2 of the final
state, either

* ``weights`` w_J:  L = sum_J w_J p_J  (d L / d p_J = w_J), or
* ``counts`` n_J:  L = sum_J n_J log p_J (the multinomial log-likelihood).

Gradients with respect to every angle of every parameterised gate (RX, RY, RZ,
U1, CP: 1 angle; U2: 2; U3: 3), returned as an array [n_gates, 3] (unused
entries 0).  Two independent methods:

* :func:`grad_fd`: central differences of L, step h;
* :func:`grad_adjoint`: lambda = dL/d psi^* propagated backwards,
  dL/dtheta_g = 2 Re <lambda_g | dU_g/dtheta | psi_{g-1}>, states kept
  for every gate (small n only).
"""
from __future__ import annotations

import numpy as np

from . import gates as G
from .statevector import apply_circuit, apply_matrix, basis, probabilities


def objective(psi, weights=None, counts=None) -> float:
    p = probabilities(psi)
    if counts is not None:
        c = np.asarray(counts, dtype=np.float64)
        m = c > 0
        return float(np.sum(c[m] * np.log(p[m])))
    return float(np.dot(weights, p))


def _seed(psi, weights=None, counts=None):
    """lambda = dL/d psi^* = (dL/dp_J) psi_J."""
    p = probabilities(psi)
    if counts is not None:
        c = np.asarray(counts, dtype=np.float64)
        w = np.where(c > 0, c / np.where(p > 0, p, 1.0), 0.0)
    else:
        w = np.asarray(weights, dtype=np.float64)
    return w * psi


def grad_fd(ops, n, psi0=None, weights=None, counts=None, h=1e-6) -> np.ndarray:
    psi0 = basis(n) if psi0 is None else psi0
    g = np.zeros((len(ops), 3))
    for i, (name, qs, ps, m) in enumerate(ops):
        for k in range(G.N_PARAMS.get(name, 0)):
            for sgn in (+1, -1):
                pp = list(ps)
                pp[k] += sgn * h
                o2 = list(ops)
                o2[i] = (name, qs, tuple(pp), m)
                g[i, k] += sgn * objective(apply_circuit(psi0.copy(), n, o2), weights, counts)
            g[i, k] /= 2 * h
    return g


def grad_adjoint(ops, n, psi0=None, weights=None, counts=None):
    """(L, gradient) by the adjoint sweep; keeps every intermediate state."""
    psi = basis(n) if psi0 is None else psi0.copy()
    states = [psi]
    for op in ops:
        psi = apply_matrix(psi, n, G.matrix(op[0], op[2], op[3]), op[1])
        states.append(psi)
    L = objective(psi, weights, counts)
    lam = _seed(psi, weights, counts)
    g = np.zeros((len(ops), 3))
    for i in range(len(ops) - 1, -1, -1):
        name, qs, ps, m = ops[i]
        for k in range(G.N_PARAMS.get(name, 0)):
            dpsi = apply_matrix(states[i], n, G.dmatrix(name, ps, k), qs)
            g[i, k] = 2.0 * float(np.real(np.vdot(lam, dpsi)))
        U = G.matrix(name, ps, m)
        lam = apply_matrix(lam, n, U.conj().T, qs)
    return L, g
