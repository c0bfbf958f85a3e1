"""GST predictions for repeated gates (test infrastructure only).

Eq. (GSTPrediction): p_J = <<E_J| (G_s)^r G_(prep) |rho>>, with Pauli transfer
matrices G (Eq. (paulitransfermatrix)) acting on Pauli vectors |rho>>
(Eq. (GSTVectorizedRho)) and effects <<E_J| (Eq. (GSTVectorizedEJ)).

* :func:`series` -- p(r) for r = 1..r_max by applying G_s r times to
  G_(prep)|rho>> (the definition, one matrix-vector product per repetition);
* :func:`power` -- p at one r as <<E| (G_s^r) G_(prep)|rho>>, G_s^r formed by r - 1
  matrix products (r <= 4096) or numpy's matrix_power.

A preparation is the list of PTMs applied to |rho>> in time order (the first
listed acts first): the thesis's |Psi^-> preparation G_CNOT G_YI G_XI G_XI G_IX
G_IX |rho>> is [IX, IX, XI, XI, YI, CNOT].
"""
from __future__ import annotations

import numpy as np


def prepared(ptms, rho, prep) -> np.ndarray:
    v = np.asarray(rho, dtype=np.float64)
    for k in prep:
        v = ptms[k] @ v
    return v


def series(ptms, rho, effects, gate: int, prep, r_max: int) -> np.ndarray:
    """(r_max, 2^n): row r - 1 = <<E_J| G_s^r G_(prep) |rho>>."""
    v = prepared(ptms, rho, prep)
    G = np.asarray(ptms[gate], dtype=np.float64)
    E = np.asarray(effects, dtype=np.float64)
    out = np.empty((r_max, E.shape[0]))
    for r in range(r_max):
        v = G @ v
        out[r] = E @ v
    return out


def power(ptms, rho, effects, gate: int, prep, r: int) -> np.ndarray:
    G = np.asarray(ptms[gate], dtype=np.float64)
    if r <= 4096:
        M = np.eye(G.shape[0])
        for _ in range(r):
            M = G @ M
    else:
        M = np.linalg.matrix_power(G, r)
    return np.asarray(effects, dtype=np.float64) @ (M @ prepared(ptms, rho, prep))


def statistical_distance(p, q) -> float:
    """D = (1/2) sum_J |p_J - q_J| (Eq. (statisticaldistance))."""
    return 0.5 * float(np.sum(np.abs(np.asarray(p) - np.asarray(q))))
