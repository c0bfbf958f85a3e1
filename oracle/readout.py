"""Readout transforms (test infrastructure only, like the rest of this package).

* :func:`measurement_error` -- the measurement-error model of Eq.
  (errordetectionMeasurementError): every bit of an outcome string is misread
  independently, so

      p_J -> sum_{J'} p_{J'} prod_q P_q(j_q | j'_q),

  with P_q(1 | 0) = e01[q] (a 0 counted as a 1) and P_q(0 | 1) = e10[q].  The
  thesis's model has e01[q] = e10[q] = eps for every qubit, where the product is
  eps^Delta(J,J') (1 - eps)^(n - Delta(J,J')), Delta the Hamming distance.  Written
  as that sum over J' (O(4^n); n <= 12).
* :func:`measurement_error_kron` -- the same map as one 2x2 matrix per qubit
  axis of the (2,)*n view of p (the product over bits above is a Kronecker
  product), for the sizes the sum cannot reach; pinned to the sum.
* :func:`bloch_vectors` -- r_q = (<sigma^x_q>, <sigma^y_q>, <sigma^z_q>) of Eq.
  (multiqubitblochvector) for every qubit q (bit position): sums over the
  amplitude pairs that differ only in bit q of 2 Re(a0* a1), 2 Im(a0* a1) and
  |a0|^2 - |a1|^2.
* :func:`bloch_vectors_expectation` -- the same as <psi| sigma^alpha_q |psi> with
  the full 2^n x 2^n embedded Pauli matrix (n <= 8), the definition on the left
  of Eq. (multiqubitblochvector).
"""
from __future__ import annotations

import numpy as np

from .statevector import embed

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),      # Eq. (paulimatrices)
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def _rates(n: int, e01, e10):
    e01 = np.broadcast_to(np.asarray(e01, dtype=np.float64), (n,))
    e10 = e01 if e10 is None else np.broadcast_to(np.asarray(e10, dtype=np.float64), (n,))
    return e01, e10


def flip_matrix(e01: float, e10: float) -> np.ndarray:
    """P[read, true] for one bit: column-stochastic."""
    return np.array([[1.0 - e01, e10], [e01, 1.0 - e10]])


def measurement_error(p: np.ndarray, n: int, e01, e10=None) -> np.ndarray:
    """Eq. (errordetectionMeasurementError) as the sum over true strings J'."""
    if n > 12:
        raise ValueError("the O(4^n) sum is for n <= 12")
    e01, e10 = _rates(n, e01, e10)
    N = 1 << n
    J = np.arange(N)[:, None]      # read string
    Jp = np.arange(N)[None, :]     # true string
    T = np.ones((N, N))
    for q in range(n):
        P = flip_matrix(e01[q], e10[q])
        T *= P[(J >> q) & 1, (Jp >> q) & 1]
    return T @ np.asarray(p, dtype=np.float64)


def measurement_error_kron(p: np.ndarray, n: int, e01, e10=None) -> np.ndarray:
    """The same map, one 2x2 matrix per axis of the (2,)*n view (axis a <-> bit n-1-a)."""
    e01, e10 = _rates(n, e01, e10)
    t = np.asarray(p, dtype=np.float64).reshape((2,) * n)
    for q in range(n):
        ax = n - 1 - q
        t = np.moveaxis(np.tensordot(flip_matrix(e01[q], e10[q]), t, axes=([1], [ax])), 0, ax)
    return t.reshape(-1)


def hamming(J: int, K: int) -> int:
    return bin(J ^ K).count("1")


def bloch_vectors(psi: np.ndarray, n: int) -> np.ndarray:
    """(n, 3) array: row q = (r^x, r^y, r^z) of qubit q by the pair sums of Eq.
    (multiqubitblochvector)."""
    psi = np.asarray(psi, dtype=np.complex128)
    J = np.arange(1 << n)
    r = np.zeros((n, 3))
    for q in range(n):
        J0 = J[((J >> q) & 1) == 0]
        a0, a1 = psi[J0], psi[J0 | (1 << q)]
        c = np.conj(a0) * a1
        r[q] = (2.0 * c.real.sum(), 2.0 * c.imag.sum(), (np.abs(a0) ** 2 - np.abs(a1) ** 2).sum())
    return r


def bloch_vectors_expectation(psi: np.ndarray, n: int) -> np.ndarray:
    """<psi| sigma^alpha_q |psi> with the embedded 2^n x 2^n Pauli matrix (n <= 8)."""
    if n > 8:
        raise ValueError("full matrices only for n <= 8")
    psi = np.asarray(psi, dtype=np.complex128)
    r = np.zeros((n, 3))
    for q in range(n):
        for a in range(3):
            r[q, a] = np.vdot(psi, embed(SIGMA[a], [q], n) @ psi).real
    return r
