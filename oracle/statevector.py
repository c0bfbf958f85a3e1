"""State-vector oracle (complex128).

An n-qubit state is the vector of 2^n amplitudes a_J of Eq. (multiqubitstate).
Library convention: a qubit is named by its bit position b in J (b = 0 least
significant); the thesis's qubit i (i-th tensor factor, j_0 most significant)
is bit n-1-i.

Two independent ways to apply a circuit are provided:

* :func:`apply_circuit` -- each gate acts on its qubits' axes of the
  (2,)*n tensor view (the embedding R_i = I x ... x R x ... x I of Eq.
  (singlequbitrotationmultiplequbits)), one ``tensordot`` per gate;
* :func:`circuit_unitary` -- the product of the full 2^n x 2^n embedded gate
  matrices in reversed time order (Eq. (twoqubitqft) and the paragraph before
  it), each embedded matrix built entry by entry (:func:`embed`).
"""
from __future__ import annotations

import math

import numpy as np

from . import gates as G


def basis(n: int, J: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[J] = 1.0
    return psi


def apply_matrix(psi: np.ndarray, n: int, U: np.ndarray, qubits) -> np.ndarray:
    """psi <- (U on `qubits`) psi; qubits[0] is the most significant local bit."""
    k = len(qubits)
    if len(set(qubits)) != k or any(q < 0 or q >= n for q in qubits):
        raise ValueError("bad qubits")
    t = psi.reshape((2,) * n)                       # axis a <-> bit n-1-a
    axes = [n - 1 - q for q in qubits]
    Ut = U.reshape((2,) * (2 * k))                  # (out_0..out_k-1, in_0..in_k-1)
    out = np.tensordot(Ut, t, axes=(list(range(k, 2 * k)), axes))
    out = np.moveaxis(out, list(range(k)), axes)
    return np.ascontiguousarray(out).reshape(-1)


def apply_gate(psi: np.ndarray, n: int, op) -> np.ndarray:
    name, qubits, params, mat = op
    return apply_matrix(psi, n, G.matrix(name, params, mat), qubits)


def apply_circuit(psi: np.ndarray, n: int, ops) -> np.ndarray:
    """Gates in time order (left to right in a circuit diagram)."""
    for op in ops:
        psi = apply_gate(psi, n, op)
    return psi


def probabilities(psi: np.ndarray) -> np.ndarray:
    """Born rule p_J = |a_J|^2."""
    return psi.real ** 2 + psi.imag ** 2


def marginal(p: np.ndarray, n: int, mask: int) -> np.ndarray:
    """Marginal distribution over the bits in `mask` (output index packs those
    bits in increasing bit order)."""
    bits = [b for b in range(n) if (mask >> b) & 1]
    out = np.zeros(1 << len(bits))
    J = np.arange(1 << n)
    K = np.zeros_like(J)
    for i, b in enumerate(bits):
        K |= ((J >> b) & 1) << i
    np.add.at(out, K, p)
    return out


def embed(U: np.ndarray, qubits, n: int) -> np.ndarray:
    """Full 2^n x 2^n matrix of U acting on `qubits`, entry by entry.

    E[J', J] = U[loc(J'), loc(J)] when J' and J agree on every other bit.
    """
    k = len(qubits)
    N = 1 << n
    E = np.zeros((N, N), dtype=np.complex128)
    others = [b for b in range(n) if b not in qubits]
    for rest in range(1 << len(others)):
        base = 0
        for i, b in enumerate(others):
            if (rest >> i) & 1:
                base |= 1 << b
        idx = []
        for loc in range(1 << k):
            J = base
            for i, q in enumerate(qubits):
                if (loc >> (k - 1 - i)) & 1:
                    J |= 1 << q
            idx.append(J)
        for lo in range(1 << k):
            for li in range(1 << k):
                E[idx[lo], idx[li]] = U[lo, li]
    return E


def circuit_unitary(ops, n: int) -> np.ndarray:
    """U = U_L ... U_2 U_1 for gates applied in time order (n <= 8)."""
    if n > 8:
        raise ValueError("full unitary only for n <= 8")
    U = np.eye(1 << n, dtype=np.complex128)
    for name, qubits, params, mat in ops:
        U = embed(G.matrix(name, params, mat), qubits, n) @ U
    return U


def qft_amplitudes(n: int, J: int, K=None) -> np.ndarray:
    """Closed form of Eq. (multiqubitqft): <K|QFT|J> = 2^{-n/2} e^{2 pi i J K / 2^n}.

    J*K is reduced modulo 2^n in exact integer arithmetic before the angle is
    formed.
    """
    N = 1 << n
    if K is None:
        K = np.arange(N, dtype=np.int64)
    K = np.asarray(K, dtype=np.int64)
    # (J*K) mod N with Python integers (exact for any n <= 62)
    jk = np.array([(int(J) * int(k)) % N for k in K.reshape(-1)], dtype=np.float64).reshape(K.shape)
    return np.exp(2j * math.pi * jk / N) / math.sqrt(N)


def overlap(psi: np.ndarray, phi: np.ndarray) -> float:
    """Global-phase-free overlap of Eq. (overlapPsitau1Psitau2)."""
    num = abs(np.vdot(psi, phi)) ** 2
    return float(num / (np.vdot(psi, psi).real * np.vdot(phi, phi).real))


def statistical_distance(p: np.ndarray, q: np.ndarray) -> float:
    """Total variation distance of Eq. (statisticaldistance)."""
    return 0.5 * float(np.abs(np.asarray(p) - np.asarray(q)).sum())


def matrix_distance(M: np.ndarray, U: np.ndarray) -> float:
    """min_z ||M - z U||_F^2 over complex phases z (Eq. (matrixdistanceobjective))."""
    t = np.vdot(U, M)               # Tr U^dagger M
    z = t / abs(t) if abs(t) > 0 else 1.0
    return float(np.linalg.norm(M - z * U) ** 2)
