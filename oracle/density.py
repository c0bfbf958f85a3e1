"""Density-matrix oracle: unitary maps, Kraus channels, Pauli transfer matrices.

rho is a 2^n x 2^n complex128 matrix in the same bit convention as the state
vector (row/column index J, bit 0 least significant).

* rho -> U rho U^dagger (Eq. (mixedstatesQuantumGate)),
* rho -> sum_a M_a rho M_a^dagger (Eqs. (krausrepresentation),
  (singletKrausOperatorEvolution)),
* depolarizing channel of Eq. (singletDepolarizingChannel), amplitude damping
  of Eqs. (singletAmplitudeDampingChannel1), (singletAmplitudeDampingChannel2),
* Pauli basis P (Eq. (paulibasis)): P_0 = I...I, P_1 = I...I sigma^x, ... so
  the LAST tensor factor is the least significant base-4 digit.  With the
  library's bit convention (thesis qubit i = bit n-1-i) base-4 digit b of the
  Pauli index belongs to bit b.  Digit values 0,1,2,3 = I, x, y, z.
* Pauli transfer matrix G_ij = Tr(P_i E(P_j)) / N (Eq. (paulitransfermatrix)),
* Pauli vector rho_i = Tr(P^_i rho), P^_i = P_i / sqrt(N)
  (Eq. (GSTVectorizedRho)); outcome probability p_J = <<E_J|G|rho>>
  (Eq. (GSTBornRuleVectorized)).

The density-matrix routines never use PTMs; PTMs are built from their
definition only to produce inputs and to cross-check.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

from . import gates as G
from .statevector import apply_matrix


# ---------------------------------------------------------------------------
# density matrices
# ---------------------------------------------------------------------------

def pure(psi: np.ndarray) -> np.ndarray:
    return np.outer(psi, psi.conj())


def apply_unitary(rho: np.ndarray, n: int, U: np.ndarray, qubits) -> np.ndarray:
    """rho -> (U on qubits) rho (U on qubits)^dagger.

    rho is viewed as a 2n-qubit vector vec(rho)[J_row * 2^n + J_col]: row bit b
    sits at position n+b, column bit b at position b; U acts on the row bits
    and U* on the column bits.
    """
    v = rho.reshape(-1)
    v = apply_matrix(v, 2 * n, U, [q + n for q in qubits])
    v = apply_matrix(v, 2 * n, U.conj(), list(qubits))
    return v.reshape(rho.shape)


def apply_kraus(rho: np.ndarray, n: int, kraus, qubits) -> np.ndarray:
    """rho -> sum_a M_a rho M_a^dagger with every M_a acting on `qubits`."""
    out = np.zeros_like(rho)
    for M in kraus:
        out += apply_unitary(rho, n, M, qubits)   # same sandwich, M need not be unitary
    return out


def probabilities(rho: np.ndarray) -> np.ndarray:
    """p_J = Tr(|J><J| rho) = rho_JJ (Eq. (GSTBornRule) with E_J = |J><J|)."""
    return np.real(np.diag(rho)).copy()


# ---------------------------------------------------------------------------
# channels
# ---------------------------------------------------------------------------

def depolarizing_kraus(px: float, py: float, pz: float):
    """Kraus operators of Eq. (singletDepolarizingChannel)."""
    return [math.sqrt(1 - px - py - pz) * G.I2, math.sqrt(px) * G.SX,
            math.sqrt(py) * G.SY, math.sqrt(pz) * G.SZ]


def amplitude_damping_kraus(p: float, gamma: float):
    """M_0..M_3 of Eqs. (singletAmplitudeDampingChannel1-2)."""
    s = math.sqrt(1 - gamma)
    g = math.sqrt(gamma)
    return [math.sqrt(p) * np.array([[1, 0], [0, s]], dtype=np.complex128),
            math.sqrt(p) * np.array([[0, g], [0, 0]], dtype=np.complex128),
            math.sqrt(1 - p) * np.array([[s, 0], [0, 1]], dtype=np.complex128),
            math.sqrt(1 - p) * np.array([[0, 0], [g, 0]], dtype=np.complex128)]


def kraus_sum(kraus) -> np.ndarray:
    """sum_a M_a^dagger M_a (= identity iff trace preserving)."""
    return sum(M.conj().T @ M for M in kraus)


# ---------------------------------------------------------------------------
# Pauli basis, PTMs, Pauli vectors
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def pauli(i: int, n: int) -> np.ndarray:
    """P_i of Eq. (paulibasis); digit b (base 4) of i acts on bit b."""
    M = np.ones((1, 1), dtype=np.complex128)
    # Kronecker order: the most significant bit (n-1) is the first factor
    for b in range(n - 1, -1, -1):
        d = (i >> (2 * b)) & 3
        M = np.kron(M, G.PAULI[d])
    return M


def ptm_of_map(apply_map, n: int) -> np.ndarray:
    """G_ij = Tr(P_i E(P_j)) / N for a linear map rho -> apply_map(rho) on n qubits."""
    N = 1 << n
    D = N * N
    Gm = np.zeros((D, D))
    for j in range(D):
        img = apply_map(pauli(j, n))
        for i in range(D):
            Gm[i, j] = np.real(np.trace(pauli(i, n) @ img)) / N
    return Gm


def ptm_unitary(U: np.ndarray) -> np.ndarray:
    n = int(round(math.log2(U.shape[0])))
    return ptm_of_map(lambda P: U @ P @ U.conj().T, n)


def ptm_kraus(kraus) -> np.ndarray:
    n = int(round(math.log2(kraus[0].shape[0])))
    return ptm_of_map(lambda P: sum(M @ P @ M.conj().T for M in kraus), n)


def pauli_vector(rho: np.ndarray, n: int) -> np.ndarray:
    """rho_i = Tr(P^_i rho) (Eq. (GSTVectorizedRho))."""
    N = 1 << n
    return np.array([np.real(np.trace(pauli(i, n) @ rho)) / math.sqrt(N) for i in range(N * N)])


def rho_from_pauli_vector(r: np.ndarray, n: int) -> np.ndarray:
    N = 1 << n
    return sum(r[i] * pauli(i, n) for i in range(N * N)) / math.sqrt(N)


def effect_vector(J: int, n: int) -> np.ndarray:
    """<<E_J| for the projective measurement E_J = |J><J| (Eq. (GSTVectorizedEJ))."""
    N = 1 << n
    E = np.zeros((N, N), dtype=np.complex128)
    E[J, J] = 1.0
    return pauli_vector(E, n)


def apply_ptm_digits(r: np.ndarray, n: int, Gm: np.ndarray, qubits) -> np.ndarray:
    """Pauli vector update by a k-qubit PTM on the base-4 digits of `qubits`
    (first qubit = most significant local digit)."""
    k = len(qubits)
    t = r.reshape((4,) * n)                         # axis a <-> digit n-1-a
    axes = [n - 1 - q for q in qubits]
    Gt = Gm.reshape((4,) * (2 * k))
    out = np.tensordot(Gt, t, axes=(list(range(k, 2 * k)), axes))
    out = np.moveaxis(out, list(range(k)), axes)
    return np.ascontiguousarray(out).reshape(-1)

