"""Gate matrices of the thesis's gate model, complex128.

Conventions (the thesis's own, sections "Multiple qubits" and "Elementary
quantum gates"): a matrix acts as U[out][in]; for two-qubit gates the local
index is 2*j_first + j_second with the first listed qubit the most
significant (the CNOT matrix of Eq. (cnotgate) with the control first).
Explicit gate-table matrices are taken verbatim from the table of
elementary gates (Tab. (elementarygateset)), i.e. including its choice of
global phase.
"""
from __future__ import annotations

import math

import numpy as np

SQ2 = 1.0 / math.sqrt(2.0)

# Pauli matrices (Eq. (paulimatrices))
I2 = np.eye(2, dtype=np.complex128)
SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = (I2, SX, SY, SZ)


def rx(t: float) -> np.ndarray:
    """R^x(theta) = exp(-i theta sigma^x / 2), closed form of Eq. (singlequbitrotationx)."""
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(t: float) -> np.ndarray:
    """R^y(theta), closed form of Eq. (singlequbitrotationy)."""
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(t: float) -> np.ndarray:
    """R^z(theta), closed form of Eq. (singlequbitrotationz)."""
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)


def u1(lam: float) -> np.ndarray:
    """U1 as printed in Tab. (elementarygateset)."""
    return np.array([[1, 0], [0, np.exp(1j * lam)]], dtype=np.complex128)


def u2(phi: float, lam: float) -> np.ndarray:
    """U2 as printed in Tab. (elementarygateset)."""
    return SQ2 * np.array([[1, -np.exp(1j * lam)],
                           [np.exp(1j * phi), np.exp(1j * (phi + lam))]], dtype=np.complex128)


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    """U3 as printed in Tab. (elementarygateset)."""
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def rk(k: float) -> np.ndarray:
    """Phase gate R(k) = diag(1, exp(2 pi i / 2^k)) (Tab. (elementarygateset))."""
    return np.array([[1, 0], [0, np.exp(2j * math.pi / (2.0 ** k))]], dtype=np.complex128)


_FIXED_1Q = {
    "I": I2,
    "X": SX,
    "Y": SY,
    "Z": SZ,
    "H": SQ2 * np.array([[1, 1], [1, -1]], dtype=np.complex128),
    "S": np.array([[1, 0], [0, 1j]], dtype=np.complex128),
    "T": np.array([[1, 0], [0, np.exp(0.25j * math.pi)]], dtype=np.complex128),
    # +X, -X, +Y, -Y rows of the gate table
    "PX": SQ2 * np.array([[1, 1j], [1j, 1]], dtype=np.complex128),
    "MX": SQ2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128),
    "PY": SQ2 * np.array([[1, 1], [-1, 1]], dtype=np.complex128),
    "MY": SQ2 * np.array([[1, -1], [1, 1]], dtype=np.complex128),
}
_FIXED_1Q["SDG"] = _FIXED_1Q["S"].conj().T
_FIXED_1Q["TDG"] = _FIXED_1Q["T"].conj().T

# CNOT of Eq. (cnotgate) (control = first qubit = most significant local bit)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
# CZ = diag(1, 1, 1, -1) (Sec. "Encoded gates" of the [[4,2,2]] chapter)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def cp(lam: float) -> np.ndarray:
    """Controlled phase: the controlled version of U1(lam), diag(1, 1, 1, e^{i lam})."""
    return np.diag([1, 1, 1, np.exp(1j * lam)]).astype(np.complex128)


def matrix(name: str, params=(), mat=None) -> np.ndarray:
    """Matrix of a gate record (see the ``workloads`` module for the record format)."""
    if name in _FIXED_1Q:
        return _FIXED_1Q[name].copy()
    if name == "RX":
        return rx(params[0])
    if name == "RY":
        return ry(params[0])
    if name == "RZ":
        return rz(params[0])
    if name == "U1":
        return u1(params[0])
    if name == "U2":
        return u2(params[0], params[1])
    if name == "U3":
        return u3(params[0], params[1], params[2])
    if name == "RK":
        return rk(params[0])
    if name == "CNOT":
        return CNOT.copy()
    if name == "CZ":
        return CZ.copy()
    if name == "CP":
        return cp(params[0])
    if name == "SWAP":
        return SWAP.copy()
    if name in ("MAT1", "MAT2"):
        m = np.asarray(mat, dtype=np.complex128)
        d = 2 if name == "MAT1" else 4
        if m.shape != (d, d):
            raise ValueError(f"{name} needs a {d}x{d} matrix")
        return m.copy()
    raise ValueError(f"unknown gate {name}")


def dmatrix(name: str, params, k: int) -> np.ndarray:
    """Derivative of the gate matrix with respect to its k-th parameter.

    Differentiated from the closed forms above (rotations: d/dt exp(-i t s/2)
    = -i/2 s exp(-i t s/2)).
    """
    if name == "RX":
        return -0.5j * SX @ rx(params[0])
    if name == "RY":
        return -0.5j * SY @ ry(params[0])
    if name == "RZ":
        return -0.5j * SZ @ rz(params[0])
    if name == "U1":
        return np.array([[0, 0], [0, 1j * np.exp(1j * params[0])]], dtype=np.complex128)
    if name == "CP":
        return np.diag([0, 0, 0, 1j * np.exp(1j * params[0])]).astype(np.complex128)
    if name == "U2":
        phi, lam = params[0], params[1]
        if k == 0:
            return SQ2 * np.array([[0, 0], [1j * np.exp(1j * phi), 1j * np.exp(1j * (phi + lam))]])
        return SQ2 * np.array([[0, -1j * np.exp(1j * lam)], [0, 1j * np.exp(1j * (phi + lam))]])
    if name == "U3":
        th, phi, lam = params
        c, s = math.cos(th / 2), math.sin(th / 2)
        if k == 0:
            return 0.5 * np.array([[-s, -np.exp(1j * lam) * c],
                                   [np.exp(1j * phi) * c, -np.exp(1j * (phi + lam)) * s]])
        if k == 1:
            return np.array([[0, 0], [1j * np.exp(1j * phi) * s, 1j * np.exp(1j * (phi + lam)) * c]])
        return np.array([[0, -1j * np.exp(1j * lam) * s], [0, 1j * np.exp(1j * (phi + lam)) * c]])
    raise ValueError(f"{name} has no parameters")


N_PARAMS = {"RX": 1, "RY": 1, "RZ": 1, "U1": 1, "CP": 1, "U2": 2, "U3": 3}
