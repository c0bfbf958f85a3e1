"""FP64 state-vector oracle in plain C (``sv_ref.c``), for sizes where numpy is slow.

TEST INFRASTRUCTURE ONLY (tests, ``__graft_entry__.smoke()``, the benchmark's
CPU legs).  The gate matrices come from :mod:`oracle.gates`; the C code applies
each gate, embedded in the n-qubit space (Eq. (singlequbitrotationmultiplequbits)),
to every group of amplitudes that differ only in the gate's bits, in FP64 with
OpenMP over those groups.  ``build()`` compiles it with gcc (no CUDA, nothing
shared with the library).

Also here: :func:`permute_qubits`, the exact relabelling of qubits as a
permutation of amplitude indices (what a SWAP network computes, Sec. "Quantum
circuits"), written with integer index arithmetic only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import gates as G

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "sv_ref.c")
_LIB = os.path.join(_DIR, "libsv_ref.so")
_lib = None


def build() -> str:
    """Compile sv_ref.c into oracle/libsv_ref.so (gcc, OpenMP, portable flags)."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp, i32 = ctypes.POINTER(ctypes.c_double), ctypes.c_int
        lib.orc_apply1.argtypes = [dp, i32, i32, dp]
        lib.orc_apply2.argtypes = [dp, i32, i32, i32, dp]
        lib.orc_probs.argtypes = [dp, i32, dp]
        lib.orc_probs.restype = ctypes.c_double
        lib.orc_threads.restype = i32
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the C oracle uses (OMP_NUM_THREADS, else the host's cores)."""
    return int(_load().orc_threads())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def apply_matrix(psi: np.ndarray, n: int, U: np.ndarray, qubits) -> np.ndarray:
    """In place: psi <- (U on `qubits`) psi; qubits[0] is the most significant local bit."""
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.size != 1 << n:
        raise ValueError("psi must be a contiguous complex128 vector of 2^n amplitudes")
    k = len(qubits)
    if len(set(qubits)) != k or any(q < 0 or q >= n for q in qubits) or k not in (1, 2):
        raise ValueError("bad qubits")
    m = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(1 << k, 1 << k))
    flat = np.empty(2 * m.size)
    flat[0::2] = m.real.reshape(-1)
    flat[1::2] = m.imag.reshape(-1)
    lib = _load()
    if k == 1:
        lib.orc_apply1(_dptr(psi.view(np.float64)), n, int(qubits[0]), _dptr(flat))
    else:
        lib.orc_apply2(_dptr(psi.view(np.float64)), n, int(qubits[0]), int(qubits[1]), _dptr(flat))
    return psi


def apply_circuit(psi: np.ndarray, n: int, ops) -> np.ndarray:
    """Gates in time order, in place on a complex128 copy of psi (returned)."""
    psi = np.array(psi, dtype=np.complex128, copy=True)
    for name, qubits, params, mat in ops:
        apply_matrix(psi, n, G.matrix(name, params, mat), qubits)
    return psi


def probabilities(psi: np.ndarray, n: int):
    """(p_J = |a_J|^2, sum_J p_J)."""
    p = np.empty(1 << n)
    s = _load().orc_probs(_dptr(psi.view(np.float64)), n, _dptr(p))
    return p, float(s)


def permute_qubits(psi: np.ndarray, n: int, dest) -> np.ndarray:
    """Relabel qubits: the bit at position b of every index moves to position dest[b].

    out[J'] = psi[J] where bit dest[b] of J' equals bit b of J (dest a permutation
    of 0..n-1).  Only index arithmetic: the values are moved, never computed, so
    the result is exact in any precision.  SWAP(a, b) is the transposition of a and b.
    """
    dest = [int(d) for d in dest]
    if sorted(dest) != list(range(n)):
        raise ValueError("dest must be a permutation of 0..n-1")
    J = np.arange(1 << n, dtype=np.int64)
    Jp = np.zeros_like(J)
    for b in range(n):
        Jp |= ((J >> b) & 1) << dest[b]
    out = np.empty_like(psi)
    out[Jp] = psi
    return out


def source_index(K, n: int, dest):
    """Index J whose amplitude :func:`permute_qubits` moves to K (vectorised)."""
    K = np.asarray(K, dtype=np.int64)
    J = np.zeros_like(K)
    for b in range(n):
        J |= ((K >> int(dest[b])) & 1) << b
    return J


def permutation_gates(psi: np.ndarray, n: int, ops) -> np.ndarray:
    """X, CNOT and SWAP gates as what they are: permutations of basis states.

    X on q maps |J> to |J xor 2^q>; CNOT(c, t) flips bit t of J when bit c is 1
    (Eq. (cnotgate)); SWAP(a, b) exchanges bits a and b.  Each gate moves the
    amplitude of J to its image; no arithmetic touches the values.
    """
    J = np.arange(1 << n, dtype=np.int64)
    out = np.array(psi, copy=True)
    for name, qubits, _, _ in ops:
        if name == "X":
            img = J ^ (1 << qubits[0])
        elif name == "CNOT":
            c, t = qubits
            img = J ^ (((J >> c) & 1) << t)
        elif name == "SWAP":
            a, b = qubits
            d = ((J >> a) ^ (J >> b)) & 1
            img = J ^ ((d << a) | (d << b))
        else:
            raise ValueError(f"{name} is not a permutation gate")
        nxt = np.empty_like(out)
        nxt[img] = out
        out = nxt
    return out


def permutation_source(K, n: int, ops):
    """Index J whose amplitude :func:`permutation_gates` moves to K (vectorised).

    Every X, CNOT and SWAP is its own inverse, so J is K mapped by the gates in
    reverse order."""
    K = np.array(K, dtype=np.int64, copy=True)
    for name, qubits, _, _ in reversed(ops):
        if name == "X":
            K ^= 1 << qubits[0]
        elif name == "CNOT":
            c, t = qubits
            K ^= ((K >> c) & 1) << t
        elif name == "SWAP":
            a, b = qubits
            d = ((K >> a) ^ (K >> b)) & 1
            K ^= (d << a) | (d << b)
        else:
            raise ValueError(f"{name} is not a permutation gate")
    return K


def swap_network_dest(n: int, swaps) -> list:
    """Final position of each qubit's bit after SWAPs (a, b) in time order."""
    where = list(range(n))            # where[b]: current position of the bit that started at b
    at = list(range(n))               # at[p]: original bit now at position p
    for a, b in swaps:
        at[a], at[b] = at[b], at[a]
        where[at[a]], where[at[b]] = a, b
    return where
