"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and lays out circuit *structure*; it
holds none of the simulation arithmetic (no gate matrices from gate names, no
state updates, no channels, no probabilities).  Both the CUDA path and the
oracle receive exactly the same records from here.

Circuit record: a list of ops ``(name, qubits, params, matrix)``

* ``name``   -- gate name from the elementary gate set of the thesis
  (Tab. (elementarygateset)): ``I X Y Z H S SDG T TDG PX MX PY MY
  RX RY RZ U1 U2 U3 RK`` for one qubit, ``CNOT CZ CP SWAP`` for two qubits,
  ``MAT1``/``MAT2`` for an explicit 2x2 / 4x4 complex matrix.
* ``qubits`` -- bit positions (bit 0 = least significant bit of the amplitude
  index J).  For two-qubit gates ``qubits[0]`` is the most significant bit of
  the gate's local 2-bit index (the control of CNOT/CZ/CP).
* ``params`` -- angles (radians) or the integer k of R(k).
* ``matrix`` -- ``None`` or a complex128 array (explicit gates only), laid out
  ``U[out][in]`` in the local index above.

Noisy batches (the gate-set-tomography-like workload) use their own record,
see :func:`noisy_batch`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng", "haar_su2", "random_state", "layered_haar_cnot", "layered_haar_cz",
    "qft_circuit", "random_basis_index", "inverse_circuit", "random_gate_mix",
    "NoisyBatch", "noisy_batch", "multinomial_counts", "serving_stream",
    "singlet_circuit", "ghz_circuit",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-based seeded generator (Philox) so every consumer draws the same stream."""
    return np.random.Generator(np.random.Philox(seed))


def haar_su2(g: np.random.Generator) -> np.ndarray:
    """Haar-random SU(2) from a normalised complex Gaussian pair (a, b).

    The pair is a random pure one-qubit state drawn as in the thesis's recipe
    for random states (normal real and imaginary parts, then normalised;
    Sec. "Unitarity" of the gate-metrics chapter).  The unitary is [[a, -b*], [b, a*]].
    """
    v = g.normal(size=4)
    a = complex(v[0], v[1])
    b = complex(v[2], v[3])
    s = math.sqrt(abs(a) ** 2 + abs(b) ** 2)
    a /= s
    b /= s
    return np.array([[a, -b.conjugate()], [b, a.conjugate()]], dtype=np.complex128)


def random_state(n: int, g: np.random.Generator) -> np.ndarray:
    """Random pure state: complex Gaussian coefficients, normalised (Sec. "Unitarity")."""
    v = g.normal(size=(2, 1 << n))
    psi = v[0] + 1j * v[1]
    return psi / np.linalg.norm(psi)


def random_basis_index(n: int, seed: int) -> int:
    return int(rng(seed).integers(0, 1 << n))


def layered_haar_cnot(n: int, layers: int, seed: int):
    """Layers of Haar SU(2) on every qubit, then CNOTs on a random perfect matching.

    Matching: Fisher-Yates shuffle of the qubits, pairs (2k, 2k+1), control =
    first of the pair.  With odd n one qubit idles in each layer.
    """
    g = rng(seed)
    ops = []
    for _ in range(layers):
        for q in range(n):
            ops.append(("MAT1", (q,), (), haar_su2(g)))
        perm = list(range(n))
        for i in range(n - 1, 0, -1):
            j = int(g.integers(0, i + 1))
            perm[i], perm[j] = perm[j], perm[i]
        for k in range(n // 2):
            ops.append(("CNOT", (perm[2 * k], perm[2 * k + 1]), (), None))
    return ops


def layered_haar_cz(n: int, layers: int, seed: int):
    """Layers of Haar SU(2) on every qubit plus brickwork CZ.

    Layer l (0-based) even pairs (0,1),(2,3),...; odd pairs (1,2),(3,4),...
    """
    g = rng(seed)
    ops = []
    for layer in range(layers):
        for q in range(n):
            ops.append(("MAT1", (q,), (), haar_su2(g)))
        for a in range(layer % 2, n - 1, 2):
            ops.append(("CZ", (a, a + 1), (), None))
    return ops


def haar_su4(g: np.random.Generator) -> np.ndarray:
    """Haar-random 4x4 unitary: QR of a complex Gaussian matrix with the phases of R's
    diagonal moved into Q."""
    z = g.normal(size=(4, 4)) + 1j * g.normal(size=(4, 4))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def layered_su4(n: int, depth: int, seed: int):
    """`depth` brickwork layers of dense random two-qubit gates (MAT2): layer l acts on
    the pairs (a, a+1), a = l % 2, l % 2 + 2, ..."""
    g = rng(seed)
    ops = []
    for layer in range(depth):
        for a in range(layer % 2, n - 1, 2):
            ops.append(("MAT2", (a + 1, a), (), haar_su4(g)))
    return ops


def code422_sequences(count: int, seed: int, max_len: int = 10):
    """`count` logical gate sequences for the error-detection experiment: lengths
    uniform in 1..max_len over {X1, X2, Z1, Z2, HHS, CZ}; each used with the three
    initial states |00>, |0+>, |Phi+> (3 x count circuits, as (state, sequence))."""
    g = rng(seed)
    names = ["X1", "X2", "Z1", "Z2", "HHS", "CZ"]
    seqs = [[names[int(k)] for k in g.integers(0, 6, size=int(g.integers(1, max_len + 1)))]
            for _ in range(count)]
    return [(state, seq) for state in ("00", "0+", "Phi+") for seq in seqs]


def qft_circuit(n: int):
    """Textbook QFT on n qubits written in the thesis's gate set.

    Thesis qubit i (i-th tensor factor, j_0 most significant) is bit n-1-i.
    For i = 0..n-1: H on qubit i, then a controlled R(k) (k = j-i+1) from every
    later qubit j; finally the qubit order is reversed with SWAPs.  The
    controlled R(k) is the diagonal CP(2*pi/2^k).
    """
    ops = []
    bit = lambda i: n - 1 - i  # noqa: E731
    for i in range(n):
        ops.append(("H", (bit(i),), (), None))
        for j in range(i + 1, n):
            k = j - i + 1
            ops.append(("CP", (bit(j), bit(i)), (2.0 * math.pi / (1 << k),), None))
    for i in range(n // 2):
        ops.append(("SWAP", (bit(i), bit(n - 1 - i)), (), None))
    return ops


def ghz_circuit(n: int):
    """H on the most significant bit, then a CNOT chain down to bit 0."""
    ops = [("H", (n - 1,), (), None)]
    for b in range(n - 1, 0, -1):
        ops.append(("CNOT", (b, b - 1), (), None))
    return ops


def singlet_circuit(theta0: float, theta1: float):
    """Fig. (singletcircuit): X on both, H_0, CNOT_01, then H U1(t) H per qubit.

    Thesis qubit 0 is bit 1, thesis qubit 1 is bit 0.
    """
    q0, q1 = 1, 0
    return [
        ("X", (q0,), (), None), ("X", (q1,), (), None),
        ("H", (q0,), (), None),
        ("CNOT", (q0, q1), (), None),
        ("H", (q0,), (), None), ("U1", (q0,), (theta0,), None), ("H", (q0,), (), None),
        ("H", (q1,), (), None), ("U1", (q1,), (theta1,), None), ("H", (q1,), (), None),
    ]


_INVERSE_NAME = {"S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T", "PX": "MX", "MX": "PX",
                 "PY": "MY", "MY": "PY"}


def inverse_circuit(ops):
    """Structural inverse: reversed order, each gate replaced by its inverse.

    Self-inverse names are kept, rotation angles negated, explicit matrices
    conjugate-transposed (a data transform of the input record, not a state
    update).  U2/U3/RK are emitted as explicit MAT-free equivalents by negating
    and swapping their angles where the inverse stays in the family.
    """
    out = []
    for name, qs, ps, m in reversed(ops):
        if name in ("MAT1", "MAT2"):
            out.append((name, qs, ps, np.conjugate(m.T).copy()))
        elif name in ("RX", "RY", "RZ", "U1", "CP"):
            out.append((name, qs, tuple(-p for p in ps), None))
        elif name == "U3":
            th, ph, la = ps
            out.append(("U3", qs, (-th, -la, -ph), None))
        elif name in _INVERSE_NAME:
            out.append((_INVERSE_NAME[name], qs, ps, None))
        elif name in ("I", "X", "Y", "Z", "H", "CNOT", "CZ", "SWAP"):
            out.append((name, qs, ps, None))
        else:
            raise ValueError(f"no structural inverse for {name}")
    return out


_ONE_Q_NAMES = ["I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "PX", "MX", "PY", "MY",
                "RX", "RY", "RZ", "U1", "U2", "U3", "RK", "MAT1"]
_TWO_Q_NAMES = ["CNOT", "CZ", "CP", "SWAP", "MAT2"]


def random_gate_mix(n: int, count: int, seed: int, two_q_fraction: float = 0.3,
                    names1=None, names2=None):
    """Random sequence over the whole gate set (every name, random qubits)."""
    g = rng(seed)
    names1 = list(names1 or _ONE_Q_NAMES)
    names2 = list(names2 or _TWO_Q_NAMES)
    ops = []
    for _ in range(count):
        if n >= 2 and g.random() < two_q_fraction:
            name = names2[int(g.integers(0, len(names2)))]
            a, b = (int(x) for x in g.choice(n, size=2, replace=False))
            params = (float(g.uniform(-math.pi, math.pi)),) if name == "CP" else ()
            m = None
            if name == "MAT2":
                z = g.normal(size=(4, 4)) + 1j * g.normal(size=(4, 4))
                qm, r = np.linalg.qr(z)
                m = qm * (np.diag(r) / np.abs(np.diag(r)))
            ops.append((name, (a, b), params, m))
        else:
            name = names1[int(g.integers(0, len(names1)))]
            q = int(g.integers(0, n))
            if name in ("RX", "RY", "RZ", "U1"):
                params = (float(g.uniform(-math.pi, math.pi)),)
            elif name == "U2":
                params = tuple(float(x) for x in g.uniform(-math.pi, math.pi, size=2))
            elif name == "U3":
                params = tuple(float(x) for x in g.uniform(-math.pi, math.pi, size=3))
            elif name == "RK":
                params = (float(int(g.integers(1, 8))),)
            else:
                params = ()
            m = haar_su2(g) if name == "MAT1" else None
            ops.append((name, (q,), params, m))
    return ops


# ---------------------------------------------------------------------------
# Noisy batches of small circuits (gate-set-tomography-shaped workload)
# ---------------------------------------------------------------------------

# op codes of a noisy circuit: X90(theta_x) on q, Y90(theta_y) on q, CZ on (a, b),
# IDLE on the whole register.
OP_X90, OP_Y90, OP_CZ, OP_IDLE = 0, 1, 2, 3


@dataclass
class NoisyBatch:
    """A batch of small noisy circuits.

    ``nq[c]``: qubits of circuit c; ``op_off[c]:op_off[c+1]`` its ops in
    ``ops`` (int32 rows ``(code, a, b)``, ``b`` = -1 when unused);
    ``params[c] = (theta_x, theta_y, p_dep, gamma_ad)``; ``counts`` holds the
    multinomial outcome counts of circuit c at ``cnt_off[c]:cnt_off[c+1]``
    (2^nq[c] entries) or is None until filled in.
    """
    nq: np.ndarray
    op_off: np.ndarray
    ops: np.ndarray
    params: np.ndarray
    cnt_off: np.ndarray
    counts: np.ndarray | None = None

    @property
    def size(self) -> int:
        return int(self.nq.shape[0])

    def circuit(self, c: int):
        return int(self.nq[c]), self.ops[self.op_off[c]:self.op_off[c + 1]], self.params[c]

    def subset(self, idx):
        idx = np.asarray(idx, dtype=np.int64)
        nq = self.nq[idx]
        lens = self.op_off[idx + 1] - self.op_off[idx]
        op_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        ops = np.concatenate([self.ops[self.op_off[c]:self.op_off[c + 1]] for c in idx]) \
            if len(idx) else np.zeros((0, 3), np.int32)
        cnt_off = np.concatenate([[0], np.cumsum(1 << nq.astype(np.int64))]).astype(np.int64)
        counts = None
        if self.counts is not None:
            counts = np.concatenate([self.counts[self.cnt_off[c]:self.cnt_off[c + 1]] for c in idx])
        return NoisyBatch(nq.copy(), op_off, ops.astype(np.int32), self.params[idx].copy(),
                          cnt_off, counts)


def noisy_batch(count: int = 4096, seed: int = 4001, n_range=(1, 6), len_range=(1, 256),
                theta_sigma: float = 0.02, p_range=(1e-4, 1e-2), gamma_range=(1e-4, 1e-2)):
    """Batch shaped like the thesis's two-qubit GST data set, widened to 1-6 qubits.

    n ~ U{n_range}, L ~ U{len_range}; gates uniform over {X90, Y90, CZ, idle};
    X90/Y90 on a uniform qubit, CZ on a uniform ordered pair (an X90 when
    n = 1); theta ~ pi/2 + N(0, theta_sigma^2) per circuit and gate kind;
    p ~ U[p_range], gamma ~ U[gamma_range] per circuit.
    """
    g = rng(seed)
    nq = g.integers(n_range[0], n_range[1] + 1, size=count).astype(np.int32)
    lens = g.integers(len_range[0], len_range[1] + 1, size=count).astype(np.int64)
    op_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ops = np.full((int(op_off[-1]), 3), -1, dtype=np.int32)
    for c in range(count):
        n = int(nq[c])
        L = int(lens[c])
        codes = g.integers(0, 4, size=L)
        for k in range(L):
            code = int(codes[k])
            row = ops[op_off[c] + k]
            if code == OP_CZ and n == 1:
                code = OP_X90
            if code in (OP_X90, OP_Y90):
                row[:] = (code, int(g.integers(0, n)), -1)
            elif code == OP_CZ:
                a, b = (int(x) for x in g.choice(n, size=2, replace=False))
                row[:] = (code, a, b)
            else:
                row[:] = (OP_IDLE, -1, -1)
    params = np.empty((count, 4), dtype=np.float64)
    params[:, 0] = math.pi / 2 + theta_sigma * g.normal(size=count)
    params[:, 1] = math.pi / 2 + theta_sigma * g.normal(size=count)
    params[:, 2] = g.uniform(p_range[0], p_range[1], size=count)
    params[:, 3] = g.uniform(gamma_range[0], gamma_range[1], size=count)
    cnt_off = np.concatenate([[0], np.cumsum(1 << nq.astype(np.int64))]).astype(np.int64)
    return NoisyBatch(nq, op_off, ops, params, cnt_off, None)


def multinomial_counts(probs_per_circuit, shots: int, seed: int) -> np.ndarray:
    """1000-shot style multinomial draws, one per distribution (concatenated)."""
    g = rng(seed)
    out = []
    for p in probs_per_circuit:
        p = np.clip(np.asarray(p, dtype=np.float64), 0.0, None)
        p = p / p.sum()
        out.append(g.multinomial(shots, p).astype(np.int32))
    return np.concatenate(out) if out else np.zeros(0, np.int32)


def synthetic_counts(batch: NoisyBatch, shots: int, seed: int) -> np.ndarray:
    """Counts that do not depend on any simulation: a multinomial over a
    random distribution concentrated on a few outcomes per circuit."""
    g = rng(seed)
    out = []
    for c in range(batch.size):
        d = 1 << int(batch.nq[c])
        w = g.exponential(size=d) ** 4 + 1e-3
        out.append(g.multinomial(shots, w / w.sum()).astype(np.int32))
    return np.concatenate(out)


def serving_stream(count: int, seed: int, n_range=(8, 28), depth_range=(10, 200),
                   rate_hz: float = 50.0):
    """Poisson arrivals of layered Haar+brickwork-CZ circuits.

    Returns a list of (arrival_time_s, n, depth, circuit_seed).  Circuits are
    built lazily with :func:`layered_haar_cz` from ``circuit_seed``.
    """
    g = rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(g.exponential(1.0 / rate_hz))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        d = int(g.integers(depth_range[0], depth_range[1] + 1))
        out.append((t, n, d, int(g.integers(0, 2**31 - 1))))
    return out


def perturbed_params(batch: NoisyBatch, seed: int, theta_sigma: float = 0.01,
                     rate_rel: float = 0.2) -> np.ndarray:
    """Parameters near a batch's true ones, where a likelihood is evaluated:
    theta + N(0, theta_sigma^2), p and gamma scaled by U[1 - rate_rel, 1 + rate_rel]."""
    g = rng(seed)
    out = batch.params.copy()
    out[:, 0:2] += theta_sigma * g.normal(size=(batch.size, 2))
    out[:, 2:4] *= g.uniform(1 - rate_rel, 1 + rate_rel, size=(batch.size, 2))
    return out
