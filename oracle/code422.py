"""The [[4,2,2]] error-detection experiment, simulation side (test infrastructure
only).

Logical two-qubit circuits (an initial state from Tab. (errordetectionstates) and
gates from Tab. (errordetectiongates)) in a bare version on qubits (q3, q4) and an
encoded version on q0 (ancilla) and q1..q4.  Qubit q_b is bit b of the outcome
index.

* bare gates: X1 = X on q3, X2 = X on q4, Z1 = Z on q3, Z2 = Z on q4,
  HHS = CNOT12 CNOT21 CNOT12 H1 H2 (drawn as H H, CNOT(q3->q4), H H, CNOT, H H,
  CNOT), CZ = H on q4, CNOT(q3->q4), H on q4;
* encoded gates, Eqs. (errordetectionX1L)-(errordetectionCZL): X1 = X1 X3,
  X2 = X1 X2, Z1 = Z1 Z2, Z2 = Z1 Z3, HHS = H1 H2 H3 H4, CZ = Z2 Z3 S1 S2 S3 S4;
* preparations: bare |00> (nothing), |0+> (H on q4), |Phi+> (H on q3,
  CNOT(q3->q4)); encoded |00> (H q3, CNOT(q3->q2), CNOT(q2->q1), CNOT(q3->q4),
  then the ancilla checks CNOT(q1->q0), CNOT(q4->q0)), |0+> (H q2, CNOT(q2->q1),
  H q3, CNOT(q3->q4)), |Phi+> (H q3, CNOT(q3->q2), H q1, CNOT(q1->q4));
* evaluation: bare p(j0 j1) = p(q3 = j0, q4 = j1); encoded: outcomes with q0 = 1 or
  an odd number of 1's on q1 q2 q3 q4 are discarded (postselection), the rest map
  to logical strings by Eqs. (errordetection00L)-(errordetection11L) (q1q2q3q4 =
  0000/1111 -> 00, 1100/0011 -> 01, 1010/0101 -> 10, 0110/1001 -> 11) and are
  renormalised; the kept fraction is the postselection ratio;
* D_bare/enc = (1/2) sum |p^(bare/enc) - p^(id)| (Eq. (errordetectionDbareenc)),
  p^(id) the noiseless bare distribution.

Noise (a reading; the thesis's data come from transmon simulations and hardware):
after every physical gate, a depolarizing channel (p_x = p_y = p_z = p/3) and then
amplitude damping (gamma) on each qubit the gate acts on, applied as Kraus maps to
the density matrix.
"""
from __future__ import annotations

import numpy as np

from . import density as D
from . import gates as G

LOGICAL = ["X1", "X2", "Z1", "Z2", "HHS", "CZ"]
STATES = ["00", "0+", "Phi+"]

_BARE_GATES = {
    "X1": [("X", (3,))], "X2": [("X", (4,))], "Z1": [("Z", (3,))], "Z2": [("Z", (4,))],
    "HHS": [("H", (3,)), ("H", (4,)), ("CNOT", (3, 4)), ("H", (3,)), ("H", (4,)), ("CNOT", (3, 4)),
            ("H", (3,)), ("H", (4,)), ("CNOT", (3, 4))],
    "CZ": [("H", (4,)), ("CNOT", (3, 4)), ("H", (4,))],
}
_ENC_GATES = {
    "X1": [("X", (1,)), ("X", (3,))], "X2": [("X", (1,)), ("X", (2,))],
    "Z1": [("Z", (1,)), ("Z", (2,))], "Z2": [("Z", (1,)), ("Z", (3,))],
    "HHS": [("H", (1,)), ("H", (2,)), ("H", (3,)), ("H", (4,))],
    "CZ": [("S", (1,)), ("S", (2,)), ("S", (3,)), ("S", (4,)), ("Z", (2,)), ("Z", (3,))],
}
_BARE_PREP = {"00": [], "0+": [("H", (4,))], "Phi+": [("H", (3,)), ("CNOT", (3, 4))]}
_ENC_PREP = {
    "00": [("H", (3,)), ("CNOT", (3, 2)), ("CNOT", (2, 1)), ("CNOT", (3, 4)), ("CNOT", (1, 0)),
           ("CNOT", (4, 0))],
    "0+": [("H", (2,)), ("CNOT", (2, 1)), ("H", (3,)), ("CNOT", (3, 4))],
    "Phi+": [("H", (3,)), ("CNOT", (3, 2)), ("H", (1,)), ("CNOT", (1, 4))],
}
# logical string (j0 j1) of each kept q1q2q3q4 pattern (Eqs. (errordetection00L)-(11L))
_CODEWORDS = {"0000": 0, "1111": 0, "1100": 1, "0011": 1, "1010": 2, "0101": 2, "0110": 3, "1001": 3}


def physical(state: str, seq, encoded: bool):
    """Physical gate list (name, qubits) of a logical circuit, in time order."""
    prep = (_ENC_PREP if encoded else _BARE_PREP)[state]
    table = _ENC_GATES if encoded else _BARE_GATES
    out = list(prep)
    for g in seq:
        out += table[g]
    return out


def _matrix(name):
    return {"X": G.matrix("X"), "Z": G.matrix("Z"), "H": G.matrix("H"), "S": G.matrix("S"),
            "CNOT": G.matrix("CNOT")}[name]


def run(ops, n: int = 5, p: float = 0.0, gamma: float = 0.0) -> np.ndarray:
    """Outcome probabilities (index bit b = qubit q_b) of a physical circuit from
    |0...0>, noise after every gate on the qubits it touches."""
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1.0
    dep = D.depolarizing_kraus(p / 3, p / 3, p / 3)
    ad = D.amplitude_damping_kraus(1.0, gamma)
    for name, qs in ops:
        # two-qubit matrices: the first listed qubit is the most significant local bit
        rho = D.apply_unitary(rho, n, _matrix(name), list(qs))
        if p > 0 or gamma > 0:
            for q in qs:
                rho = D.apply_kraus(rho, n, dep, [q])
                rho = D.apply_kraus(rho, n, ad, [q])
    return D.probabilities(rho)


def bare_distribution(probs5: np.ndarray) -> np.ndarray:
    """p(j0 j1), j0 = q3, j1 = q4, from the outcome probabilities of 5 qubits."""
    out = np.zeros(4)
    for J, pj in enumerate(probs5):
        out[2 * ((J >> 3) & 1) + ((J >> 4) & 1)] += pj
    return out


def postselect(probs5: np.ndarray):
    """(p^(enc) over logical j0 j1, postselection ratio)."""
    out = np.zeros(4)
    for J, pj in enumerate(probs5):
        if J & 1:                                   # ancilla q0 = 1
            continue
        w = "".join(str((J >> b) & 1) for b in (1, 2, 3, 4))
        if w.count("1") % 2:                        # odd parity: discarded
            continue
        out[_CODEWORDS[w]] += pj
    ratio = float(out.sum())
    return (out / ratio if ratio > 0 else out), ratio


def distance(p, q) -> float:
    return 0.5 * float(np.sum(np.abs(np.asarray(p) - np.asarray(q))))


def evaluate(state: str, seq, p: float = 0.0, gamma: float = 0.0):
    """(p_id, p_bare, p_enc, ratio, D_bare, D_enc) of one logical circuit."""
    p_id = bare_distribution(run(physical(state, seq, False)))
    p_bare = bare_distribution(run(physical(state, seq, False), p=p, gamma=gamma))
    p_enc, ratio = postselect(run(physical(state, seq, True), p=p, gamma=gamma))
    return p_id, p_bare, p_enc, ratio, distance(p_bare, p_id), distance(p_enc, p_id)
