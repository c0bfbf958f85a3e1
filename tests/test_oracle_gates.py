"""Pins of the oracle's gate matrices against the thesis (not its own formulas).

* rotations against the matrix exponential exp(-i t sigma / 2) (the definition
  in section "Elementary quantum gates"), computed by scipy's expm;
* U1/U2/U3 of Tab. (elementarygateset) against the rotation products of Eqs.
  (singlequbitU1)-(singlequbitU3) with their printed phase factors c_1..c_3;
* the table's "In U gates" and "Alternatives" columns (equal up to phase);
* CNOT's XOR rule (Eq. (cnotgate)), CZ = H_2 CNOT_12 H_2 (section on encoded
  gates), the printed two-qubit QFT matrix (Eq. (twoqubitqft)).
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from conftest import golden_path
from oracle import gates as G
from oracle import statevector as SV


def _angle(tok):
    return float(tok.replace("*pi", "")) * math.pi if "pi" in tok else float(tok)


def _rows(name):
    out = []
    for line in open(golden_path(name)):
        line = line.split("#")[0].strip()
        if line:
            out.append(line.split())
    return out


@pytest.mark.parametrize("t", [-2.7, -0.4, 0.0, 0.3, 1.5707963267948966, 3.1])
def test_rotations_are_exponentials(t):
    for sig, f in ((G.SX, G.rx), (G.SY, G.ry), (G.SZ, G.rz)):
        np.testing.assert_allclose(f(t), expm(-0.5j * t * sig), atol=1e-14)


def test_u_gates_equal_rotation_products_with_printed_phases():
    rng = np.random.default_rng(7)
    for _ in range(20):
        th, ph, la = rng.uniform(-math.pi, math.pi, 3)
        c1 = np.exp(0.5j * la)
        c23 = np.exp(0.5j * (ph + la))
        np.testing.assert_allclose(G.u1(la), c1 * G.rz(la), atol=1e-14)
        np.testing.assert_allclose(
            G.u2(ph, la), c23 * G.rz(ph + math.pi / 2) @ G.rx(math.pi / 2) @ G.rz(la - math.pi / 2),
            atol=1e-14)
        np.testing.assert_allclose(
            G.u3(th, ph, la),
            c23 * G.rz(ph + 3 * math.pi) @ G.rx(math.pi / 2) @ G.rz(th + math.pi)
            @ G.rx(math.pi / 2) @ G.rz(la), atol=1e-14)


def test_table_u_gate_column():
    rows = _rows("gate_table_relations.txt")
    assert len(rows) == 10
    for gate, ug, *ps in rows:
        ang = [_angle(p) for p in ps]
        ref = G.matrix(ug, ang)
        assert SV.matrix_distance(G.matrix(gate), ref) < 1e-28, gate
    for k in range(1, 7):
        assert SV.matrix_distance(G.matrix("RK", (k,)), G.u1(2 * math.pi / 2 ** k)) < 1e-28


def test_table_alternatives_column():
    f = {"x": G.rx, "y": G.ry, "z": G.rz}
    for gate, ax, t in _rows("gate_table_alternatives.txt"):
        assert SV.matrix_distance(G.matrix(gate), f[ax](_angle(t))) < 1e-28, gate
    # +X, -X, +Y, -Y are the rotations exactly (no phase)
    np.testing.assert_allclose(G.matrix("PX"), G.rx(-math.pi / 2), atol=1e-15)
    np.testing.assert_allclose(G.matrix("MX"), G.rx(math.pi / 2), atol=1e-15)
    np.testing.assert_allclose(G.matrix("PY"), G.ry(-math.pi / 2), atol=1e-15)
    np.testing.assert_allclose(G.matrix("MY"), G.ry(math.pi / 2), atol=1e-15)


@pytest.mark.parametrize("name,params", [
    ("I", ()), ("X", ()), ("Y", ()), ("Z", ()), ("H", ()), ("S", ()), ("SDG", ()), ("T", ()),
    ("TDG", ()), ("PX", ()), ("MX", ()), ("PY", ()), ("MY", ()), ("RX", (0.3,)), ("RY", (1.1,)),
    ("RZ", (-2.0,)), ("U1", (0.7,)), ("U2", (0.2, -1.3)), ("U3", (0.9, 0.4, 2.2)), ("RK", (3,)),
    ("CNOT", ()), ("CZ", ()), ("CP", (0.6,)), ("SWAP", ())])
def test_unitary(name, params):
    U = G.matrix(name, params)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14)


def test_cnot_xor_rule():
    # control = thesis qubit 0 = first listed = most significant local bit
    for j0 in (0, 1):
        for j1 in (0, 1):
            e = np.zeros(4)
            e[2 * j0 + j1] = 1
            out = G.CNOT @ e
            assert out[2 * j0 + (j0 ^ j1)] == 1


def test_cz_from_h_cnot_h():
    # CZ = H_2 CNOT_12 H_2 (bare implementation quoted with the [[4,2,2]] gates)
    ops = [("H", (0,), (), None), ("CNOT", (1, 0), (), None), ("H", (0,), (), None)]
    np.testing.assert_allclose(SV.circuit_unitary(ops, 2), G.CZ, atol=1e-15)


def test_swap_is_three_cnots():
    ops = [("CNOT", (1, 0), (), None), ("CNOT", (0, 1), (), None), ("CNOT", (1, 0), (), None)]
    np.testing.assert_allclose(SV.circuit_unitary(ops, 2), G.SWAP, atol=1e-15)


def _qft2_golden():
    rows = _rows("qft2_matrix.txt")
    scale = float(rows[0][1])
    M = np.array([[complex(*map(float, e.split(","))) for e in r] for r in rows[1:]])
    return scale * M


def test_qft2_printed_matrix():
    # thesis qubit 0 = bit 1, thesis qubit 1 = bit 0
    q0, q1 = 1, 0
    ops = [("H", (q0,), (), None), ("TDG", (q0,), (), None), ("CNOT", (q1, q0), (), None),
           ("TDG", (q0,), (), None), ("CNOT", (q1, q0), (), None), ("S", (q0,), (), None),
           ("T", (q1,), (), None), ("H", (q1,), (), None), ("CNOT", (q0, q1), (), None),
           ("CNOT", (q1, q0), (), None), ("CNOT", (q0, q1), (), None)]
    U = SV.circuit_unitary(ops, 2)
    np.testing.assert_allclose(U, _qft2_golden(), atol=1e-15)
    # the same matrix from the general closed form of Eq. (multiqubitqft)
    cols = np.stack([SV.qft_amplitudes(2, J) for J in range(4)], axis=1)
    np.testing.assert_allclose(cols, _qft2_golden(), atol=1e-15)


def test_derivatives_match_finite_differences():
    h = 1e-6
    for name, ps in (("RX", [0.4]), ("RY", [-1.2]), ("RZ", [2.0]), ("U1", [0.3]), ("CP", [1.1]),
                     ("U2", [0.5, -0.7]), ("U3", [0.9, 0.4, -2.2])):
        for k in range(G.N_PARAMS[name]):
            pp, pm = list(ps), list(ps)
            pp[k] += h
            pm[k] -= h
            fd = (G.matrix(name, pp) - G.matrix(name, pm)) / (2 * h)
            np.testing.assert_allclose(G.dmatrix(name, ps, k), fd, atol=1e-9)
