"""Pins of the [[4,2,2]] error-detection oracle: the encoded preparations give
the codewords of Eqs. (errordetection00L)-(errordetectionPhi+L); every logical
gate of Eqs. (errordetectionX1L)-(errordetectionCZL) on the code space does what
its bare version does; the postselection rule discards single bit flips and the
ancilla flag; distances and ratios of noisy runs are proper."""

import numpy as np
import pytest

import workloads as W
from oracle import code422 as C


def _support(probs, tol=1e-12):
    return {J: round(float(p), 12) for J, p in enumerate(probs) if p > tol}


def _J(q0, word):
    # outcome index of ancilla bit q0 and data bits q1 q2 q3 q4 given as a string
    J = q0
    for b, ch in zip((1, 2, 3, 4), word):
        J |= int(ch) << b
    return J


@pytest.mark.parametrize("state,words", [("00", ["0000", "1111"]),
                                         ("0+", ["0000", "1100", "0011", "1111"]),
                                         ("Phi+", ["0000", "0110", "1001", "1111"])])
def test_encoded_preparations_are_codewords(state, words):
    probs = C.run(C.physical(state, [], True))
    w = 1.0 / len(words)
    assert _support(probs) == {_J(0, x): w for x in words}


@pytest.mark.parametrize("state", C.STATES)
@pytest.mark.parametrize("gate", C.LOGICAL)
def test_each_logical_gate_matches_bare(state, gate):
    p_id, p_bare, p_enc, ratio, d_bare, d_enc = C.evaluate(state, [gate])
    assert ratio == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(p_enc, p_id, atol=1e-12)
    assert d_bare == pytest.approx(0.0, abs=1e-12) and d_enc == pytest.approx(0.0, abs=1e-12)


def test_logical_closed_forms():
    # index 2 j0 + j1: X1 |00> = |10>, X2 |00> = |01>, CZ and Z leave |00> alone,
    # HHS |00> = |++> (uniform), HHS |0+> = swap(|+0>) = |0+>
    assert np.allclose(C.evaluate("00", ["X1"])[0], [0, 0, 1, 0])
    assert np.allclose(C.evaluate("00", ["X2"])[0], [0, 1, 0, 0])
    assert np.allclose(C.evaluate("00", ["CZ", "Z1", "Z2"])[0], [1, 0, 0, 0])
    assert np.allclose(C.evaluate("00", ["HHS"])[0], [0.25] * 4)
    assert np.allclose(C.evaluate("0+", ["HHS"])[0], [0.5, 0.5, 0, 0])
    assert np.allclose(C.evaluate("Phi+", [])[0], [0.5, 0, 0, 0.5])


def test_random_logical_circuits_are_exact_without_noise():
    g = W.rng(77)
    for _ in range(20):
        seq = [C.LOGICAL[int(k)] for k in g.integers(0, 6, size=int(g.integers(1, 11)))]
        state = C.STATES[int(g.integers(0, 3))]
        p_id, _, p_enc, ratio, _, d_enc = C.evaluate(state, seq)
        assert ratio == pytest.approx(1.0, abs=1e-12) and d_enc == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("err,qubit,kept", [("X", 2, 0.0), ("X", 4, 0.0), ("X", 0, 0.0),
                                             ("Z", 3, 1.0)])
def test_postselection_rule(err, qubit, kept):
    # one error after the encoded |00> preparation: a bit flip on a data qubit makes
    # the parity odd, one on the ancilla sets its flag; a phase flip is invisible
    ops = C.physical("00", [], True) + [(err, (qubit,))]
    _, ratio = C.postselect(C.run(ops))
    assert ratio == pytest.approx(kept, abs=1e-12)


def test_noisy_evaluation_is_proper():
    p_id, p_bare, p_enc, ratio, d_bare, d_enc = C.evaluate("Phi+", ["HHS", "CZ", "X1"], p=0.02, gamma=0.01)
    assert 0.0 < ratio < 1.0
    for p in (p_bare, p_enc):
        assert np.all(p >= -1e-15) and p.sum() == pytest.approx(1.0, abs=1e-12)
    assert 0.0 < d_bare < 1.0 and 0.0 <= d_enc < 1.0
    assert d_bare == pytest.approx(C.distance(p_bare, p_id))
    assert C.distance([1, 0, 0, 0], [0, 1, 0, 0]) == 1.0
