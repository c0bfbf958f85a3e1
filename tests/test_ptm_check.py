"""The opt-in channel check (QS_DM_VALIDATE / qs_ptm_check) on the host, no GPU.

Trace preservation is the PTM's first row (1, 0, ..., 0) and complete positivity
a positive semidefinite Choi matrix (section "Quantum operations").  The PTMs are
built by the oracle from Kraus operators and unitaries (channels that must pass)
and from maps that are not channels: a trace-decreasing amplitude damping (one
Kraus operator kept), the transpose (positive but not completely positive, PTM
diag(1, 1, -1, 1)), an over-depolarizing map (p = 1.2), and a non-finite entry.
"""
import math

import numpy as np
import pytest

import paper_2008_13490_gb300 as qs
from oracle import density as D
from oracle import gates as G


def _check(ptms, n):
    try:
        return qs.ptm_check(ptms, n), ""
    except qs.QsimError as e:
        assert e.status == qs.QS_EINVAL
        return None, str(e)


def _depol(p):
    return D.ptm_kraus(D.depolarizing_kraus(p / 3, p / 3, p / 3))


def test_channels_pass():
    good = [D.ptm_unitary(G.matrix("H")), D.ptm_unitary(G.rx(0.3)), _depol(0.01), _depol(1.0),
            D.ptm_kraus(D.amplitude_damping_kraus(1.0, 0.2)),
            D.ptm_kraus(D.amplitude_damping_kraus(0.7, 0.4)),
            _depol(0.05) @ D.ptm_kraus(D.amplitude_damping_kraus(1.0, 0.1))]
    bad, msg = _check(np.stack(good), 1)
    assert bad == -1, msg
    two = [D.ptm_unitary(G.CNOT), np.kron(_depol(0.02), D.ptm_kraus(D.amplitude_damping_kraus(1.0, 0.3))),
           D.ptm_unitary(G.matrix("CZ"))]
    bad, msg = _check(np.stack(two), 2)
    assert bad == -1, msg


def test_trace_decreasing_map_is_rejected():
    m0 = D.amplitude_damping_kraus(1.0, 0.3)[0]
    ptms = np.stack([_depol(0.1), D.ptm_kraus([m0])])
    bad, msg = _check(ptms, 1)
    assert bad is None and "PTM 1" in msg and "trace preserving" in msg


def test_transpose_is_rejected_as_not_completely_positive():
    T = D.ptm_of_map(lambda P: P.T, 1)
    np.testing.assert_allclose(T, np.diag([1.0, 1.0, -1.0, 1.0]), atol=1e-15)
    ptms = np.stack([D.ptm_unitary(G.matrix("X")), _depol(0.3), T])
    bad, msg = _check(ptms, 1)
    assert bad is None and "PTM 2" in msg and "completely positive" in msg
    T2 = D.ptm_of_map(lambda P: P.T, 2)
    bad, msg = _check(np.stack([D.ptm_unitary(G.CNOT), T2]), 2)
    assert bad is None and "PTM 1" in msg and "completely positive" in msg


def test_over_depolarizing_is_rejected():
    # PTM diag(1, l, l, l) with l = 1 - 4p/3 is a channel iff p in [0, 1]; p = 1.2
    # has a Choi eigenvalue (1 + 3 l) / 4 < 0
    lam = 1 - 4 * 1.2 / 3
    bad, msg = _check(np.diag([1.0, lam, lam, lam]), 1)
    assert bad is None and "completely positive" in msg
    lam = 1 - 4 * 1.0 / 3
    assert _check(np.diag([1.0, lam, lam, lam]), 1)[0] == -1


def test_non_finite_and_bad_arguments():
    G1 = _depol(0.1)
    G1[2, 3] = math.nan
    bad, msg = _check(G1, 1)
    assert bad is None and "not finite" in msg
    with pytest.raises(qs.QsimError):
        qs.ptm_check(np.eye(64), 3)
