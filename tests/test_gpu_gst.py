"""GPU parity of the GST predictions for repeated gates (dm_gst_series,
dm_gst_power) against the oracle.

Tolerances.  The series runs in FP32: each repetition is one 16-term
matrix-vector product (relative rounding <= 16 u, u = 6e-8) of a contractive
map, so errors add over r and stay below r_max * 16 u * max|v| ~ 5e-4 at
r_max = 1000; observed errors are far smaller and the test asks 5e-5.  The
power runs in FP64 over ~2 log2 r products: 1e-12.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import density as D
from oracle import gates as G
from oracle import gst as GS

pytestmark = pytest.mark.gpu

XI, YI, IX, IY, II, CNOT = range(6)
PREPS = [[], [XI, XI], [IY, YI], [IX, IX, XI, XI, YI, CNOT]]   # |00>, |10>, |++>, |Psi^->


def _ideal():
    I2 = np.eye(2)
    x90, y90 = G.rx(math.pi / 2), G.ry(math.pi / 2)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    Us = [np.kron(x90, I2), np.kron(y90, I2), np.kron(I2, x90), np.kron(I2, y90), np.eye(4), cnot]
    return [D.ptm_unitary(U) for U in Us]


def _tables(count, seed):
    """`count` noisy GST gate sets: each ideal gate followed by depolarizing and
    amplitude damping on both qubits, rates drawn per set."""
    g = W.rng(seed)
    ideal = _ideal()
    out = []
    for _ in range(count):
        p, gam = g.uniform(1e-3, 2e-2, size=2)
        N1 = D.ptm_kraus(D.amplitude_damping_kraus(1.0, gam)) @ D.ptm_kraus(
            D.depolarizing_kraus(p / 3, p / 3, p / 3))
        N2 = np.kron(N1, N1)
        out += [N2 @ T for T in ideal]
    return out


def _batch(nsets, seed):
    ptms = _tables(nsets, seed)
    rho = np.zeros((4, 4), dtype=complex)
    rho[0, 0] = 1
    rho_v = D.pauli_vector(rho, 2)
    E = np.array([D.effect_vector(J, 2) for J in range(4)])
    gate, prep = [], []
    for s in range(nsets):
        for gi in range(6):
            for pr in PREPS:
                gate.append(6 * s + gi)
                prep.append([6 * s + k for k in pr] + [-1] * (8 - len(pr)))
    return ptms, rho_v, E, np.array(gate, dtype=np.int32), np.array(prep, dtype=np.int32)


def _dev(qs, ptms, rho, E, gate, prep):
    f = lambda a, dt: torch.tensor(np.asarray(a), dtype=dt, device="cuda")  # noqa: E731
    return (f(np.stack(ptms), torch.float64), f(rho, torch.float64), f(E, torch.float64),
            f(gate, torch.int32), f(prep, torch.int32))


def test_series_matches_oracle(qs):
    ptms, rho, E, gate, prep = _batch(3, 1200)
    out = qs.gst_series(2, *_dev(qs, ptms, rho, E, gate, prep), r_max=1000).cpu().numpy()
    worst = 0.0
    for i in range(len(gate)):
        pr = [k for k in prep[i] if k >= 0]
        ref = GS.series(ptms, rho, E, int(gate[i]), pr, 1000)
        worst = max(worst, float(np.max(np.abs(out[i] - ref))))
    assert worst < 5e-5, worst


@pytest.mark.parametrize("r", [0, 1, 2, 7, 1000, 10**6, 2**31 + 5])
def test_power_matches_oracle(qs, r):
    ptms, rho, E, gate, prep = _batch(2, 1300)
    reps = torch.full((len(gate),), r, dtype=torch.int64, device="cuda")
    out = qs.gst_power(2, *_dev(qs, ptms, rho, E, gate, prep), reps).cpu().numpy()
    for i in range(len(gate)):
        pr = [k for k in prep[i] if k >= 0]
        ref = GS.power(ptms, rho, E, int(gate[i]), pr, r)
        np.testing.assert_allclose(out[i], ref, atol=1e-12, rtol=0)


def test_power_equals_series_on_device(qs):
    ptms, rho, E, gate, prep = _batch(1, 1400)
    dev = _dev(qs, ptms, rho, E, gate, prep)
    s = qs.gst_series(2, *dev, r_max=300).cpu().numpy()
    for r in (1, 50, 300):
        reps = torch.full((len(gate),), r, dtype=torch.int64, device="cuda")
        p = qs.gst_power(2, *dev, reps).cpu().numpy()
        np.testing.assert_allclose(s[:, r - 1], p, atol=5e-5)


def test_one_qubit_and_ideal_singlet(qs):
    # n = 1: depolarized |0> decays as 1/2 + (1 - 4p/3)^r / 2
    pdep = 0.05
    Gd = D.ptm_kraus(D.depolarizing_kraus(pdep / 3, pdep / 3, pdep / 3))
    rho = D.pauli_vector(np.array([[1, 0], [0, 0]], dtype=complex), 1)
    E = np.array([D.effect_vector(J, 1) for J in range(2)])
    gate = np.zeros(1, dtype=np.int32)
    prep = -np.ones((1, 8), dtype=np.int32)
    s = qs.gst_series(1, *_dev(qs, [Gd], rho, E, gate, prep), r_max=200).cpu().numpy()[0]
    r = np.arange(1, 201)
    np.testing.assert_allclose(s[:, 0], 0.5 + 0.5 * (1 - 4 * pdep / 3) ** r, atol=1e-5)
    # ideal gates: the thesis's |Psi^-> preparation, then repeated II keeps p = (0, 1/2, 1/2, 0)
    ideal = _ideal()
    rho2 = np.zeros((4, 4), dtype=complex)
    rho2[0, 0] = 1
    E2 = np.array([D.effect_vector(J, 2) for J in range(4)])
    prep2 = np.array([PREPS[3] + [-1, -1]], dtype=np.int32)
    s2 = qs.gst_series(2, *_dev(qs, ideal, D.pauli_vector(rho2, 2), E2, np.array([II], np.int32),
                                prep2), r_max=10).cpu().numpy()[0]
    np.testing.assert_allclose(s2, [[0, 0.5, 0.5, 0]] * 10, atol=1e-6)


def test_bad_indices_and_arguments(qs):
    ptms, rho, E, gate, prep = _batch(1, 1500)
    gate[3] = 99              # out of the table
    prep[5][0] = -7           # not an index nor the end mark
    dev = _dev(qs, ptms, rho, E, gate, prep)
    s = qs.gst_series(2, *dev, r_max=5).cpu().numpy()
    assert np.isnan(s[3]).all() and np.isnan(s[5]).all()
    assert np.isfinite(np.delete(s, [3, 5], axis=0)).all()
    reps = torch.full((len(gate),), 4, dtype=torch.int64, device="cuda")
    reps[0] = -1
    p = qs.gst_power(2, *dev, reps).cpu().numpy()
    assert np.isnan(p[[0, 3, 5]]).all() and np.isfinite(np.delete(p, [0, 3, 5], axis=0)).all()
    with pytest.raises(qs.QsimError) as e:
        qs.gst_series(3, *dev, r_max=5)
    assert e.value.status == qs.QS_EINVAL
    with pytest.raises(qs.QsimError) as e:
        qs.gst_series(2, *dev, r_max=0)
    assert e.value.status == qs.QS_EINVAL


def test_validate_flag_rejects_non_channels(qs):
    # QS_DM_VALIDATE: a table that holds a non-channel is refused before any launch,
    # with the failing index named; the same table with only channels runs unchanged
    ptms, rho, E, gate, prep = _batch(1, 1600)
    dev = _dev(qs, ptms, rho, E, gate, prep)
    plain = qs.gst_series(2, *dev, r_max=20).cpu().numpy()
    checked = qs.gst_series(2, *dev, r_max=20, validate=True).cpu().numpy()
    np.testing.assert_array_equal(plain, checked)
    T2 = D.ptm_of_map(lambda P: P.T, 2)                        # positive, not completely positive
    m0 = D.amplitude_damping_kraus(1.0, 0.3)[0]
    lossy = np.kron(D.ptm_kraus([m0]), np.eye(4))              # trace decreasing on one qubit
    for bad, word in ((T2, "completely positive"), (lossy, "trace preserving")):
        table = list(ptms) + [bad]
        devb = _dev(qs, table, rho, E, gate, prep)
        with pytest.raises(qs.QsimError) as e:
            qs.gst_power(2, *devb, torch.ones(len(gate), dtype=torch.int64, device="cuda"),
                         validate=True)
        assert e.value.status == qs.QS_EINVAL and f"ptms {len(ptms)}" in str(e.value)
        assert word in str(e.value)
        qs.gst_series(2, *devb, r_max=2)                          # unchecked: accepted as given
