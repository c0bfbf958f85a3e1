"""GPU [[4,2,2]] evaluation: 465 synthetic logical circuits (155 sequences x the
three initial states) in bare and encoded versions through the batched
density-matrix kernel (gates with their noise composed into user PTMs), then
postselection and D_bare/enc on the device, against the oracle's Kraus-map
density matrices.

Tolerance: the DM kernel's probabilities carry <= 2e-5 absolute error (FP32
Pauli vectors, <= ~60 ops); the distributions and distances built from <= 32 of
them: 1e-4 absolute.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import code422 as C
from oracle import density as D
from oracle import gates as G

pytestmark = pytest.mark.gpu

ONE = ["X", "Z", "H", "S"]


def _tables(p, gamma):
    N1 = D.ptm_kraus(D.amplitude_damping_kraus(1.0, gamma)) @ D.ptm_kraus(
        D.depolarizing_kraus(p / 3, p / 3, p / 3))
    ptm1 = [N1 @ D.ptm_unitary(G.matrix(g)) for g in ONE]
    ptm2 = [np.kron(N1, N1) @ D.ptm_unitary(G.matrix("CNOT"))]
    return np.stack(ptm1), np.stack(ptm2)


def _ops(circ, qubit_map):
    rows = []
    for name, qs in circ:
        if name == "CNOT":
            rows.append([5, qubit_map[qs[0]], qubit_map[qs[1]], 0])
        else:
            rows.append([4, qubit_map[qs[0]], 0, ONE.index(name)])
    return rows


def _run(qs, circuits, n, qubit_map, ptm1, ptm2):
    ops, off, nq, oo = [], [0], [], [0]
    for circ in circuits:
        ops += _ops(circ, qubit_map)
        off.append(len(ops))
        nq.append(n)
        oo.append(oo[-1] + (1 << n))
    t = lambda a, dt: torch.tensor(np.asarray(a), dtype=dt, device="cuda")  # noqa: E731
    probs = torch.empty(oo[-1], dtype=torch.float32, device="cuda")
    qs.dm_apply_channels(t(nq, torch.int32), t(off, torch.int64), t(ops, torch.int32).reshape(-1, 4),
                         torch.zeros(4 * len(circuits), dtype=torch.float64, device="cuda"),
                         t(oo, torch.int64), ptm1=t(ptm1, torch.float64), ptm2=t(ptm2, torch.float64),
                         probs=probs, max_qubits=n)
    return probs.reshape(len(circuits), 1 << n)


@pytest.mark.parametrize("p,gamma", [(0.0, 0.0), (0.02, 0.01)])
def test_code422_against_oracle(qs, p, gamma):
    circuits = W.code422_sequences(155, seed=4220)
    enc_c = [C.physical(s, q, True) for s, q in circuits]
    bare_c = [C.physical(s, q, False) for s, q in circuits]
    ptm1, ptm2 = _tables(p, gamma)
    ptm1_id, ptm2_id = _tables(0.0, 0.0)
    enc = _run(qs, enc_c, 5, {b: b for b in range(5)}, ptm1, ptm2)
    bare = _run(qs, bare_c, 2, {3: 1, 4: 0}, ptm1, ptm2)          # J = 2 q3 + q4
    ideal = _run(qs, bare_c, 2, {3: 1, 4: 0}, ptm1_id, ptm2_id)
    p_enc, ratio, d_bare, d_enc = (x.cpu().numpy() for x in qs.code422_eval(enc, bare, ideal))
    assert len(circuits) == 465
    for c in range(0, 465, 7):       # every 7th circuit: 67 of them through the oracle
        s, q = circuits[c]
        r_id, r_bare, r_enc, r_ratio, r_db, r_de = C.evaluate(s, q, p=p, gamma=gamma)
        np.testing.assert_allclose(p_enc[c], r_enc, atol=1e-4)
        assert ratio[c] == pytest.approx(r_ratio, abs=1e-4)
        assert d_bare[c] == pytest.approx(r_db, abs=1e-4)
        assert d_enc[c] == pytest.approx(r_de, abs=1e-4)
    if p == 0.0:
        np.testing.assert_allclose(ratio, 1.0, atol=1e-5)
        np.testing.assert_allclose(d_enc, 0.0, atol=1e-5)
        np.testing.assert_allclose(d_bare, 0.0, atol=1e-5)


def test_code422_eval_masks(qs):
    # hand-made outcome vectors: only codewords with q0 = 0 count
    enc = np.zeros((3, 32), dtype=np.float32)
    enc[0, 0] = enc[0, 30] = 0.5                    # 0000 and 1111 (q1..q4): logical 00
    enc[1, 0b00110] = 0.25                          # q1 q2 = 11: logical 01, kept
    enc[1, 0b00111] = 0.25                          # same data word, ancilla set: discarded
    enc[1, 0b00010] = 0.5                           # q1 alone: odd parity, discarded
    enc[2, 1] = 1.0                                 # ancilla only: nothing kept
    ideal = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0.25] * 4], dtype=np.float32)
    bare = np.array([[0.5, 0.5, 0, 0], [0, 1, 0, 0], [1, 0, 0, 0]], dtype=np.float32)
    t = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    p_enc, ratio, d_bare, d_enc = (x.cpu().numpy() for x in qs.code422_eval(t(enc), t(bare), t(ideal)))
    np.testing.assert_allclose(p_enc, [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 0]], atol=1e-7)
    np.testing.assert_allclose(ratio, [1.0, 0.25, 0.0], atol=1e-7)
    np.testing.assert_allclose(d_bare, [0.5, 0.0, 0.75], atol=1e-7)
    np.testing.assert_allclose(d_enc, [0.0, 0.0, 0.5], atol=1e-7)
