"""GPU parity of the batched density-matrix / PTM path against the oracle.

The oracle evolves 2^n x 2^n density matrices with Kraus operators (no PTMs),
so these tests also pin the kernel's PTM tables and Pauli-basis readout.

Tolerances, derived from the fp32 Pauli-vector arithmetic: each op rounds
every entry once (unit roundoff 6e-8) and the entries are bounded by
2^{-n/2}, so after L <= 256 ops the outcome probabilities (sums of 2^n
entries times 2^{-n/2}) carry an absolute error below ~L * 2^n * 6e-8 *
2^{-n} ~ 2e-5.  The log-likelihood and gradient are accumulated in fp64 from
fp32 terms: relative 1e-4 on the likelihood, and on the gradient an error
relative to the l1 size of the summed terms (tested against max(|g|, 1)).
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import density as D
from oracle import gates as G
from oracle import noisy as NZ
from oracle import statevector as SV

pytestmark = pytest.mark.gpu


def _with_counts(batch, seed):
    probs, _ = NZ.batch_forward(batch)
    batch.counts = W.multinomial_counts(probs, 1000, seed=seed)
    return batch, probs


def test_probs_loglik_vs_oracle(qs):
    batch = W.noisy_batch(count=48, seed=4001, len_range=(1, 60))
    batch, ref_p = _with_counts(batch, 4002)
    dev = qs.NoisyBatchDevice(batch)
    p, ll, _ = dev.run()
    p = p.cpu().numpy()
    ll = ll.cpu().numpy()
    for c in range(batch.size):
        got = p[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        np.testing.assert_allclose(got, ref_p[c], atol=2e-5)
        cnt = batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        assert ll[c] == pytest.approx(NZ.loglik(ref_p[c], cnt), rel=1e-4)


def test_long_circuits_trace_and_sampled_parity(qs):
    # full-length circuits (up to 256 ops): every distribution sums to 1;
    # a sample of small circuits is checked against the oracle
    batch = W.noisy_batch(count=256, seed=4003)
    dev = qs.NoisyBatchDevice(batch, counts=False)
    p, _, _ = dev.run(loglik=False)
    p = p.cpu().numpy()
    for c in range(batch.size):
        seg = p[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        assert abs(seg.sum() - 1) < 1e-4 and seg.min() > -1e-5
    small = [c for c in range(batch.size) if batch.nq[c] <= 3][:10]
    for c in small:
        n, ops, params = batch.circuit(c)
        ref = NZ.circuit_probabilities(n, ops, params)
        np.testing.assert_allclose(p[batch.cnt_off[c]:batch.cnt_off[c + 1]], ref, atol=2e-5)


def test_gradient_vs_oracle_adjoint_and_fd(qs):
    batch = W.noisy_batch(count=24, seed=4101, n_range=(1, 4), len_range=(1, 40))
    batch, _ = _with_counts(batch, 4102)
    dev = qs.NoisyBatchDevice(batch)
    _, ll, g = dev.run(grad=True)
    g = g.cpu().numpy()
    ll = ll.cpu().numpy()
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        cnt = batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        L, _, ref = NZ.grad_adjoint(n, ops, params, cnt)
        fd = NZ.grad_fd(n, ops, params, cnt)
        np.testing.assert_allclose(ref, fd, rtol=1e-5, atol=1e-3)      # oracle self-consistency
        scale = np.maximum(np.abs(ref), 1.0)
        assert np.all(np.abs(g[c] - ref) / scale < 2e-3), (c, g[c], ref)
        assert ll[c] == pytest.approx(L, rel=1e-4)


def test_gradient_long_circuits_use_checkpoints(qs):
    # L up to 256: sqrt(L) checkpoints and segment recomputation
    batch = W.noisy_batch(count=6, seed=4201, n_range=(2, 3), len_range=(200, 256))
    batch, _ = _with_counts(batch, 4202)
    dev = qs.NoisyBatchDevice(batch)
    _, _, g = dev.run(grad=True)
    g = g.cpu().numpy()
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        cnt = batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        _, _, ref = NZ.grad_adjoint(n, ops, params, cnt)
        scale = np.maximum(np.abs(ref), 1.0)
        assert np.all(np.abs(g[c] - ref) / scale < 5e-3), (c, g[c], ref)


def test_user_ptms_match_unitary_evolution(qs):
    # PTM1 = PTM of H, PTM2 = PTM of CNOT (control = q0), built from the definition
    H = D.ptm_unitary(G.matrix("H"))
    CN = D.ptm_unitary(G.CNOT)
    ptm1 = torch.tensor(H.reshape(1, 16), device="cuda")
    ptm2 = torch.tensor(CN.reshape(1, 256), device="cuda")
    n = 3
    ops = np.array([[4, 2, 0, 0], [5, 2, 1, 0], [5, 1, 0, 0], [4, 0, 0, 0]], dtype=np.int32)
    nq = torch.tensor([n], dtype=torch.int32, device="cuda")
    op_off = torch.tensor([0, len(ops)], dtype=torch.int64, device="cuda")
    out_off = torch.tensor([0, 1 << n], dtype=torch.int64, device="cuda")
    params = torch.tensor([[1.0, 1.0, 1e-3, 1e-3]], dtype=torch.float64, device="cuda")
    probs = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qs.dm_apply_channels(nq, op_off, torch.tensor(ops, device="cuda"), params, out_off,
                         ptm1=ptm1, ptm2=ptm2, probs=probs, max_qubits=n)
    circ = [("H", (2,), (), None), ("CNOT", (2, 1), (), None), ("CNOT", (1, 0), (), None),
            ("H", (0,), (), None)]
    ref = SV.probabilities(SV.apply_circuit(SV.basis(n), n, circ))
    np.testing.assert_allclose(probs.cpu().numpy(), ref, atol=1e-6)


def test_user_ptms_on_small_registers_in_every_orientation(qs):
    # one- and two-qubit registers run one circuit per warp with the Pauli vector in
    # registers: user PTMs on either qubit and both orientations of a two-qubit PTM
    # (local digit order a, b), beside a 3-qubit circuit on a whole CTA
    H = D.ptm_unitary(G.matrix("H"))
    CN = D.ptm_unitary(G.CNOT)
    ptm1 = torch.tensor(H.reshape(1, 16), device="cuda")
    ptm2 = torch.tensor(CN.reshape(1, 256), device="cuda")
    circuits = [
        (2, [[4, 0, 0, 0], [5, 0, 1, 0], [4, 1, 0, 0]], [("H", (0,)), ("CNOT", (0, 1)), ("H", (1,))]),
        (2, [[4, 1, 0, 0], [5, 1, 0, 0], [4, 0, 0, 0], [5, 0, 1, 0]],
         [("H", (1,)), ("CNOT", (1, 0)), ("H", (0,)), ("CNOT", (0, 1))]),
        (1, [[4, 0, 0, 0]], [("H", (0,))]),
        (3, [[4, 2, 0, 0], [5, 2, 0, 0]], [("H", (2,)), ("CNOT", (2, 0))]),
        (2, [], []),
    ]
    nq = torch.tensor([c[0] for c in circuits], dtype=torch.int32, device="cuda")
    lens = [len(c[1]) for c in circuits]
    op_off = torch.tensor(np.concatenate([[0], np.cumsum(lens)]), dtype=torch.int64, device="cuda")
    sizes = [1 << c[0] for c in circuits]
    out_off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int64, device="cuda")
    ops = torch.tensor(np.array([o for c in circuits for o in c[1]], dtype=np.int32), device="cuda")
    params = torch.tensor([[1.0, 1.0, 1e-3, 1e-3]] * len(circuits), dtype=torch.float64, device="cuda")
    probs = torch.empty(sum(sizes), dtype=torch.float32, device="cuda")
    qs.dm_apply_channels(nq, op_off, ops, params, out_off, ptm1=ptm1, ptm2=ptm2, probs=probs, max_qubits=3)
    p = probs.cpu().numpy()
    o = 0
    for n, _, gates in circuits:
        circ = [(g, q, (), None) for g, q in gates]
        ref = SV.probabilities(SV.apply_circuit(SV.basis(n), n, circ))
        np.testing.assert_allclose(p[o:o + (1 << n)], ref, atol=1e-6)
        o += 1 << n


def test_invalid_ops_give_nan_and_do_not_disturb_others(qs):
    batch, _ = _with_counts(W.noisy_batch(count=3, seed=5, n_range=(2, 2), len_range=(3, 3)), 1)
    good = batch.ops.copy()
    batch.ops[batch.op_off[1]] = (0, 7, -1)      # qubit 7 on a 2-qubit circuit
    dev = qs.NoisyBatchDevice(batch)
    p, ll, _ = dev.run()
    p = p.cpu().numpy()
    ll = ll.cpu().numpy()
    assert np.isnan(ll[1]) and np.all(np.isnan(p[batch.cnt_off[1]:batch.cnt_off[2]]))
    batch.ops = good
    for c in (0, 2):
        n, ops, params = batch.circuit(c)
        np.testing.assert_allclose(p[batch.cnt_off[c]:batch.cnt_off[c + 1]],
                                   NZ.circuit_probabilities(n, ops, params), atol=1e-6)


def test_empty_and_single_qubit_circuits(qs):
    batch = W.noisy_batch(count=5, seed=8, n_range=(1, 1), len_range=(1, 5))
    # make circuit 0 empty
    lens = np.diff(batch.op_off)
    lens[0] = 0
    ops = np.concatenate([batch.ops[batch.op_off[c]:batch.op_off[c] + lens[c]] for c in range(5)])
    batch.ops = ops
    batch.op_off = np.concatenate([[0], np.cumsum(lens)])
    dev = qs.NoisyBatchDevice(batch, counts=False)
    p, _, _ = dev.run(loglik=False)
    p = p.cpu().numpy()
    np.testing.assert_allclose(p[0:2], [1, 0], atol=1e-7)
    for c in range(1, 5):
        n, o, params = batch.circuit(c)
        np.testing.assert_allclose(p[batch.cnt_off[c]:batch.cnt_off[c + 1]],
                                   NZ.circuit_probabilities(n, o, params), atol=1e-6)


def test_full_batch_4096_properties(qs):
    batch = W.noisy_batch(count=4096, seed=4001)
    batch.counts = W.synthetic_counts(batch, 1000, seed=4002)
    dev = qs.NoisyBatchDevice(batch)
    p, ll, g = dev.run(grad=True)
    p = p.cpu().numpy()
    sums = np.add.reduceat(p, batch.cnt_off[:-1])
    assert np.all(np.abs(sums - 1) < 1e-4)
    assert np.all(np.isfinite(ll.cpu().numpy())) and np.all(np.isfinite(g.cpu().numpy()))
    # sampled circuits against the oracle: two of every register size, from the
    # gradient pass (one circuit per warp up to 4 qubits, per CTA above) and from the
    # forward pass (one per warp in registers for 1-2 qubits, per CTA above)
    p_fwd = dev.run()[0].cpu().numpy()
    rng = np.random.default_rng(0)
    for nq in range(1, 7):
        for c in rng.choice(np.where(batch.nq == nq)[0], size=2, replace=False):
            n, ops, params = batch.circuit(int(c))
            ref = NZ.circuit_probabilities(n, ops, params)
            np.testing.assert_allclose(p[batch.cnt_off[c]:batch.cnt_off[c + 1]], ref, atol=2e-5)
            np.testing.assert_allclose(p_fwd[batch.cnt_off[c]:batch.cnt_off[c + 1]], ref, atol=2e-5)


def test_gradient_is_reproducible(qs):
    # one circuit's arithmetic does not depend on which CTA runs it or when: three
    # runs of the full batch (circuits handed out by an atomic counter, so the
    # assignment changes) give bit-identical gradients.  A missing barrier between
    # the sub-op state copies and the next sub-op showed up here as ~1e-4 jitter.
    batch = W.noisy_batch(count=4096, seed=4001)
    batch.counts = W.synthetic_counts(batch, 1000, seed=4002)
    dev = qs.NoisyBatchDevice(batch)
    runs = [tuple(x.cpu().numpy().copy() for x in dev.run(grad=True)) for _ in range(3)]
    for p, ll, g in runs[1:]:
        assert np.array_equal(p, runs[0][0])
        assert np.array_equal(ll, runs[0][1])
        assert np.array_equal(g, runs[0][2])


def test_batch_beyond_the_sort_limit(qs):
    # more circuits than the one-CTA sort takes (16384): the gradient pass hands
    # them out through the stable partition too (small registers one per warp); a
    # sample of circuits against the oracle, the gradients against the oracle's
    # adjoint within their derived FP32 bound
    batch = W.noisy_batch(count=20000, seed=4501, n_range=(1, 4), len_range=(1, 24))
    batch.counts = W.synthetic_counts(batch, 1000, seed=4502)
    dev = qs.NoisyBatchDevice(batch)
    p, ll, g = dev.run(grad=True)
    p, ll, g = p.cpu().numpy(), ll.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    p_fwd, ll_fwd, _ = dev.run()
    np.testing.assert_allclose(p_fwd.cpu().numpy(), p, atol=1e-6)   # the forward pass agrees
    for c in W.rng(4503).choice(batch.size, size=6, replace=False):
        c = int(c)
        n, ops, params = batch.circuit(c)
        cnt = batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        np.testing.assert_allclose(p[batch.cnt_off[c]:batch.cnt_off[c + 1]],
                                   NZ.circuit_probabilities(n, ops, params), atol=2e-5)
        _, _, ref = NZ.grad_adjoint(n, ops, params, cnt)
        assert np.all(np.abs(g[c] - ref) <= _gradient_bound(n, ops, params, cnt)), (c, g[c], ref)


def test_long_circuits_five_and_six_qubits_vs_oracle(qs):
    # the largest registers at full length (L = 200..256): every outcome against the
    # Kraus-map oracle, within the fp32 bound L * u ~ 1.5e-5 of the docstring
    batch = W.noisy_batch(count=12, seed=4301, n_range=(5, 6), len_range=(200, 256))
    dev = qs.NoisyBatchDevice(batch, counts=False)
    p, _, _ = dev.run(loglik=False)
    p = p.cpu().numpy()
    assert set(int(x) for x in batch.nq) == {5, 6}
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        assert len(ops) >= 200
        ref = NZ.circuit_probabilities(n, ops, params)
        np.testing.assert_allclose(p[batch.cnt_off[c]:batch.cnt_off[c + 1]], ref, atol=2e-5)


def _gradient_bound(n, ops, params, counts, h=1e-6):
    """Error bound of the fp32 gradient from its arithmetic.

    g_k = sum_J n_J (d p_J / d t_k) / p_J.  The fp32 Pauli-vector sweeps leave an
    absolute error of at most eps = L u (u = 2^-24, L ops) on each p_J and on each
    d p_J / d t_k, so to first order
        |g_k - g_k,exact| <= eps sum_J n_J (1 + |d p_J / d t_k| / p_J) / p_J.
    The derivatives come from central differences of the oracle's probabilities."""
    eps = len(ops) * 2.0 ** -24
    p0 = NZ.circuit_probabilities(n, ops, params)
    bound = np.zeros(4)
    m = counts > 0
    for k in range(4):
        pp = np.array(params, dtype=np.float64)
        pm = pp.copy()
        pp[k] += h
        pm[k] -= h
        dp = (NZ.circuit_probabilities(n, ops, pp) - NZ.circuit_probabilities(n, ops, pm)) / (2 * h)
        bound[k] = eps * np.sum(counts[m] * (1 + np.abs(dp[m]) / p0[m]) / p0[m])
    return bound


def test_gradient_within_derived_bound_large_registers(qs):
    # n = 5..6 and L = 200..256 (checkpointed sweeps): the gradient against the
    # oracle's adjoint within the first-order bound of its fp32 arithmetic
    batch = W.noisy_batch(count=4, seed=4401, n_range=(5, 6), len_range=(200, 256))
    batch, _ = _with_counts(batch, 4402)
    dev = qs.NoisyBatchDevice(batch)
    _, ll, g = dev.run(grad=True)
    g = g.cpu().numpy()
    ll = ll.cpu().numpy()
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        cnt = batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        L, _, ref = NZ.grad_adjoint(n, ops, params, cnt)
        bound = _gradient_bound(n, ops, params, cnt)
        assert np.all(np.abs(g[c] - ref) <= bound), (c, g[c], ref, bound)
        assert ll[c] == pytest.approx(L, rel=1e-4)


def test_gradient_within_derived_bound_small_registers(qs):
    batch = W.noisy_batch(count=16, seed=4111, n_range=(1, 4), len_range=(1, 120))
    batch, _ = _with_counts(batch, 4112)
    dev = qs.NoisyBatchDevice(batch)
    _, _, g = dev.run(grad=True)
    g = g.cpu().numpy()
    for c in range(batch.size):
        n, ops, params = batch.circuit(c)
        cnt = batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]]
        _, _, ref = NZ.grad_adjoint(n, ops, params, cnt)
        bound = _gradient_bound(n, ops, params, cnt)
        assert np.all(np.abs(g[c] - ref) <= bound), (c, g[c], ref, bound)


def test_validate_flag(qs):
    # QS_DM_VALIDATE: user PTMs must be channels and p, gamma in [0, 1]; a failure
    # names the index and launches nothing (the output buffer keeps its fill value)
    n = 2
    good1 = D.ptm_unitary(G.matrix("H"))
    good2 = D.ptm_unitary(G.CNOT)
    T = D.ptm_of_map(lambda P: P.T, 1)
    ops = torch.tensor(np.array([[4, 0, 0, 0], [5, 1, 0, 0], [4, 1, 0, 1]], dtype=np.int32), device="cuda")
    nq = torch.tensor([n], dtype=torch.int32, device="cuda")
    op_off = torch.tensor([0, 3], dtype=torch.int64, device="cuda")
    out_off = torch.tensor([0, 1 << n], dtype=torch.int64, device="cuda")
    params = torch.tensor([[1.0, 1.0, 1e-3, 1e-3]], dtype=torch.float64, device="cuda")
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")  # noqa: E731

    def run(ptm1, par, validate):
        probs = torch.full((1 << n,), -7.0, dtype=torch.float32, device="cuda")
        qs.dm_apply_channels(nq, op_off, ops, par, out_off, ptm1=t(ptm1), ptm2=t(good2.reshape(1, 256)),
                             probs=probs, max_qubits=n, validate=validate)
        return probs.cpu().numpy()

    ok = np.stack([good1, good1]).reshape(2, 16)
    np.testing.assert_array_equal(run(ok, params, True), run(ok, params, False))
    bad = np.stack([good1, T]).reshape(2, 16)
    with pytest.raises(qs.QsimError) as e:
        run(bad, params, True)
    assert e.value.status == qs.QS_EINVAL and "ptm1 1" in str(e.value)
    assert "completely positive" in str(e.value)
    assert np.all(run(bad, params, False) != -7.0)           # unchecked: used as given
    bad_p = params.clone()
    bad_p[0, 2] = 1.5
    with pytest.raises(qs.QsimError) as e:
        run(ok, bad_p, True)
    assert "circuit 0" in str(e.value)
