"""Serving loop (continuous batching): results alone vs in the mix, admission by memory.

Tolerance: the packed small-circuit kernel and the tiled pipeline are both
complex64 with fp64 marginal accumulation, so a marginal equals the oracle's
to 2e-6 absolute and the same circuit alone vs in the mix to 1e-6 (the same
kernels run on the same inputs; only scheduling differs).
"""
import time

import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV

pytestmark = pytest.mark.gpu


def _mask(n):
    return (1 << min(n, 10)) - 1


def _oracle_marginal(n, ops):
    p = SV.probabilities(SV.apply_circuit(SV.basis(n), n, ops))
    return SV.marginal(p, n, _mask(n))


def test_mix_equals_alone_and_oracle(qs):
    rng = np.random.default_rng(5)
    specs = [(int(n), int(d)) for n, d in zip(rng.choice([6, 9, 12, 14, 15, 17, 19], size=24),
                                               rng.integers(3, 25, size=24))]
    circuits = [W.layered_haar_cz(n, d, seed=100 + i) for i, (n, d) in enumerate(specs)]
    srv = qs.Server(max_inflight=3)
    tickets = []
    for (n, _), ops in zip(specs, circuits):
        tickets.append(srv.submit(n, ops, _mask(n)))
        time.sleep(float(rng.exponential(0.002)))      # Poisson arrivals while others run
    mixed = [srv.wait(t) for t in tickets]
    st = srv.stats()
    assert st["completed"] == st["submitted"] == 24
    assert st["packed_launches"] >= 1 and st["large_circuits"] >= 1
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    # each circuit alone on a fresh server
    for (n, _), ops, (res, lat) in zip(specs, circuits, mixed):
        alone = qs.Server(max_inflight=1)
        r2, _ = alone.wait(alone.submit(n, ops, _mask(n)))
        alone.close()
        np.testing.assert_allclose(res, r2, atol=1e-6)
        np.testing.assert_allclose(res, _oracle_marginal(n, ops), atol=2e-6)
        assert lat > 0
    srv.close()


def test_admission_by_memory(qs):
    # budget for one 20-qubit complex64 state (8 MiB + scratch) but not two
    budget = (8 << 20) + (1 << 20) + (4 << 20) + (6 << 20)
    srv = qs.Server(max_inflight=4, mem_budget=budget)
    ops = [W.layered_haar_cz(20, 6, seed=s) for s in range(3)]
    tickets = [srv.submit(20, o, _mask(20)) for o in ops]
    for t, o in zip(tickets, ops):
        res, _ = srv.wait(t)
        np.testing.assert_allclose(res, _oracle_marginal(20, o), atol=2e-6)
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    # a circuit that can never fit is rejected, not hung
    t = srv.submit(24, W.layered_haar_cz(24, 1, seed=1), _mask(24))
    with pytest.raises(qs.QsimError) as e:
        srv.wait(t)
    assert e.value.status == qs.QS_ENOMEM
    srv.close()


@pytest.mark.parametrize("n", [8, 12])
def test_failed_completion_query_returns_error(qs, n):
    # a completion query of the persistent packed kernel that reports an error
    # (injected on the host: no device fault) ends the queued circuits' waits with
    # QS_ECUDA; the queue starts over and the server keeps serving.  The failing
    # circuit is deep (milliseconds in the kernel), so the scheduler's first
    # completion query comes while its job still runs: a short job could finish
    # and be retired before that query.
    srv = qs.Server(max_inflight=2)
    ops = W.layered_haar_cz(n, 4, seed=n)
    qs.server_inject_query_error(srv, 999)   # cudaErrorUnknown
    t = srv.submit(n, W.layered_haar_cz(n, 100, seed=n + 1), _mask(n))
    with pytest.raises(qs.QsimError) as e:
        srv.wait(t)
    assert e.value.status == qs.QS_ECUDA
    res, _ = srv.wait(srv.submit(n, ops, _mask(n)))
    np.testing.assert_allclose(res, _oracle_marginal(n, ops), atol=2e-6)
    assert srv.stats()["completed"] == 2
    srv.close()


def test_idle_limit_ends_the_persistent_kernel(qs):
    # no producer: the packed kernel's bounded wait runs out (a host-side stall of
    # 60 ms against a 2 ms limit), the kernel ends reporting QS_ETIMEOUT (counted),
    # and the next circuit launches it again
    srv = qs.Server(idle_ms=2)
    ops = W.layered_haar_cz(9, 5, seed=3)
    res, _ = srv.wait(srv.submit(9, ops, _mask(9)))
    time.sleep(0.06)
    st = srv.stats()
    assert st["idle_timeouts"] >= 1 and st["packed_launches"] == 1
    res2, _ = srv.wait(srv.submit(9, ops, _mask(9)))
    np.testing.assert_array_equal(res, res2)
    np.testing.assert_allclose(res, _oracle_marginal(9, ops), atol=2e-6)
    assert srv.stats()["packed_launches"] == 2
    srv.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_thousand_small_circuits_through_the_queue(qs, prec):
    # 1200 circuits of 6..12 qubits submitted as fast as the host can: every one
    # completes; a sample equals the oracle (complex128: 1e-12; complex64: 2e-6)
    rng = np.random.default_rng(11 + prec)
    count = 1200
    specs = [(int(n), int(d)) for n, d in zip(rng.integers(6, 13, size=count), rng.integers(2, 12, size=count))]
    circuits = [qs.gates_array(W.layered_haar_cz(n, d, seed=2000 + i)) for i, (n, d) in enumerate(specs)]
    srv = qs.Server(prec=prec, small_max_qubits=12)
    tickets = [srv.submit(n, c, _mask(n)) for (n, _), c in zip(specs, circuits)]
    results = [srv.wait(t)[0] for t in tickets]
    st = srv.stats()
    assert st["completed"] == count and st["packed_circuits"] == count and st["large_circuits"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    tol = 1e-12 if prec else 2e-6
    for i in rng.choice(count, size=12, replace=False):
        n, d = specs[i]
        ops = W.layered_haar_cz(n, d, seed=2000 + int(i))
        np.testing.assert_allclose(results[i], _oracle_marginal(n, ops), atol=tol)
    srv.close()
