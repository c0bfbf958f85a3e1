"""GPU parity of the state-vector path (C ABI via the binding) against the oracle.

Tolerances (from the stated targets): complex128 <= 1e-12 max |a - a_ref|;
complex64 relative L2 ||a - a_ref|| / ||a_ref|| <= 1e-5 (depth <= 40), plus
1e-6 absolute on probabilities.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def run(qs, n, ops, prec, method=0, J=0, psi0=None):
    st = qs.State(n, prec)
    if psi0 is not None:
        qs.sv_copy_in(st, psi0)
    elif J:
        qs.sv_set_basis(st, J)
    stats = qs.sv_apply_circuit(st, ops, method)
    out = qs.sv_copy_out(st)
    st.close()
    return out, stats


def check(out, ref, prec):
    if prec == 1:
        assert np.max(np.abs(out - ref)) <= TOL64, np.max(np.abs(out - ref))
    else:
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= TOL32, err


ALL1 = ["I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "PX", "MX", "PY", "MY", "RX", "RY", "RZ",
        "U1", "U2", "U3", "RK", "MAT1"]
ALL2 = ["CNOT", "CZ", "CP", "SWAP", "MAT2"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_small_all_gates(qs, n, prec):
    ops = W.random_gate_mix(n, 120, seed=10 * n + prec)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, _ = run(qs, n, ops, prec)
    check(out, ref, prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [12, 13, 15, 17])
def test_tiled_all_gates(qs, n, prec):
    ops = W.random_gate_mix(n, 300, seed=1000 + n)
    g = W.rng(n)
    psi0 = W.random_state(n, g)
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out, stats = run(qs, n, ops, prec, psi0=psi0.astype(np.complex64 if prec == 0 else np.complex128))
    if prec == 0:
        ref = SV.apply_circuit(psi0.astype(np.complex64).astype(np.complex128), n, ops)
    check(out, ref, prec)
    assert stats["passes"] >= 1


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [12, 13, 16])
def test_tiled_diagonal_runs(qs, n, prec):
    # long runs of commuting diagonals (CZ, CP, RZ, S, T, U1, R(k)) on register,
    # lane, warp and tile-constant bits, broken up by a few H gates
    ops = W.random_gate_mix(n, 500, seed=3000 + n, two_q_fraction=0.6,
                            names1=["RZ", "S", "T", "TDG", "U1", "RK", "Z", "H"],
                            names2=["CZ", "CP"])
    g = W.rng(n + 17)
    psi0 = W.random_state(n, g)
    if prec == 0:
        psi0 = psi0.astype(np.complex64)
    ref = SV.apply_circuit(psi0.astype(np.complex128), n, ops)
    out, _ = run(qs, n, ops, prec, psi0=psi0)
    check(out, ref, prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [12, 13, 16])
def test_tiled_dense_two_qubit_ops(qs, n, prec):
    # dense 4x4 ops (random SU(4), SWAP without relabeling via MAT2) inside tile passes:
    # both qubits in registers, one on a lane and one in a register (either order),
    # or both on lanes
    g = W.rng(4000 + n)
    ops = []
    for i in range(160):
        a, b = (int(x) for x in g.choice(n, size=2, replace=False))
        if i % 3 == 2:
            ops.append(("MAT1", (a,), (), W.haar_su2(g)))
            continue
        z = g.normal(size=(4, 4)) + 1j * g.normal(size=(4, 4))
        qm, r = np.linalg.qr(z)
        ops.append(("MAT2", (a, b), (), qm * (np.diag(r) / np.abs(np.diag(r)))))
    psi0 = W.random_state(n, g)
    if prec == 0:
        psi0 = psi0.astype(np.complex64)
    ref = SV.apply_circuit(psi0.astype(np.complex128), n, ops)
    out, stats = run(qs, n, ops, prec, psi0=psi0)
    check(out, ref, prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [3, 12, 16])
def test_plain_method(qs, n, prec):
    ops = W.random_gate_mix(n, 80, seed=77 + n)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, stats = run(qs, n, ops, prec, method=1)
    check(out, ref, prec)
    assert stats["launches"] == len(ops)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [12, 14, 18, 20])
def test_layered_haar_cz(qs, n, prec):
    depth = 40 if n <= 18 else 20
    ops = W.layered_haar_cz(n, depth, seed=2001 + n)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, stats = run(qs, n, ops, prec)
    check(out, ref, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_layered_haar_cnot_n10(qs, prec):
    # 10-qubit, 20-layer Haar + random CNOT matching, all 1024 probabilities
    n = 10
    ops = W.layered_haar_cnot(n, 20, seed=1001)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, _ = run(qs, n, ops, prec)
    check(out, ref, prec)
    st = qs.State(n, prec)
    qs.sv_apply_circuit(st, ops)
    p, norm = qs.sv_probs(st, fp64=True)
    np.testing.assert_allclose(p.cpu().numpy(), SV.probabilities(ref), atol=1e-12 if prec else 1e-6)
    assert abs(norm - 1) < (1e-12 if prec else 1e-5)
    st.close()


@pytest.mark.parametrize("n", [12, 13, 16])
def test_layered_haar_cnot_tiled(qs, n):
    ops = W.layered_haar_cnot(n, 12, seed=n)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    out, _ = run(qs, n, ops, 1)
    check(out, ref, 1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [4, 12, 14, 17])
def test_qft_closed_form(qs, n, prec):
    ops = W.qft_circuit(n)
    J = W.random_basis_index(n, 2002 + n)
    out, _ = run(qs, n, ops, prec, J=J)
    check(out, SV.qft_amplitudes(n, J), prec)


@pytest.mark.parametrize("n", [2, 12, 19])
def test_ghz(qs, n):
    out, _ = run(qs, n, W.ghz_circuit(n), 1)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(out - ref)) <= TOL64


def test_singlet_distribution(qs):
    for t0, t1 in [(0.3, 1.9), (-2.0, 0.5)]:
        st = qs.State(2, 1)
        qs.sv_apply_circuit(st, W.singlet_circuit(t0, t1))
        p, norm = qs.sv_probs(st, fp64=True)
        p = p.cpu().numpy()
        for J in range(4):
            assert abs(p[J] - (1 - (-1) ** ((J >> 1) + (J & 1)) * math.cos(t1 - t0)) / 4) < 1e-14
        st.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [6, 13])
def test_probs_marginal_norm(qs, n, prec):
    ops = W.random_gate_mix(n, 60, seed=5 + n)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    st = qs.State(n, prec)
    qs.sv_apply_circuit(st, ops)
    tol = 1e-13 if prec else 2e-6
    for fp64 in (False, True):
        p, norm = qs.sv_probs(st, fp64=fp64)
        np.testing.assert_allclose(p.cpu().numpy(), SV.probabilities(ref), atol=tol)
        assert abs(norm - 1) < (1e-12 if prec else 1e-5)
    for mask in (0b1, 0b101, (1 << n) - 2, 1 << (n - 1)):
        m, _ = qs.sv_probs(st, fp64=True, marg_mask=mask)
        np.testing.assert_allclose(m.cpu().numpy(), SV.marginal(SV.probabilities(ref), n, mask),
                                   atol=tol * 4)
    st.close()


def test_loglik(qs):
    import torch
    n = 8
    ops = W.random_gate_mix(n, 50, seed=3)
    ref = SV.apply_circuit(SV.basis(n), n, ops)
    p = SV.probabilities(ref)
    counts = W.multinomial_counts([p], 1000, seed=1)
    st = qs.State(n, 1)
    qs.sv_apply_circuit(st, ops)
    ll, clamped = qs.sv_loglik(st, torch.tensor(counts.astype(np.int32), device="cuda"))
    m = counts > 0
    assert ll == pytest.approx(float(np.sum(counts[m] * np.log(p[m]))), rel=1e-12)
    assert clamped == 0
    st.close()


def test_u_udagger_identity_and_edge_cases(qs):
    n = 16
    ops = W.layered_haar_cz(n, 10, seed=9)
    out, _ = run(qs, n, ops + W.inverse_circuit(ops), 1)
    ref = SV.basis(n)
    assert np.max(np.abs(out - ref)) <= TOL64
    # empty circuit leaves the state alone; highest basis index
    out, stats = run(qs, 13, [], 1, J=(1 << 13) - 1)
    assert out[-1] == 1 and np.count_nonzero(out) == 1 and stats["passes"] == 0


def test_invalid_arguments(qs):
    st = qs.State(4, 0)
    before = qs.sv_copy_out(st)
    for bad in ([("H", (4,), (), None)], [("CNOT", (1, 1), (), None)],
                [("RX", (0,), (float("nan"),), None)]):
        with pytest.raises(qs.QsimError) as e:
            qs.sv_apply_circuit(st, bad)
        assert e.value.status == qs.QS_EINVAL
    with pytest.raises(qs.QsimError):
        qs.sv_set_basis(st, 16)
    np.testing.assert_array_equal(qs.sv_copy_out(st), before)
    st.close()
    with pytest.raises(qs.QsimError) as e:
        qs.State(0)
    assert e.value.status == qs.QS_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
def test_probs_to_host_buffer(qs, prec):
    # sv_probs_host: the same values as sv_probs, delivered into host memory
    import torch
    n = 14
    st = qs.State(n, prec)
    ops = W.random_gate_mix(n, 60, seed=321)
    qs.sv_apply_circuit(st, ops)
    ref = SV.probabilities(SV.apply_circuit(SV.basis(n), n, ops))
    for fp64 in (False, True):
        dev, dnorm = qs.sv_probs(st, fp64=fp64)
        host, norm = qs.sv_probs_host(st, fp64=fp64, want_norm=True)
        np.testing.assert_array_equal(host, dev.cpu().numpy())
        assert norm == dnorm
        np.testing.assert_allclose(host, ref, atol=1e-12 if (prec and fp64) else 2e-6)
    pinned = torch.empty(1 << n, dtype=torch.float32, pin_memory=True)
    qs.sv_probs_host(st, out=pinned)
    np.testing.assert_allclose(pinned.numpy(), ref, atol=2e-6)
    mask = 0b1010110
    m, _ = qs.sv_probs_host(st, fp64=True, marg_mask=mask)
    np.testing.assert_allclose(m, SV.marginal(ref, n, mask), atol=1e-12 if prec else 2e-6)
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_probs_to_host_without_waiting(qs, prec):
    # sv_probs_host_async: three distributions queued back to back while the state
    # changes after each call (the third call reuses the first device buffer, so the
    # state's stream waits for the first copy); after sv_probs_wait every host buffer
    # holds its own step's values, equal to sv_probs bit for bit.  Then pageable
    # memory, and an fp64 call after fp32 ones (larger buffers)
    import torch
    n = 16
    st = qs.State(n, prec)
    steps = [W.random_gate_mix(n, 50, seed=700 + i) for i in range(3)]
    bufs = [torch.full((1 << n,), -1.0, dtype=torch.float32, pin_memory=True) for _ in steps]
    refs = []
    for ops, buf in zip(steps, bufs):
        qs.sv_apply_circuit(st, ops)
        refs.append(qs.sv_probs(st, want_norm=False)[0])   # device values, no synchronisation
        qs.sv_probs_host_async(st, buf)
    qs.sv_probs_wait(st)
    for ref, buf in zip(refs, bufs):
        np.testing.assert_array_equal(buf.numpy(), ref.cpu().numpy())
    psi = SV.basis(n)
    for ops in steps:
        psi = SV.apply_circuit(psi, n, ops)
    np.testing.assert_allclose(bufs[2].numpy(), SV.probabilities(psi), atol=2e-6)
    page = np.full(1 << n, -1.0, dtype=np.float32)
    qs.sv_probs_host_async(st, page)
    qs.sv_probs_wait(st)
    np.testing.assert_array_equal(page, refs[2].cpu().numpy())
    p64 = torch.empty(1 << n, dtype=torch.float64, pin_memory=True)
    qs.sv_probs_host_async(st, p64, fp64=True)
    qs.sv_set_basis(st, 5)
    qs.sv_probs_wait(st)
    np.testing.assert_allclose(p64.numpy(), SV.probabilities(psi), atol=1e-12 if prec else 2e-6)
    st.close()


def test_alu_peak_microbenchmark(qs):
    # the measured FP32 / FP64 peaks used as roofline denominators: plausible and
    # consistent with the device's SM count (FP32 at most 128 FMA lanes per SM at 2.1 GHz)
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = qs.alu_peak(0)
    f64 = qs.alu_peak(1)
    assert f32["sm_count"] == sms
    bound32 = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * bound32 < f32["tflops"] <= bound32, f32
    assert 0 < f64["tflops"] < f32["tflops"], (f64, f32)
