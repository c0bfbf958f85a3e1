"""GPU adjoint gradient (sv_grad, autograd wrapper) vs the oracle's adjoint and FD.

Tolerance: the fp64 path matches the oracle to 1e-9 absolute; the complex64
path carries fp32 rounding in every state (relative 1e-6 per gate over <= 200
gates) and fp64 reductions, so gradients are compared with 2e-4 relative to
max(|g|, 1).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import gradient as GR
from oracle import statevector as SV

pytestmark = pytest.mark.gpu

NAMES1 = ["RX", "RY", "RZ", "U1", "U2", "U3", "H", "MAT1", "S", "T"]
NAMES2 = ["CNOT", "CZ", "CP", "SWAP"]


def _circ(n, count, seed):
    return W.random_gate_mix(n, count, seed, names1=NAMES1, names2=NAMES2)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,ckpt", [(3, 0), (6, 0), (12, 0), (13, 5), (6, 7)])
def test_sv_grad_weights(qs, n, prec, ckpt):
    ops = _circ(n, 60, 500 + n)
    w = W.rng(n).normal(size=1 << n)
    Lref, gref = GR.grad_adjoint(ops, n, weights=w)
    st = qs.State(n, prec)
    L, g = qs.sv_grad(st, ops, torch.tensor(w, device="cuda"), mode=0, checkpoint_every=ckpt)
    tol = 1e-9 if prec else 2e-4
    scale = np.maximum(np.abs(gref), 1.0)
    assert np.all(np.abs(g - gref) / scale < tol), np.max(np.abs(g - gref) / scale)
    assert abs(L - Lref) < (1e-10 if prec else 1e-4)
    # the state is restored to psi_0 = |0...0>
    out = qs.sv_copy_out(st)
    assert abs(out[0] - 1) < 1e-6 and np.sum(np.abs(out[1:])) < 1e-5
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,count,ckpt", [(14, 160, 0), (16, 220, 0), (16, 220, 50)])
def test_sv_grad_fused_passes(qs, n, count, prec, ckpt):
    # several fused backward tile passes (and checkpoint segments), every gate kind
    ops = _circ(n, count, 700 + n + ckpt)
    w = W.rng(n + 1).normal(size=1 << n)
    Lref, gref = GR.grad_adjoint(ops, n, weights=w)
    st = qs.State(n, prec)
    L, g = qs.sv_grad(st, ops, torch.tensor(w, device="cuda"), mode=0, checkpoint_every=ckpt)
    st.close()
    tol = 1e-9 if prec else 2e-4
    scale = np.maximum(np.abs(gref), 1.0)
    assert np.all(np.abs(g - gref) / scale < tol), np.max(np.abs(g - gref) / scale)
    assert abs(L - Lref) < (1e-10 if prec else 1e-4)


@pytest.mark.parametrize("prec", [0, 1])
def test_sv_grad_loglik_vs_fd(qs, prec):
    n = 5
    ops = _circ(n, 40, 77)
    p = SV.probabilities(SV.apply_circuit(SV.basis(n), n, ops))
    counts = W.multinomial_counts([p], 1000, seed=3).astype(np.float64)
    Lref, gref = GR.grad_adjoint(ops, n, counts=counts)
    fd = GR.grad_fd(ops, n, counts=counts)
    np.testing.assert_allclose(gref, fd, rtol=1e-5, atol=1e-4)
    st = qs.State(n, prec)
    L, g = qs.sv_grad(st, ops, torch.tensor(counts, device="cuda"), mode=1)
    scale = np.maximum(np.abs(gref), 1.0)
    assert np.all(np.abs(g - gref) / scale < (1e-8 if prec else 5e-4))
    assert L == pytest.approx(Lref, rel=1e-9 if prec else 1e-5)
    st.close()


def test_autograd_function(qs):
    from paper_2008_13490_gb300.autograd import circuit_probabilities
    n = 4
    ops = _circ(n, 30, 9)
    arr = qs.gates_array(ops)
    theta = torch.tensor(arr["param"], dtype=torch.float64, requires_grad=True)
    target = torch.tensor(W.rng(1).random(1 << n), device="cuda")
    p = circuit_probabilities(theta, n, arr, prec=qs.QS_C128)
    loss = ((p - target) ** 2).sum()
    loss.backward()
    w = (2 * (p.detach() - target)).cpu().numpy()
    _, gref = GR.grad_adjoint(ops, n, weights=w)
    np.testing.assert_allclose(theta.grad.numpy(), gref, atol=1e-9)
