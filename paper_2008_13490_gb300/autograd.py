"""torch.autograd.Function over the C ABI: circuit angles -> outcome probabilities.

Forward runs ``sv_apply_circuit`` + ``sv_probs``; backward runs the adjoint
kernel ``sv_grad`` (mode 0: L = sum_J w_J p_J with w = dL/dp from autograd),
so any downstream loss on the probabilities differentiates through the
circuit's gate angles.
"""
from __future__ import annotations

import numpy as np
import torch

from . import GATE_DTYPE, QS_C64, State, gates_array, sv_apply_circuit, sv_grad, sv_probs


class CircuitProbabilities(torch.autograd.Function):
    """p = |U(theta) |0...0>|^2 with theta[g, k] = param k of gate g."""

    @staticmethod
    def forward(ctx, theta, n, template, prec, checkpoint_every):
        gates = np.array(template, dtype=GATE_DTYPE, copy=True)
        gates["param"] = theta.detach().to("cpu", torch.float64).numpy()
        st = State(n, prec)
        sv_apply_circuit(st, gates)
        p, _ = sv_probs(st, fp64=True, want_norm=False)
        st.close()
        ctx.save_for_backward(theta)
        ctx.gates, ctx.n, ctx.prec, ctx.ckpt = gates, n, prec, checkpoint_every
        return p

    @staticmethod
    def backward(ctx, grad_p):
        (theta,) = ctx.saved_tensors
        st = State(ctx.n, ctx.prec)
        _, g = sv_grad(st, ctx.gates, grad_p.detach().to(torch.float64).contiguous(), mode=0,
                       checkpoint_every=ctx.ckpt)
        st.close()
        return torch.from_numpy(g).to(theta.device, theta.dtype), None, None, None, None


def circuit_probabilities(theta: torch.Tensor, n: int, ops, prec: int = QS_C64,
                          checkpoint_every: int = 0) -> torch.Tensor:
    """Differentiable probabilities; ``ops`` are gate records, theta is [len(ops), 3]."""
    template = ops if isinstance(ops, np.ndarray) else gates_array(ops)
    return CircuitProbabilities.apply(theta, n, template, prec, checkpoint_every)
