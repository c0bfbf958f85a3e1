"""Sharded state vector over 2^s ranks: planner and exchange executor.

Layout: physical amplitude index J (n bits); the top s physical bits select the
rank, the low n-s bits index the rank's shard.  A gate can be applied by every
rank on its own shard only if all its qubits sit at local (low) physical
positions.  Before a gate that touches a qubit at a global position, that
qubit is swapped with a local one: for global bit g and local bit l, ranks r
and r ^ 2^(g-(n-s)) exchange the halves of their shards in which bit l differs
from the rank's bit g (each sends 2^(n-s-1) amplitudes and receives as many).
The local victim is the local qubit whose next use lies farthest ahead
(Belady).  At the end the layout is restored so that physical position q holds
qubit q.  Between exchanges each rank applies its gates through a callback
(the CUDA library on a GPU, any reference implementation in tests).

This is the only step of the method that exchanges data between devices; the
batched density-matrix path and the serving loop shard by independent units
and need no exchange.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ShardPlan:
    n: int
    s: int
    steps: list = field(default_factory=list)   # ("gates", [records]) | ("swap", gpos, lpos)

    @property
    def n_local(self) -> int:
        return self.n - self.s

    def exchanges(self) -> int:
        return sum(1 for st in self.steps if st[0] == "swap")


def plan_sharded(ops, n: int, s: int) -> ShardPlan:
    """Schedule gate records for an n-qubit state sharded over 2^s ranks."""
    if s < 0 or s >= n:
        raise ValueError("need 0 <= s < n")
    nl = n - s
    l2p = list(range(n))          # logical qubit -> physical position
    p2l = list(range(n))
    plan = ShardPlan(n, s)
    pending: list = []

    uses = {q: [] for q in range(n)}
    for i, (_, qs, _, _) in enumerate(ops):
        for q in qs:
            uses[q].append(i)
    ptr = {q: 0 for q in range(n)}

    def next_use(q, i):
        u = uses[q]
        while ptr[q] < len(u) and u[ptr[q]] < i:
            ptr[q] += 1
        return u[ptr[q]] if ptr[q] < len(u) else 1 << 60

    def flush():
        if pending:
            plan.steps.append(("gates", list(pending)))
            pending.clear()

    def swap(gpos, lpos):
        flush()
        plan.steps.append(("swap", gpos, lpos))
        a, b = p2l[gpos], p2l[lpos]
        p2l[gpos], p2l[lpos] = b, a
        l2p[a], l2p[b] = lpos, gpos

    for i, (name, qs, params, mat) in enumerate(ops):
        for q in qs:
            if l2p[q] >= nl:
                protect = {l2p[x] for x in qs}
                cands = [p for p in range(nl) if p not in protect]
                victim = max(cands, key=lambda p: next_use(p2l[p], i))
                swap(l2p[q], victim)
        pending.append((name, tuple(l2p[q] for q in qs), params, mat))
    flush()
    # restore: physical q holds logical q (local permutations are relabeled as SWAP gates)
    for gpos in range(nl, n):
        q = gpos
        if p2l[gpos] != q:
            if l2p[q] < nl:
                swap(gpos, l2p[q])
            else:   # q is at another global position: route it through local position 0
                swap(l2p[q], 0)
                swap(gpos, 0)
    local_fix = []
    for p in range(nl):
        while p2l[p] != p:
            q = p2l[p]                  # logical q sits at p and belongs at physical q (< nl)
            local_fix.append(("SWAP", (p, q), (), None))
            a, b = p2l[p], p2l[q]
            p2l[p], p2l[q] = b, a
            l2p[a], l2p[b] = q, p
    if local_fix:
        plan.steps.append(("gates", local_fix))
    return plan


class ShardedState:
    """One rank's shard.  ``shard`` is a complex torch tensor of 2^(n-s) values;
    ``apply_local(shard, n_local, records) -> shard`` applies gate records whose
    qubits are local physical positions.  The half-shard exchanges go through the
    process group directly, or, with ``stage_host=True`` (a CPU-only backend such as
    gloo with shards in device memory), through host copies of the halves."""

    def __init__(self, n: int, s: int, rank: int, shard, apply_local, group=None, stage_host: bool = False):
        self.n, self.s, self.rank = n, s, rank
        self.shard = shard
        self.apply_local = apply_local
        self.group = group
        self.stage_host = stage_host

    def run(self, plan: ShardPlan):
        for step in plan.steps:
            if step[0] == "gates":
                self.shard = self.apply_local(self.shard, plan.n_local, step[1])
            else:
                self._exchange(step[1], step[2])
        return self.shard

    def _exchange(self, gpos: int, lpos: int):
        import torch
        import torch.distributed as dist
        nl = self.n - self.s
        gbit = gpos - nl
        partner = self.rank ^ (1 << gbit)
        mine = (self.rank >> gbit) & 1
        view = self.shard.view(1 << (nl - lpos - 1), 2, 1 << lpos)
        # send the half whose local bit differs from my global bit; receive the partner's
        send = view[:, 1 - mine, :].contiguous()
        if self.stage_host:
            send = send.cpu()
        recv = torch.empty_like(send)
        ops = [dist.P2POp(dist.isend, torch.view_as_real(send), partner, self.group),
               dist.P2POp(dist.irecv, torch.view_as_real(recv), partner, self.group)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        view[:, 1 - mine, :] = recv.to(self.shard.device) if self.stage_host else recv


class CudaLocalEngine:
    """Local gate engine backed by the CUDA library, in place on the shard: the
    shard tensor (complex64 / complex128 on the device) is wrapped once as a state
    (sv_wrap) and every gate segment runs on it directly -- no state allocation and
    no copy sweeps per segment.  ``wraps`` counts the wrappings (one per shard)."""

    def __init__(self, method=None):
        self.method = method
        self.state = None
        self.ptr = None
        self.wraps = 0

    def __call__(self, shard, n_local, records):
        from . import METHOD_AUTO, WrappedState, sv_apply_circuit
        if self.ptr != shard.data_ptr():
            if self.state is not None:
                self.state.close()
            self.state = WrappedState(shard)
            self.ptr = shard.data_ptr()
            self.wraps += 1
        sv_apply_circuit(self.state, records, METHOD_AUTO if self.method is None else self.method)
        return shard

    def close(self):
        if self.state is not None:
            self.state.close()
            self.state = None


def cuda_apply_local(method=None):
    """The in-place CUDA engine (see CudaLocalEngine)."""
    return CudaLocalEngine(method)


def scatter_state(full: np.ndarray, n: int, s: int, rank: int) -> np.ndarray:
    """Rank's shard of a full state in the canonical layout."""
    nl = n - s
    return full[rank << nl:(rank + 1) << nl].copy()
