"""Sharded state vector on CPU ranks (gloo, world sizes 2, 4 and 8).

Each rank holds 2^(n-s) amplitudes; gates on rank bits trigger pairwise
half-shard exchanges planned by ``plan_sharded``.  The gathered result must equal
the single-process oracle (the oracle is the local gate engine here; on a GPU
the CUDA library is).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from oracle import statevector as SV
from paper_2008_13490_gb300.sharding import ShardedState, plan_sharded, scatter_state


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_apply(shard, n_local, records):
    psi = shard.numpy()
    psi = SV.apply_circuit(psi, n_local, records)
    return torch.from_numpy(np.ascontiguousarray(psi))


def _worker(rank, world, port, n, s, seed, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ops = W.random_gate_mix(n, 60, seed=seed)
    full = W.random_state(n, W.rng(seed + 1))
    shard = torch.from_numpy(scatter_state(full, n, s, rank))
    plan = plan_sharded(ops, n, s)
    st = ShardedState(n, s, rank, shard, _oracle_apply)
    res = st.run(plan)
    np.save(os.path.join(out_dir, f"shard{rank}.npy"), res.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n,s,seed", [(7, 1, 3), (8, 2, 4), (10, 3, 5)])
def test_sharded_matches_oracle(tmp_path, n, s, seed):
    world = 1 << s
    mp.spawn(_worker, args=(world, _free_port(), n, s, seed, str(tmp_path)), nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / f"shard{r}.npy") for r in range(world)])
    ops = W.random_gate_mix(n, 60, seed=seed)
    ref = SV.apply_circuit(W.random_state(n, W.rng(seed + 1)), n, ops)
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_plan_swaps_only_for_global_qubits():
    n, s = 10, 2
    local_only = [("H", (q,), (), None) for q in range(n - s)]
    assert plan_sharded(local_only, n, s).exchanges() == 0
    touching = local_only + [("X", (n - 1,), (), None)]
    p = plan_sharded(touching, n, s)
    assert p.exchanges() >= 1
    # every gate record in the plan refers to local positions only
    for step in p.steps:
        if step[0] == "gates":
            assert all(q < n - s for rec in step[1] for q in rec[1])
