"""The sharded state vector on the GPU: two gloo ranks on the one device.

Each rank keeps its shard (2^(n-1) amplitudes) in device memory and applies its
gate segments in place through the library (sv_wrap: the shard tensor is wrapped
once, no state is allocated and no copy sweep runs per segment); the half-shard
exchanges are staged through host memory (gloo moves CPU tensors).  No kernel of
one rank waits for the other's: the ranks only meet on the host.  The gathered
state must equal the oracle's (complex128: 1e-12; complex64: relative L2 1e-5).
Also: sv_wrap itself, in place on a caller's tensor.
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

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, s, seed, prec, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import paper_2008_13490_gb300 as qs
    from paper_2008_13490_gb300.sharding import ShardedState, cuda_apply_local, plan_sharded, scatter_state
    torch.cuda.set_device(0)
    qs.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ops = W.random_gate_mix(n, 120, seed=seed)
    full = W.random_state(n, W.rng(seed + 1))
    dt = torch.complex128 if prec else torch.complex64
    shard = torch.from_numpy(scatter_state(full, n, s, rank)).to(dt).cuda()
    plan = plan_sharded(ops, n, s)
    engine = cuda_apply_local()
    st = ShardedState(n, s, rank, shard, engine, stage_host=True)
    res = st.run(plan)
    torch.cuda.synchronize()
    np.save(os.path.join(out_dir, f"shard{rank}.npy"), res.cpu().numpy())
    np.save(os.path.join(out_dir, f"meta{rank}.npy"),
            np.array([engine.wraps, plan.exchanges(), res.data_ptr() == shard.data_ptr()]))
    engine.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec", [0, 1])
def test_two_ranks_on_one_gpu_match_oracle(tmp_path, prec):
    n, s, seed = 14, 1, 21
    world = 1 << s
    mp.spawn(_worker, args=(world, _free_port(), n, s, seed, prec, str(tmp_path)), nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / f"shard{r}.npy") for r in range(world)])
    ops = W.random_gate_mix(n, 120, seed=seed)
    psi0 = W.random_state(n, W.rng(seed + 1))
    if prec == 0:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    ref = SV.apply_circuit(psi0, n, ops)
    if prec:
        assert np.max(np.abs(got - ref)) <= 1e-12
    else:
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    for r in range(world):
        wraps, exchanges, same = np.load(tmp_path / f"meta{r}.npy")
        assert wraps == 1 and exchanges >= 1 and same   # one wrap, in place, real exchanges


def test_wrap_updates_the_callers_tensor_in_place(qs):
    n = 13
    psi0 = W.random_state(n, W.rng(8))
    ops = W.random_gate_mix(n, 100, seed=9)
    t = torch.tensor(psi0, dtype=torch.complex128, device="cuda")
    ptr = t.data_ptr()
    st = qs.sv_wrap(t)
    qs.sv_apply_circuit(st, ops)
    p, norm = qs.sv_probs(st, fp64=True)
    st.close()
    torch.cuda.synchronize()
    assert t.data_ptr() == ptr
    ref = SV.apply_circuit(psi0, n, ops)
    assert np.max(np.abs(t.cpu().numpy() - ref)) <= 1e-12     # the tensor, still alive, holds the result
    assert abs(norm - 1) < 1e-12
    import ctypes
    h = ctypes.c_void_p()
    assert qs.load().sv_wrap(n, 1, t.data_ptr() + 8, None, None, ctypes.byref(h)) == qs.QS_EINVAL   # misaligned
