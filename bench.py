#!/usr/bin/env python
"""Benchmark of the state-vector hot path on one GB300 (or N replicas).

Workload (the 30-qubit configuration): n = 30 qubits, complex64 (8 GiB
state), 40 layers of Haar-random SU(2) on every qubit plus brickwork CZ
(seed 2001) = 1780 gates, started from |0...0>, followed by the Born-rule
probabilities (4 GiB fp32) and their fp64 norm.  One step = one such circuit,
by default through the library's default method (QS_METHOD_AUTO: dense 5-qubit
blocks on the tcgen05 tensor cores with the BF16 three-part split and FP32
accumulation, sparse stretches on tile passes; for this circuit 93 of the 100
blocks are dense and the gates of the other 7 take 3 tile passes; --method
selects another), the tiled FP32 SIMT path reported as a row of the same line.

metric: reported in "gates/s" = gates of the circuit applied to the
full 2^30-amplitude state per second (the real HBM sweeps per second are in
hbm.sweeps_per_s: fused methods apply many gates per sweep).
The JSON line also carries the real HBM sweeps and bytes, the roofline of the
dominant kernel (block passes: HBM-bound; tile passes: FP32-ALU bound against
the FP32 peak measured in the same run), the CPU oracle baseline, the
end-to-end number through the public C ABI with host buffers (gates from a host
array, probabilities into a pinned host buffer through sv_probs_host), launch
counts and the SM clocks sampled during the timed region.

Multi-GPU: replicas only (each rank simulates its own copy of the workload;
there is no exchange), value = all ranks' gates / max rank time.

--impl reference times the FP64 C oracle (oracle/sv_ref.c, OpenMP on all host
cores) on the same workload at full size: each step applies the next
CPU_STEP_GATES gates of the 30-qubit circuit to a resident complex128 state.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate-passes/sec & HBM GB/s (% of peak) at 30 qubits; circuits/sec, p50/p99 served"
UNIT = "gates/s"
N_QUBITS = 30
LAYERS = 40
SEED = 2001
CPU_STEP_GATES = 15    # gates per step of the CPU oracle at 30 qubits


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


_PEAKS = {}


def alu_peaks(qs, torch):
    """Arithmetic peaks measured on this GPU in this run (cached): FP32 and FP64 FMA
    (the library's qs_alu_peak microbenchmark: every SM full of independent FMA
    chains, CUDA events) and TF32 tensor (cuBLAS TF32 GEMM 8192^3 through torch,
    best of 10, CUDA events), with the SM count read from the device."""
    if _PEAKS:
        return _PEAKS
    f32 = qs.alu_peak(0)
    f64 = qs.alu_peak(1)
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    torch.matmul(a, b)
    best = 1e30
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b
    _PEAKS.update({"fp32_tflops": f32["tflops"], "fp64_tflops": f64["tflops"],
                   "tf32_tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "sm_count": f32["sm_count"],
                   "how": "FP32/FP64: qs_alu_peak (8 independent FMA chains per thread, 2048 threads "
                          "per SM, best of 3 launches); TF32: cuBLAS TF32 GEMM 8192^3, best of 10"})
    return _PEAKS


METHOD_NOTE = {
    "auto": "the library's default: the circuit cut into 5-qubit blocks, dense blocks as BF16-split "
            "GEMMs on tcgen05 tensor cores (FP32 accumulation, per-row norm correction), runs of "
            "sparse blocks replayed through 12-qubit shared-memory tile passes",
    "blocks_bf16": "5-qubit fused blocks on tcgen05 tensor cores, BF16 three-part split products, "
                   "FP32 accumulation, per-row norm correction",
    "blocks_tf32": "5-qubit fused blocks on tcgen05 tensor cores, TF32 two-part split products, "
                   "FP32 accumulation, per-row norm correction",
    "tiled": "12-qubit shared-memory tile passes, FP32 SIMT",
    "plain": "one launch per gate, FP32",
}

# sources each kernel is compiled from: a stored ncu traffic figure is used only while
# their hash is unchanged
KERNEL_SOURCES = {
    "tile": ("sv_kernels.cu", "dev_common.cuh", "internal.h", "tile_cp.h"),
    "block": ("block_tc.cu", "internal.h"),
}
TRAFFIC_FILES = {
    ("tile", "tiled"): "tile_pass_kernel_traffic_n30_layered_haar_cz.json",
    ("block", "blocks_bf16"): "block_pipe_kernel_bf16_traffic_n30_layered_haar_cz.json",
    ("block", "auto"): "block_pipe_kernel_bf16_traffic_n30_layered_haar_cz.json",
}


def workload_name(n, gates):
    return (f"{n}-qubit state, {LAYERS} layers Haar SU(2) + brickwork CZ ({gates} gates, seed {SEED}) "
            f"from |0..0>, then Born-rule probabilities")


def kernel_src_hash(kind):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2008_13490_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def stored_traffic(kind, method):
    """DRAM bytes per launch of the dominant kernel at 30 qubits from the committed ncu
    summary, or None when there is none or the kernel's sources have changed since."""
    name = TRAFFIC_FILES.get((kind, method))
    if not name:
        return None
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        tr = json.load(f)
    return tr.get("bytes_per_launch") if tr.get("kernel_src_sha256") == kernel_src_hash(kind) else None


def block_products(tf32):
    """Split products per block pass: A0.B0 plus 3 (TF32, two parts) or 5 (BF16, three
    parts) corrections; each is a real [2^(n-5) x 64] x [64 x 64] GEMM = 2^(n+8) flops."""
    return 4 if tf32 else 6


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        loaded = [s for s in sm if s > 0.5 * (max(sm) if sm else 1)]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle
# The FP64 oracle in plain C (oracle/sv_ref.c) with OpenMP on all host cores, in a
# child process (its threads never share the GPU process).  Modes:
#   steps K k   the 30-qubit workload at full size: a resident complex128 state
#               (16 GiB) from |0..0>, each step applies the next k gates of the
#               circuit; prints the seconds of every step
#   full24      the same circuit family at 24 qubits, all 1420 gates, once
#   small10     the 10-qubit complex128 circuit (20 layers Haar + CNOT matching)
#               and its 1024 probabilities, repeated: seconds per circuit
_CPU_CHILD = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import workloads as W
from oracle import cstate as C
from oracle import gates as G
mode = sys.argv[2]
out = {"threads": C.threads()}
if mode == "steps":
    K, k, n = int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5])
    ops = W.layered_haar_cz(n, %(layers)d, seed=%(seed)d)
    mats = [G.matrix(name, params, mat) for name, _, params, mat in ops]
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    times, g = [], 0
    for _ in range(K):
        t = time.perf_counter()
        for _ in range(k):
            C.apply_matrix(psi, n, mats[g %% len(ops)], ops[g %% len(ops)][1])
            g += 1
        times.append(time.perf_counter() - t)
    out["step_s"] = times
    out["norm"] = float(C.probabilities(psi, n)[1])
elif mode == "full24":
    n = 24
    ops = W.layered_haar_cz(n, %(layers)d, seed=%(seed)d)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    t = time.perf_counter()
    for name, qubits, params, mat in ops:
        C.apply_matrix(psi, n, G.matrix(name, params, mat), qubits)
    C.probabilities(psi, n)
    out["s"] = time.perf_counter() - t
    out["gates"] = len(ops)
else:
    n, reps = 10, 200
    ops = W.layered_haar_cnot(n, 20, seed=1001)
    mats = [G.matrix(name, params, mat) for name, _, params, mat in ops]
    t = time.perf_counter()
    for _ in range(reps):
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
        for (_, qubits, _, _), m in zip(ops, mats):
            C.apply_matrix(psi, n, m, qubits)
        C.probabilities(psi, n)
    out["s_per_circuit"] = (time.perf_counter() - t) / reps
print(json.dumps(out))
""" % {"layers": LAYERS, "seed": SEED}


def cpu_oracle(mode, *args, timeout=900):
    """Runs the C oracle child (OMP threads = the host's cores) and returns its JSON."""
    from oracle import cstate
    cstate.build()
    env = dict(os.environ, OMP_NUM_THREADS=str(os.cpu_count() or 1))
    out = subprocess.run([sys.executable, "-c", _CPU_CHILD, ROOT, mode, *map(str, args)],
                         capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_block(steps=3):
    """The C oracle on all host cores: the 30-qubit workload at full size on a bounded
    sample (`steps` x CPU_STEP_GATES gates in circuit order, gates/s), the whole
    24-qubit circuit of the same family, and the 10-qubit circuits in full."""
    r = cpu_oracle("steps", steps, CPU_STEP_GATES, N_QUBITS)
    timed = r["step_s"][1:] if steps > 1 else r["step_s"]      # the first step touches the state
    gps = CPU_STEP_GATES * len(timed) / sum(timed)
    f24 = cpu_oracle("full24")
    s10 = cpu_oracle("small10")
    return {"value": gps, "unit": UNIT, "cores": r["threads"], "kind": "oracle",
            "sample": f"FP64 C oracle (OpenMP, {r['threads']} threads) on the {N_QUBITS}-qubit workload "
                      f"at full size (complex128, 16 GiB host state): {len(timed)} timed steps of "
                      f"{CPU_STEP_GATES} gates in circuit order after one untimed step",
            "full_24_qubit_circuit": {"gates": f24["gates"], "s": f24["s"],
                                      "gates_per_s": f24["gates"] / f24["s"]},
            "small_10_qubit_circuit_us": s10["s_per_circuit"] * 1e6}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import workloads as W
    r = cpu_oracle("steps", args.warmup + args.steps, CPU_STEP_GATES, N_QUBITS,
                   timeout=3600)
    timed = r["step_s"][args.warmup:]
    value = CPU_STEP_GATES * len(timed) / sum(timed)
    gates = len(W.layered_haar_cz(N_QUBITS, LAYERS, seed=SEED))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(timed) / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(N_QUBITS, gates), "n_qubits": N_QUBITS,
                       "precision": "complex128 (FP64 oracle)", "gates": gates,
                       "method": "FP64 C oracle on the host, OpenMP over amplitude pairs / quads",
                       "step": f"the next {CPU_STEP_GATES} gates of the circuit applied to the resident "
                               f"{N_QUBITS}-qubit state"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["threads"], "kind": "oracle",
                             "sample": f"each step: {CPU_STEP_GATES} gates of the {N_QUBITS}-qubit "
                                       f"workload in circuit order at full size; {args.warmup} untimed "
                                       f"steps first"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- noisy-batch inputs
# Counts of the noisy batch: 1000-shot multinomial draws from the oracle's
# probabilities at the batch's true parameters (seed 4001); the library evaluates
# the likelihood and gradient at perturbed parameters (seed 4002).  The oracle runs
# in a pool of spawned processes, one per host core (spawned, so it may start after
# the GPU is in use; the full run starts it after the timed and end-to-end regions).
NOISY = {"count": 4096, "seed": 4001, "perturb_seed": 4002, "shots": 1000}


_NOISY_BATCH = []


def _noisy_chunk(idx):
    import time as _t

    import workloads as W
    from oracle import noisy as NZ
    if not _NOISY_BATCH:                     # built once per worker process
        _NOISY_BATCH.append(W.noisy_batch(count=NOISY["count"], seed=NOISY["seed"]))
    b = _NOISY_BATCH[0]
    out = []
    t0 = _t.perf_counter()
    for c in idx:
        n, ops, params = b.circuit(int(c))
        out.append(NZ.circuit_probabilities(n, ops, params))
    return list(idx), out, _t.perf_counter() - t0


def noisy_oracle_inputs():
    import multiprocessing as mp

    import numpy as np

    import workloads as W
    b = W.noisy_batch(count=NOISY["count"], seed=NOISY["seed"])
    workers = os.cpu_count() or 1
    # longest circuits first, dealt round-robin so the chunks cost about the same
    cost = np.array([(np.diff(b.op_off)[c] + 1) * 4.0 ** b.nq[c] for c in range(b.size)])
    order = np.argsort(-cost)
    chunks = [order[i::4 * workers] for i in range(4 * workers)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    t0 = time.perf_counter()
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_noisy_chunk, chunks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = time.perf_counter() - t0
    probs = [None] * b.size
    cpu_s = 0.0
    for idx, ps, dt in res:
        cpu_s += dt
        for c, p in zip(idx, ps):
            probs[c] = p
    counts = W.multinomial_counts(probs, NOISY["shots"], seed=NOISY["seed"])
    return {"counts": counts, "params": W.perturbed_params(b, NOISY["perturb_seed"]),
            "oracle_forward": {"wall_s": wall, "cpu_s": cpu_s, "workers": workers,
                               "circuits_per_s": b.size / wall}}


# ---------------------------------------------------------------- GPU arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2008_13490_gb300 as qs
    import workloads as W

    torch.cuda.set_device(local)
    qs.load()
    n = args.n
    ops = W.layered_haar_cz(n, LAYERS, seed=SEED)
    arr = qs.gates_array(ops)
    gates = len(arr)
    st = qs.State(n, qs.QS_C64)
    probs = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    method = {"tiled": qs.METHOD_TILED, "plain": qs.METHOD_PLAIN, "auto": qs.METHOD_AUTO,
              "blocks_tf32": qs.METHOD_BLOCKS_TF32, "blocks_bf16": qs.METHOD_BLOCKS_BF16}[args.method]

    def step():
        qs.sv_set_basis(st, 0)
        s = qs.sv_apply_circuit(st, arr, method)
        qs.sv_probs(st, out=probs, want_norm=False)
        return s

    for _ in range(args.warmup):
        stats = step()
    torch.cuda.synchronize()
    _, norm = qs.sv_probs(st, out=probs)

    # ---- timed region: K steps, CUDA events on the launching stream
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    qs.qs_profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        stats = step()
    e1.record(stream)
    torch.cuda.synchronize()
    kms, kcnt = qs.qs_profile_end()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(world, ms)
    ms_per_step = ms_max / args.steps

    # ---- end to end through the C ABI with host buffers: the gate array from host
    # memory (planner + descriptor upload inside sv_apply_circuit), the probabilities
    # into a pinned host buffer (sv_probs_host: the kernel writes them straight into
    # it), the same number of steps as `value`
    host_probs = torch.empty(1 << n, dtype=torch.float32, pin_memory=True)
    qs.sv_probs_host(st, out=host_probs)               # warm the path of the copy
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        qs.sv_set_basis(st, 0)
        s2 = qs.sv_apply_circuit(st, arr, method)
        qs.sv_probs_host(st, out=host_probs)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(world, e2e_s)

    if rank != 0:
        st.close()
        return 0

    peaks, peak_src = measured_peaks()
    alu = alu_peaks(qs, torch)
    bytes_per_pass = 2 * (1 << n) * 8
    dominant = max(kms, key=lambda k: kms[k])
    avg_ms = kms[dominant] / max(1, kcnt[dominant])
    hbm_gbs = bytes_per_pass / (avg_ms * 1e-3) / 1e9
    if dominant == "tile":
        # tile pass: FP32-ALU bound; flops counted per amplitude per fused op
        per_launch = stats["tile_flops"] / max(1, stats["tile_launches"])
        roof = {"bound": "alu", "kernel": "tile_pass_kernel<float>", "unit": "TFLOP/s",
                "peak": alu["fp32_tflops"],
                "peak_source": "FP32 FMA peak measured in this run (qs_alu_peak)"}
    elif dominant == "block":
        # block GEMM: one HBM sweep per launch (its roof; the tensor work, 4 (TF32) or
        # 6 (BF16) split products of 2^(n+8) flops, is far below the tensor peak)
        per_launch = bytes_per_pass
        tf32 = args.method == "blocks_tf32"   # (the default method uses the BF16 split)
        roof = {"bound": "hbm", "kernel": "block_pipe_kernel<%s>" % ("TF32" if tf32 else "BF16"),
                "unit": "GB/s", "peak": peaks["hbm_gbs"], "peak_source": "measured copy bandwidth",
                "tensor_tflops": block_products(tf32) * 2.0 ** (n + 8) / (avg_ms * 1e-3) / 1e12,
                "tensor_peak_tflops": alu["tf32_tflops"] if tf32 else peaks["bf16_tflops"],
                "tensor_peak_source": "TF32: cuBLAS GEMM measured in this run" if tf32
                else "bf16 burst, MEASURED_PEAKS.json"}
    else:
        per_launch = bytes_per_pass * 1e-12 * 1e12
        roof = {"bound": "hbm", "kernel": dominant, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                "peak_source": "measured copy bandwidth"}
    scale = 1e9 if roof["unit"] == "GB/s" else 1e12
    achieved = per_launch / (avg_ms * 1e-3) / scale
    traffic = stored_traffic(dominant, args.method) if n == N_QUBITS else None
    launches_per_step = 1 + stats["launches"] + 1   # set_basis, circuit, probabilities
    gates_per_s = world * gates * args.steps / (ms_max * 1e-3)
    line = {
        "metric": METRIC, "value": gates_per_s, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(n, gates),
                   "n_qubits": n, "precision": "complex64", "gates": gates,
                   "method": METHOD_NOTE[args.method],
                   "l2": "state (8 GiB) is larger than L2; no flush needed", "parallelism": "replicas"},
        "circuits_per_s": world * args.steps / (ms_max * 1e-3),
        "passes_per_circuit": stats["passes"], "ops_after_fusion": stats["ops_fused"],
        "hbm": {"sweeps_per_s": world * stats["passes"] * args.steps / (ms_max * 1e-3),
                "pass_gbs": hbm_gbs, "peak_gbs": peaks["hbm_gbs"],
                "frac": hbm_gbs / peaks["hbm_gbs"], "bytes_per_pass": bytes_per_pass},
        "roofline": dict(roof, achieved=achieved, frac=achieved / roof["peak"],
                         traffic=traffic,
                         avg_launch_ms=avg_ms, work_per_launch=per_launch),
        "e2e": {"value": world * gates / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(s2["upload_bytes"]),
                "d2h_bytes_per_step": (1 << n) * 4, "steps": args.steps,
                "path": "sv_apply_circuit (host gate array, planner, descriptor upload) + "
                        "sv_probs_host (4 GiB of probabilities written by the kernel into pinned "
                        "host memory)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "norm": norm,
        "peaks_source": peak_src,
        "measured_alu_peaks": alu,
    }
    st.close()
    del probs, host_probs
    torch.cuda.empty_cache()
    if not args.no_extras:
        # the oracle's pool of spawned processes (safe after the GPU is in use) draws the
        # noisy batch's counts after the timed and end-to-end regions, so that its 16
        # busy processes do not share the host with them
        noisy_inputs = noisy_oracle_inputs()
        line["rows"] = {"other_method_30q": extra_other_method(qs, torch, args.method),
                        "qft": extra_qft(qs, torch),
                        "readout": extra_readout(qs, torch),
                        "dense_2q": extra_dense2q(qs, torch),
                        "gst_prediction": extra_gst(qs, torch),
                        "code422": extra_code422(qs, torch),
                        "sv_grad": extra_sv_grad(qs, torch),
                        "fp64": extra_fp64(qs, torch),
                        "small_circuits": extra_small_circuits(qs, torch),
                        "noisy_batch": extra_noisy_batch(qs, torch, noisy_inputs),
                        "serving": extra_serving(qs, torch),
                        "fused_blocks": extra_fused_blocks(qs, torch)}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_block()
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- other rows (extra keys)
def extra_small_circuits(qs, torch):
    """10-qubit complex128 circuits (20 layers Haar + CNOT matching, seed 1001), all 1024
    probabilities: one circuit at a time through the state API (latency; the whole circuit
    runs in one CTA, bound by that SM's FP64 rate), and 4000 submissions through a server
    whose persistent packed kernel runs them side by side (throughput)."""
    import workloads as W
    ops = qs.gates_array(W.layered_haar_cnot(10, 20, seed=1001))
    st = qs.State(10, qs.QS_C128)
    out = torch.empty(1024, dtype=torch.float64, device="cuda")
    for _ in range(5):
        qs.sv_set_basis(st, 0)
        qs.sv_apply_circuit(st, ops)
        qs.sv_probs(st, out=out, fp64=True, want_norm=False)
    torch.cuda.synchronize()
    reps = 200
    t0 = time.perf_counter()
    for _ in range(reps):
        qs.sv_set_basis(st, 0)
        qs.sv_apply_circuit(st, ops)
        qs.sv_probs(st, out=out, fp64=True, want_norm=False)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    st.close()
    res = {"workload": "10-qubit complex128, 20 layers Haar + CNOT matching, 1024 probabilities",
           "one_at_a_time": {"us_per_circuit": dt * 1e6, "circuits_per_s": 1.0 / dt}}
    count = 4000
    for ctas in (16, 64):
        srv = qs.Server(prec=qs.QS_C128, small_max_qubits=10, persistent_ctas=ctas)
        srv.wait(srv.submit(10, ops, 0))     # first launch
        t0 = time.perf_counter()
        tickets = [srv.submit(10, ops, 0) for _ in range(count)]
        for t in tickets:
            srv.wait(t)
        wall = time.perf_counter() - t0
        stt = srv.stats()
        srv.close()
        res[f"server_{ctas}_ctas"] = {"circuits": count, "us_per_circuit": wall / count * 1e6,
                                      "circuits_per_s": count / wall, "p50_ms": stt["p50_ms"],
                                      "p99_ms": stt["p99_ms"], "packed_launches": stt["packed_launches"]}
    return res


def extra_noisy_batch(qs, torch, inputs):
    """4096 noisy circuits of 1-6 qubits (PTM kernel): probabilities, log-likelihood and its
    gradient at perturbed parameters, for 1000-shot counts drawn from the oracle at the true
    parameters (see noisy_oracle_inputs)."""
    import numpy as np

    import workloads as W
    from oracle import noisy as NZ
    batch = W.noisy_batch(count=NOISY["count"], seed=NOISY["seed"])
    batch.counts = inputs["counts"]
    batch.params = inputs["params"]
    dev = qs.NoisyBatchDevice(batch)
    res = {"workload": "4096 circuits, n~U{1..6}, L~U{1..256}, X90/Y90/CZ/idle + depolarizing + "
                       "amplitude damping; 1000-shot counts from the oracle at the true parameters "
                       "(seed 4001), evaluated at perturbed parameters (seed 4002)"}
    # the oracle's own speed on this host: the forward pass of the whole batch (the pool
    # that drew the counts) and the adjoint gradient on a sample of circuits (one core)
    sample = [int(c) for c in W.rng(4003).choice(batch.size, size=8, replace=False)]
    t0 = time.perf_counter()
    for c in sample:
        n, ops, params = batch.circuit(c)
        NZ.grad_adjoint(n, ops, params, batch.counts[batch.cnt_off[c]:batch.cnt_off[c + 1]])
    grad_s = (time.perf_counter() - t0) / len(sample)
    res["cpu_oracle"] = dict(inputs["oracle_forward"],
                             gradient_s_per_circuit_1_core=grad_s,
                             gradient_sample="8 circuits drawn with seed 4003, Kraus-map adjoint")
    # algorithmic flops: 8 per Pauli-vector entry per one-qubit PTM (4 FMA), 1 per CZ permutation entry
    flops = 0.0
    for c in range(batch.size):
        n, ops, _ = batch.circuit(c)
        D = 4 ** n
        for code, a, b in ops:
            if code in (0, 1):
                flops += 8 * D
            elif code == 2:
                flops += D + 2 * 8 * D
            else:
                flops += n * 8 * D
    for grad in (False, True):
        for _ in range(3):
            dev.run(grad=grad)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        reps = 5
        for _ in range(reps):
            dev.run(grad=grad)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        key = "with_gradient" if grad else "forward"
        res[key] = {"ms_per_batch": ms, "circuits_per_s": batch.size / (ms * 1e-3)}
        if not grad:
            res[key]["fwd_gflops"] = flops / (ms * 1e-3) / 1e9
            res[key]["alu_frac_of_fp32_peak"] = flops / (ms * 1e-3) / 1e12 / alu_peaks(qs, torch)["fp32_tflops"]
    return res


def block_errors(qs, torch, n=20, layers=60, seed=3002):
    """Relative L2 error of the block methods against the GPU FP64 per-gate path (itself
    within 1e-12 of the FP64 oracle) on a depth-60 20-qubit circuit (151 blocks)."""
    import numpy as np

    import workloads as W
    ops = qs.gates_array(W.layered_haar_cz(n, layers, seed=seed))
    ref_st = qs.State(n, qs.QS_C128)
    qs.sv_apply_circuit(ref_st, ops, qs.METHOD_PLAIN)
    ref = qs.sv_copy_out(ref_st)
    ref_st.close()
    out = {}
    for name, method in (("tf32", qs.METHOD_BLOCKS_TF32), ("bf16", qs.METHOD_BLOCKS_BF16),
                         ("tiled_fp32", qs.METHOD_TILED)):
        st = qs.State(n, qs.QS_C64)
        qs.sv_apply_circuit(st, ops, method)
        v = qs.sv_copy_out(st).astype(np.complex128)
        st.close()
        out[name] = float(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    out["reference"] = f"complex128 per-gate GPU path, {n} qubits, depth {layers}, seed {seed}"
    return out


def extra_fused_blocks(qs, torch, n=32, layers=60, seed=3001):
    """32-qubit complex64, depth-60 Haar + brickwork CZ fused into 5-qubit blocks on the
    tensor cores (TF32 and BF16 splits), beside the tiled FP32 path on the same state."""
    import workloads as W
    ops = qs.gates_array(W.layered_haar_cz(n, layers, seed=seed))
    out = {"workload": f"{n}-qubit complex64 ({8 << (n - 30)} GiB), {layers} layers Haar + brickwork CZ "
                       f"({len(ops)} gates, seed {seed})",
           "rel_l2_error_at_20_qubits": block_errors(qs, torch)}
    peaks, _ = measured_peaks()
    st = qs.State(n, qs.QS_C64)
    warm = qs.State(14, qs.QS_C64)
    for name, method in (("tf32", qs.METHOD_BLOCKS_TF32), ("bf16", qs.METHOD_BLOCKS_BF16),
                         ("tiled_fp32", qs.METHOD_TILED)):
        qs.sv_apply_circuit(warm, qs.gates_array(W.layered_haar_cz(14, 2, seed=1)), method)
        qs.sv_set_basis(st, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = qs.sv_apply_circuit(st, ops, method, time_kernels=True)
        dt = time.perf_counter() - t0
        kms = sum(s["kernel_ms"])
        gbs = s["passes"] * 2 * 8 * (1 << n) / (kms * 1e-3) / 1e9
        row = {"s_per_circuit": dt, "passes": s["passes"], "kernel_ms": kms,
               "gates_per_s": len(ops) / dt, "hbm_gbs_per_pass": gbs, "hbm_frac": gbs / peaks["hbm_gbs"]}
        if method in (qs.METHOD_BLOCKS_TF32, qs.METHOD_BLOCKS_BF16):
            tf32 = method == qs.METHOD_BLOCKS_TF32
            tflops = s["passes"] * block_products(tf32) * 2.0 ** (n + 8) / (kms * 1e-3) / 1e12
            row["tensor_tflops"] = tflops
            row["tensor_frac"] = tflops / (peaks["bf16_tflops"] / (2 if tf32 else 1))
        out[name] = row
    warm.close()
    st.close()
    return out


def extra_other_method(qs, torch, method_name, steps=3):
    """The headline workload with the other complex64 method (tiled FP32 SIMT if the line
    used fused blocks, else fused blocks BF16): per-step time and its dominant kernel."""
    import workloads as W
    other = "tiled" if method_name != "tiled" else "auto"
    method = {"tiled": qs.METHOD_TILED, "auto": qs.METHOD_AUTO}[other]
    arr = qs.gates_array(W.layered_haar_cz(N_QUBITS, LAYERS, seed=SEED))
    st = qs.State(N_QUBITS, qs.QS_C64)
    probs = torch.empty(1 << N_QUBITS, dtype=torch.float32, device="cuda")

    def step():
        qs.sv_set_basis(st, 0)
        s = qs.sv_apply_circuit(st, arr, method)
        qs.sv_probs(st, out=probs, want_norm=False)
        return s

    s = step()
    torch.cuda.synchronize()
    qs.qs_profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        s = step()
    e1.record()
    torch.cuda.synchronize()
    kms, kcnt = qs.qs_profile_end()
    ms = e0.elapsed_time(e1) / steps
    st.close()
    del probs
    torch.cuda.empty_cache()
    dom = max(kms, key=lambda k: kms[k])
    avg = kms[dom] / max(1, kcnt[dom])
    out = {"method": METHOD_NOTE[other], "ms_per_step": ms, "gates_per_s": len(arr) / (ms * 1e-3),
           "passes": s["passes"], "dominant_kernel": dom, "avg_launch_ms": avg,
           "hbm_gbs_per_pass": 2 * (1 << N_QUBITS) * 8 / (avg * 1e-3) / 1e9}
    if dom == "tile":
        tfl = s["tile_flops"] / max(1, s["tile_launches"]) / (avg * 1e-3) / 1e12
        out["alu_tflops"] = tfl
        out["alu_frac"] = tfl / alu_peaks(qs, torch)["fp32_tflops"]
    return out


def extra_sv_grad(qs, torch, n=24, layers=20, seed=6001):
    """Adjoint gradient d(sum_J w_J p_J)/d(theta) of a parameterised circuit (layers of
    RX, RY, RZ on every qubit + brickwork CZ), complex64 at 24 qubits: time of one
    forward pass vs one gradient (fused backward steps: uncompute, or recompute from
    checkpoints every sqrt(L) gates)."""
    import math

    import numpy as np

    import workloads as W
    g = W.rng(seed)
    ops = []
    for layer in range(layers):
        for q in range(n):
            for name in ("RX", "RY", "RZ"):
                ops.append((name, (q,), (float(g.uniform(-math.pi, math.pi)),), None))
        for q in range(layer % 2, n - 1, 2):
            ops.append(("CZ", (q, q + 1), (), None))
    arr = qs.gates_array(ops)
    w = torch.tensor(g.normal(size=1 << n), device="cuda")
    st = qs.State(n, qs.QS_C64)
    out = {"workload": f"{n}-qubit complex64, {layers} layers RX RY RZ + brickwork CZ ({len(arr)} gates, "
                       f"{3 * n * layers} parameters), loss = sum_J w_J p_J",
           "gates": len(arr)}
    for key, ck in (("uncompute", 0), ("checkpoints", int(math.ceil(math.sqrt(len(arr)))))):
        qs.sv_grad(st, arr, w, mode=0, checkpoint_every=ck)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qs.sv_grad(st, arr, w, mode=0, checkpoint_every=ck)
        torch.cuda.synchronize()
        out[key] = {"ms": (time.perf_counter() - t0) * 1e3, "checkpoint_every": ck}
    qs.sv_set_basis(st, 0)
    qs.sv_apply_circuit(st, arr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qs.sv_set_basis(st, 0)
    qs.sv_apply_circuit(st, arr)
    qs.sv_probs(st, want_norm=False)
    torch.cuda.synchronize()
    out["forward_ms"] = (time.perf_counter() - t0) * 1e3
    out["grad_over_forward"] = out["uncompute"]["ms"] / out["forward_ms"]
    st.close()
    return out


def extra_qft(qs, torch, n=30, seed=2002):
    """30-qubit QFT (Eq. multiqubitqft) on a seeded random basis state |J>, complex64, tiled
    path (the final qubit reversal is a relabeling plus remap passes); 4096 sampled
    amplitudes against the closed form <K|QFT|J> = 2^(-n/2) exp(2 pi i J K / 2^n)."""
    import math

    import numpy as np

    import workloads as W
    ops = qs.gates_array(W.qft_circuit(n))
    J = W.random_basis_index(n, seed)
    st = qs.State(n, qs.QS_C64)
    qs.sv_set_basis(st, J)
    qs.sv_apply_circuit(st, ops)                     # warm-up (planner, first launch)
    qs.sv_set_basis(st, J)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = qs.sv_apply_circuit(st, ops, time_kernels=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    amps = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    qs.sv_copy_out(st, out=amps)
    K = np.random.default_rng(seed).integers(0, 1 << n, size=4096)
    got = amps[torch.from_numpy(K).cuda()].cpu().numpy().astype(np.complex128)
    N = 1 << n
    jk = np.array([(J * int(k)) % N for k in K], dtype=np.float64)
    ref = np.exp(2j * math.pi * jk / N) / math.sqrt(N)
    st.close()
    del amps
    torch.cuda.empty_cache()
    names = ["tile", "plain", "remap", "small", "block"]
    return {"workload": f"{n}-qubit QFT on |J>, J = {J} (seed {seed}), {len(ops)} gates, complex64",
            "s_per_circuit": dt, "gates_per_s": len(ops) / dt, "passes": s["passes"],
            "kernel_ms": {k: v for k, v in zip(names, s["kernel_ms"]) if v > 0},
            "max_abs_err_4096_sampled": float(np.max(np.abs(got - ref))),
            "rel_err_4096_sampled": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}


def extra_readout(qs, torch, n=30, seed=610, reps=5):
    """Readout transforms at 30 qubits: the Bloch vectors of every qubit (Eq.
    multiqubitblochvector; one read of the complex64 state per 12 or 8 qubits) of the
    product state R^z(phi_q) R^y(theta_q)|0>, checked against the single-qubit form
    (sin th cos ph, sin th sin ph, cos th); and the measurement-error model (Eq.
    errordetectionMeasurementError, eps = 0.08 as in the thesis) in place on the FP32
    probabilities (one read+write per 12 or 8 qubits).  CUDA events on the launch stream;
    the state and probabilities exceed L2."""
    import math

    import numpy as np

    import workloads as W
    g = W.rng(seed)
    th = g.uniform(0, math.pi, size=n)
    ph = g.uniform(-math.pi, math.pi, size=n)
    ops = [("RY", (q,), (float(th[q]),), None) for q in range(n)]
    ops += [("RZ", (q,), (float(ph[q]),), None) for q in range(n)]
    st = qs.State(n, qs.QS_C64)
    qs.sv_apply_circuit(st, ops)
    sweeps = 1 + math.ceil((n - 12) / 8)
    peak = measured_peaks()[0]["hbm_gbs"]

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = {}
    ms = timed(lambda: qs.sv_bloch(st))
    r = qs.sv_bloch(st)
    ref = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    byt = sweeps * (1 << n) * 8
    out["bloch"] = {"ms": ms, "sweeps": sweeps, "gbs": byt / ms / 1e6,
                    "hbm_frac": byt / ms / 1e6 / peak,
                    "max_abs_err_vs_closed_form": float(np.max(np.abs(r - ref)))}
    p, _ = qs.sv_probs(st)
    st.close()
    ms = timed(lambda: qs.meas_error(p, 0.08))
    byt = sweeps * 2 * (1 << n) * 4
    out["meas_error_fp32"] = {"ms": ms, "sweeps": sweeps, "gbs": byt / ms / 1e6,
                              "hbm_frac": byt / ms / 1e6 / peak,
                              "sum_after": float(p.double().sum())}
    del p
    torch.cuda.empty_cache()
    out["workload"] = (f"{n}-qubit complex64 product state (seed {seed}); Bloch vectors of all "
                       f"qubits; measurement error eps = 0.08 on the 2^{n} FP32 probabilities")
    return out


def extra_dense2q(qs, torch, n=30, layers=12, seed=3100):
    """30-qubit circuit of dense two-qubit gates: `layers` brickwork layers of Haar-random
    SU(4) (MAT2), complex64, through tile passes (the 4x4 ops inside the tile) and through
    fused blocks (BF16 split); the two final states compared on the device (relative L2)."""
    import workloads as W
    arr = qs.gates_array(W.layered_su4(n, layers, seed))
    out = {"workload": f"{n}-qubit complex64, {layers} brickwork layers of random SU(4) "
                       f"({len(arr)} gates, seed {seed})"}
    states = []
    for name, method in (("tiled", qs.METHOD_TILED), ("blocks_bf16", qs.METHOD_BLOCKS_BF16)):
        st = qs.State(n, qs.QS_C64)
        qs.sv_apply_circuit(st, arr, method)   # warm-up (planner, first launches)
        qs.sv_set_basis(st, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = qs.sv_apply_circuit(st, arr, method)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        amps = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        qs.sv_copy_out(st, out=amps)
        st.close()
        states.append(amps)
        out[name] = {"s_per_circuit": dt, "gates_per_s": len(arr) / dt, "passes": s["passes"],
                     "launches": s["launches"]}
    a, b = states
    out["rel_l2_tiled_vs_blocks"] = float((a - b).norm() / a.norm())
    del states, a, b
    torch.cuda.empty_cache()
    return out


def _gst_inputs(nsets, seed):
    """Inputs of the GST prediction row, built here with numpy: `nsets` noisy sets of the
    thesis's GST gates XI, YI, IX, IY, II, CNOT on 2 qubits (X90 = R^x(pi/2), Y90 =
    R^y(pi/2), qubit 0 the first tensor factor), each gate followed by depolarizing and
    amplitude damping on both qubits with rates drawn per set; PTMs G_ij = Tr(P_i E(P_j))/4
    in the normalised Pauli basis; the four preparations |00>, |10>, |++>, |Psi^->."""
    import numpy as np

    import workloads as W
    I2 = np.eye(2)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0 + 0j, -1])
    P1 = [I2.astype(complex), X, Y, Z]
    P2 = [np.kron(P1[i >> 2], P1[i & 3]) for i in range(16)]

    def rot(Pm, t):
        return np.cos(t / 2) * np.eye(2) - 1j * np.sin(t / 2) * Pm

    def ptm(kraus):
        return np.array([[np.real(np.trace(P2[i] @ sum(K @ P2[j] @ K.conj().T for K in kraus))) / 4
                          for j in range(16)] for i in range(16)])

    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    Us = [np.kron(rot(X, np.pi / 2), I2), np.kron(rot(Y, np.pi / 2), I2), np.kron(I2, rot(X, np.pi / 2)),
          np.kron(I2, rot(Y, np.pi / 2)), np.eye(4, dtype=complex), cnot]
    ideal = [ptm([U]) for U in Us]
    g = W.rng(seed)
    ptms = []
    for _ in range(nsets):
        p, gam = g.uniform(1e-3, 2e-2, size=2)
        dep = [np.sqrt(1 - p) * I2] + [np.sqrt(p / 3) * M for M in (X, Y, Z)]
        ad = [np.array([[1, 0], [0, np.sqrt(1 - gam)]]), np.array([[0, np.sqrt(gam)], [0, 0]])]
        noise = [np.kron(A @ B, C @ Dm) for A in ad for B in dep for C in ad for Dm in dep]
        N = ptm(noise)
        ptms += [N @ T for T in ideal]
    # |rho>> and <<E_J| in the normalised basis P_i / 2: entries <J|P_i|J> / 2
    rho = np.array([np.real(P2[i][0, 0]) / 2 for i in range(16)])
    E = np.array([[np.real(P2[i][J, J]) / 2 for i in range(16)] for J in range(4)])
    preps = [[], [0, 0], [3, 1], [2, 2, 0, 0, 1, 5]]
    gate, prep = [], []
    for s in range(nsets):
        for gi in range(6):
            for pr in preps:
                gate.append(6 * s + gi)
                prep.append([6 * s + k for k in pr] + [-1] * (8 - len(pr)))
    return (np.stack(ptms), rho, E, np.array(gate, dtype=np.int32), np.array(prep, dtype=np.int32))


def extra_gst(qs, torch, nsets=1000, r_max=1000, seed=4400, reps=5):
    """GST predictions for repeated gates (Eq. GSTPrediction): 1000 noisy 2-qubit gate sets
    x 6 gates x 4 preparations = 24000 sequences, p_J(r) for every r = 1..1000 (the series
    kernel, FP32) and at r = 1000 by repeated squaring (FP64); the two compared."""
    import numpy as np
    ptms, rho, E, gate, prep = _gst_inputs(nsets, seed)
    f = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")  # noqa: E731
    dev = (f(ptms, torch.float64), f(rho, torch.float64), f(E, torch.float64),
           f(gate, torch.int32), f(prep, torch.int32))
    count = len(gate)
    out = torch.empty((count, r_max, 4), dtype=torch.float32, device="cuda")
    rr = torch.full((count,), r_max, dtype=torch.int64, device="cuda")
    pw = torch.empty((count, 4), dtype=torch.float64, device="cuda")

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_s = timed(lambda: qs.gst_series(2, *dev, r_max=r_max, out=out))
    ms_p = timed(lambda: qs.gst_power(2, *dev, rr, out=pw))
    diff = float((out[:, -1, :].double() - pw).abs().max())
    tot = float(out[:, -1, :].double().sum(dim=1).sub(1).abs().max())
    del out, pw
    torch.cuda.empty_cache()
    return {"workload": f"{nsets} noisy GST gate sets x 6 gates x 4 preparations = {count} "
                        f"2-qubit sequences, r = 1..{r_max}",
            "series": {"ms": ms_s, "repetitions_per_s": count * r_max / (ms_s * 1e-3),
                       "output_gbs": count * r_max * 16 / (ms_s * 1e-3) / 1e9},
            "power_r1000": {"ms": ms_p, "sequences_per_s": count / (ms_p * 1e-3)},
            "max_abs_series_vs_power_at_r1000": diff, "max_abs_norm_error": tot}


_C422_BARE = {"X1": [("X", (3,))], "X2": [("X", (4,))], "Z1": [("Z", (3,))], "Z2": [("Z", (4,))],
              "HHS": [("H", (3,)), ("H", (4,)), ("CNOT", (3, 4))] * 3,
              "CZ": [("H", (4,)), ("CNOT", (3, 4)), ("H", (4,))]}
_C422_ENC = {"X1": [("X", (1,)), ("X", (3,))], "X2": [("X", (1,)), ("X", (2,))],
             "Z1": [("Z", (1,)), ("Z", (2,))], "Z2": [("Z", (1,)), ("Z", (3,))],
             "HHS": [("H", (q,)) for q in (1, 2, 3, 4)],
             "CZ": [("S", (q,)) for q in (1, 2, 3, 4)] + [("Z", (2,)), ("Z", (3,))]}
_C422_PREP_BARE = {"00": [], "0+": [("H", (4,))], "Phi+": [("H", (3,)), ("CNOT", (3, 4))]}
_C422_PREP_ENC = {"00": [("H", (3,)), ("CNOT", (3, 2)), ("CNOT", (2, 1)), ("CNOT", (3, 4)),
                         ("CNOT", (1, 0)), ("CNOT", (4, 0))],
                  "0+": [("H", (2,)), ("CNOT", (2, 1)), ("H", (3,)), ("CNOT", (3, 4))],
                  "Phi+": [("H", (3,)), ("CNOT", (3, 2)), ("H", (1,)), ("CNOT", (1, 4))]}


def extra_code422(qs, torch, nseq=155, settings=100, seed=4220, reps=5):
    """[[4,2,2]] error-detection experiment, simulation side: 155 synthetic logical
    sequences x 3 initial states = 465 circuits, each in its encoded (5 qubits) and bare
    (2 qubits) versions plus the noiseless bare reference, for `settings` noise levels
    (depolarizing p and amplitude damping gamma after every physical gate) through the
    batched density-matrix kernel (gates and noise composed into PTMs here with numpy),
    then postselection and D_bare/enc on the device."""
    import numpy as np

    import workloads as W
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0 + 0j, -1])
    I2 = np.eye(2, dtype=complex)
    P1 = [I2, X, Y, Z]
    P2 = [np.kron(P1[i >> 2], P1[i & 3]) for i in range(16)]

    def ptm(kraus, P):
        d = P[0].shape[0]
        return np.array([[np.real(np.trace(P[i] @ sum(K @ P[j] @ K.conj().T for K in kraus))) / d
                          for j in range(len(P))] for i in range(len(P))])

    U1 = {"X": X, "Z": Z, "H": np.array([[1, 1], [1, -1]]) / np.sqrt(2), "S": np.diag([1, 1j])}
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    names1 = ["X", "Z", "H", "S"]
    ps = np.linspace(0.0, 0.03, settings)
    ptm1, ptm2 = [], []
    for p in ps:
        gam = p / 2
        dep = [np.sqrt(1 - p) * I2] + [np.sqrt(p / 3) * M for M in (X, Y, Z)]
        ad = [np.array([[1, 0], [0, np.sqrt(1 - gam)]]), np.array([[0, np.sqrt(gam)], [0, 0]])]
        N1 = ptm([A @ B for A in ad for B in dep], P1)
        ptm1 += [N1 @ ptm([U1[g]], P1) for g in names1]
        ptm2.append(np.kron(N1, N1) @ ptm([cnot], P2))
    circuits = W.code422_sequences(nseq, seed)

    def batch(encoded, ideal):
        ops, off, oo = [], [0], [0]
        n = 5 if encoded else 2
        qmap = {b: b for b in range(5)} if encoded else {3: 1, 4: 0}
        for si in range(settings):
            for state, seq in circuits:
                phys = list((_C422_PREP_ENC if encoded else _C422_PREP_BARE)[state])
                for g in seq:
                    phys += (_C422_ENC if encoded else _C422_BARE)[g]
                for name, q in phys:
                    k = 0 if ideal else si
                    if name == "CNOT":
                        ops.append([5, qmap[q[0]], qmap[q[1]], k])
                    else:
                        ops.append([4, qmap[q[0]], 0, 4 * k + names1.index(name)])
                off.append(len(ops))
                oo.append(oo[-1] + (1 << n))
        C = len(off) - 1
        t = lambda a, dt: torch.tensor(np.asarray(a), dtype=dt, device="cuda")  # noqa: E731
        return dict(nq=t([n] * C, torch.int32), op_off=t(off, torch.int64),
                    ops=t(ops, torch.int32).reshape(-1, 4),
                    params=torch.zeros(4 * C, dtype=torch.float64, device="cuda"),
                    out_off=t(oo, torch.int64), max_qubits=n,
                    max_ops=int(np.max(np.diff(off))),
                    probs=torch.empty(oo[-1], dtype=torch.float32, device="cuda")), C

    t1 = lambda a: torch.tensor(np.stack(a), dtype=torch.float64, device="cuda")  # noqa: E731
    tabs = dict(ptm1=t1(ptm1), ptm2=t1(ptm2))
    (enc, C), (bare, _), (ideal, _) = batch(True, False), batch(False, False), batch(False, True)

    def step():
        for b in (enc, bare, ideal):
            qs.dm_apply_channels(**b, **tabs)
        return qs.code422_eval(enc["probs"].reshape(C, 32), bare["probs"].reshape(C, 4),
                               ideal["probs"].reshape(C, 4))

    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        res = step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    p_enc, ratio, d_bare, d_enc = res
    per = len(circuits)
    mid = settings // 3
    return {"workload": f"{per} logical circuits ({nseq} synthetic sequences x 3 states) x {settings} "
                        f"noise levels (p = 0..0.03, gamma = p/2) = {C} circuits, each encoded (5 qubits), "
                        f"bare (2) and noiseless bare",
            "ms": ms, "logical_circuits_per_s": C / (ms * 1e-3),
            "at_p": float(ps[mid]),
            "mean_d_bare": float(d_bare[mid * per:(mid + 1) * per].mean()),
            "mean_d_enc": float(d_enc[mid * per:(mid + 1) * per].mean()),
            "mean_ratio": float(ratio[mid * per:(mid + 1) * per].mean()),
            "noiseless_max_d_enc": float(d_enc[:per].max())}


def extra_fp64(qs, torch, seed=SEED):
    """complex128 runs of the 40-layer workload: the plain per-gate FP64 GPU path at 30
    qubits (16 GiB; the baseline the fused FP32 forms are measured against) and the tiled
    FP64 path at 31 qubits (32 GiB)."""
    import workloads as W
    out = {}
    for key, n, method in (("plain_fp64_30q", 30, qs.METHOD_PLAIN), ("tiled_fp64_31q", 31, qs.METHOD_TILED)):
        ops = qs.gates_array(W.layered_haar_cz(n, LAYERS, seed=seed))
        st = qs.State(n, qs.QS_C128)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = qs.sv_apply_circuit(st, ops, method, time_kernels=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st.close()
        torch.cuda.empty_cache()
        kms = sum(s["kernel_ms"])
        gbs = s["passes"] * 2 * 16 * (1 << n) / (kms * 1e-3) / 1e9
        out[key] = {"n": n, "gates": len(ops), "s_per_circuit": dt, "gates_per_s": len(ops) / dt,
                    "passes": s["passes"], "hbm_gbs_per_pass": gbs}
    return out


def extra_serving(qs, torch, count=1000, pool=100, seed=5001, rate_hz=None):
    """Poisson stream of `count` arrivals of layered Haar + brickwork-CZ circuits, n~U{8..28},
    depth~U{10..200}, complex64, marginal over <= 10 qubits.  The arrivals draw (seeded) from a
    pool of `pool` distinct circuits, which the host builds once.  Compared with a one-at-a-time
    plain per-gate server under the same arrivals: its service times are measured on the first
    40 pool circuits and, for the rest, taken from a least-squares fit of time against
    gates x 2^n (the plain path sweeps the state once per gate)."""
    import numpy as np

    import workloads as W
    spec = W.serving_stream(pool, seed=seed, rate_hz=1.0)
    circuits = [qs.gates_array(W.layered_haar_cz(n, d, seed=cs)) for _, n, d, cs in spec]
    nq = [n for _, n, _, _ in spec]
    masks = [(1 << min(n, 10)) - 1 for n in nq]
    pick = W.rng(seed + 1).integers(0, pool, size=count)
    # one-at-a-time plain per-gate service times
    service = {}
    for i in range(min(40, pool)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = qs.State(nq[i], qs.QS_C64)
        qs.sv_apply_circuit(st, circuits[i], qs.METHOD_PLAIN)
        qs.sv_probs(st, fp64=True, marg_mask=masks[i] if nq[i] > 10 else 0)
        torch.cuda.synchronize()
        service[i] = time.perf_counter() - t0
        st.close()
    x = np.array([len(circuits[i]) * 2.0 ** nq[i] for i in service])
    y = np.array([service[i] for i in service])
    A = np.stack([x, np.ones_like(x)], axis=1)
    coef = np.linalg.lstsq(A, y, rcond=None)[0]
    for i in range(pool):
        if i not in service:
            service[i] = float(max(coef[0] * len(circuits[i]) * 2.0 ** nq[i] + coef[1], 1e-5))
    plain_service = [service[int(c)] for c in pick]
    # the fused server: capacity on a burst of the whole stream, then the Poisson stream at
    # ~80% of it
    srv = qs.Server()
    t0 = time.perf_counter()
    for t in [srv.submit(nq[c], circuits[c], masks[c]) for c in pick[:200]]:
        srv.wait(t)
    fused_cap = 200 / (time.perf_counter() - t0)
    srv.close()
    rate = rate_hz or 0.8 * fused_cap
    gaps = W.rng(seed + 2).exponential(1.0 / rate, size=count)
    srv = qs.Server()
    tickets, arrivals = [], []
    t_start = time.perf_counter()
    for i, c in enumerate(pick):
        target = t_start + float(np.sum(gaps[: i + 1]))
        while time.perf_counter() < target:
            time.sleep(min(0.0005, max(0.0, target - time.perf_counter())))
        arrivals.append(time.perf_counter() - t_start)
        tickets.append(srv.submit(nq[c], circuits[c], masks[c]))
    results = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    # each pool circuit's result is the same wherever it fell in the mix
    first, worst = {}, 0.0
    for c, (res, _) in zip(pick, results):
        c = int(c)
        if c in first:
            worst = max(worst, float(np.max(np.abs(res - first[c]))))
        else:
            first[c] = res
    done, plain_lat = 0.0, []
    for a, sv in zip(arrivals, plain_service):
        done = max(done, a) + sv
        plain_lat.append(1e3 * (done - a))
    return {"workload": f"{count} Poisson arrivals at {rate:.1f}/s (80% of the fused server's burst "
                        f"capacity), drawn from {pool} circuits n~U{{8..28}}, depth~U{{10..200}}, complex64, "
                        f"marginal over <=10 qubits",
            "circuits_per_s": stats["circuits_per_s"], "p50_ms": stats["p50_ms"],
            "p99_ms": stats["p99_ms"], "mean_ms": stats["mean_ms"], "completed": stats["completed"],
            "packed_launches": stats["packed_launches"], "packed_circuits": stats["packed_circuits"],
            "large_circuits": stats["large_circuits"], "idle_timeouts": stats["idle_timeouts"],
            "same_result_in_the_mix_max_abs": worst,
            "plain_one_at_a_time": {"capacity_circuits_per_s": count / sum(plain_service),
                                    "p50_ms": float(np.percentile(plain_lat, 50)),
                                    "p99_ms": float(np.percentile(plain_lat, 99)),
                                    "service_times": "measured on 40 circuits, fitted for the rest"},
            "fused_capacity_circuits_per_s": fused_cap}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other rows' measurements")
    ap.add_argument("--method", default="auto", choices=["auto", "tiled", "plain", "blocks_tf32", "blocks_bf16"],
                    help="state-vector method of the timed workload (default: the library's default "
                         "method; the tiled path is reported as a row)")
    ap.add_argument("--only", default=None,
                    choices=["dm", "serve", "blocks", "small", "qft", "fp64", "grad", "other",
                             "readout", "dense2q", "gst", "code422"],
                    help="run one extra row alone (for profiling) and print it")
    args = ap.parse_args()
    if args.only:
        noisy_inputs = noisy_oracle_inputs() if args.only == "dm" else None
        import torch

        import paper_2008_13490_gb300 as qs
        qs.load()
        fn = {"dm": lambda q, t: extra_noisy_batch(q, t, noisy_inputs), "serve": extra_serving, "blocks": extra_fused_blocks,
              "small": extra_small_circuits, "qft": lambda q, t: extra_qft(q, t, n=args.n), "fp64": extra_fp64,
              "grad": extra_sv_grad, "readout": lambda q, t: extra_readout(q, t, n=args.n),
              "dense2q": extra_dense2q, "gst": extra_gst, "code422": extra_code422,
              "other": lambda q, t: extra_other_method(q, t, args.method)}[args.only]
        print(json.dumps({"only": args.only, "row": fn(qs, torch)}), flush=True)
        return 0
    if args.impl == "reference":
        # the host-only arm needs no process group: rank 0 runs and prints, the
        # other ranks exit at once
        return run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
    world, rank, local = dist_setup()
    rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
