"""The host tile-pass planner on the CPU: the plan the library makes of a
circuit (fused ops, passes with their stages, register / lane / warp / tile bit
assignments, remaps, plain ops), executed op by op with numpy in the meaning the
tile kernel gives each field, reproduces the oracle's state.  This pins the
fusion (merged one-qubit runs, folded diagonals, SWAP relabelling) and the stage
and remap bookkeeping without a GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from conftest import ROOT
from oracle import statevector as SV

CS_NONE, CS_TILE, CS_LANE, CS_WARP, CS_REG = 0, 1, 2, 3, 4
TK_REG, TK_LANE, TK_DIAG, TK_G2, TK_G2C = 0, 1, 2, 3, 4
F_G1, F_G1C, F_D, F_G2 = 0, 1, 2, 3


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2008_13490_gb300 import _build
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path_factory.mktemp("tplanner") / "tile_plan_dump"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["g++", "-O1", "-std=c++17", os.path.join(ROOT, "tests", "tile_plan_dump.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    return exe


def _cplx(vals, k):
    v = np.asarray(vals[:2 * k], dtype=np.float64)
    return v[0::2] + 1j * v[1::2], vals[2 * k:]


def _op(vals):
    out = {}
    out["m0"], vals = _cplx(vals, 4)
    out["m1"], vals = _cplx(vals, 4)
    out["d"], vals = _cplx(vals, 4)
    out["g"], vals = _cplx(vals, 16)
    return out


def _plan(exe, tmp_path, n, ops, fuse, relabel, limits=()):
    import paper_2008_13490_gb300 as qs
    gin, out = tmp_path / "g.bin", tmp_path / "plan.txt"
    qs.gates_array(ops).tofile(gin)
    subprocess.run([str(exe), str(gin), str(n), str(int(fuse)), str(int(relabel)), str(out)]
                   + [str(x) for x in limits], check=True)
    lines = open(out).read().split("\n")
    plan, i = {}, 0
    for sec in ("steps", "passes", "stages", "tileops", "plainops", "remaps"):
        head, cnt = lines[i].split()
        assert head == sec
        rows = [lines[i + 1 + k].split() for k in range(int(cnt))]
        plan[sec] = rows
        i += 1 + int(cnt)
    return plan


def _bits(N, p):
    return (np.arange(N) >> p) & 1


def _apply_1q(psi, n, t, M0, M1=None, c=None):
    N = 1 << n
    idx = np.arange(N)
    i0 = idx[_bits(N, t) == 0]
    i1 = i0 | (1 << t)
    if c is None:
        M = [np.full(i0.size, M0[k]) for k in range(4)]
    else:
        sel = ((i0 >> c) & 1).astype(bool)
        M = [np.where(sel, M1[k], M0[k]) for k in range(4)]
    a, b = psi[i0].copy(), psi[i1].copy()
    psi[i0] = M[0] * a + M[1] * b
    psi[i1] = M[2] * a + M[3] * b


def _apply_diag(psi, n, a, b, d):
    N = 1 << n
    k = _bits(N, a) if b is None else 2 * _bits(N, a) + _bits(N, b)
    psi *= np.asarray(d)[k]


def _apply_2q(psi, n, a, b, G):
    N = 1 << n
    idx = np.arange(N)
    base = idx[(_bits(N, a) == 0) & (_bits(N, b) == 0)]
    quad = [base | (((l >> 1) & 1) << a) | ((l & 1) << b) for l in range(4)]
    old = [psi[q].copy() for q in quad]
    G = np.asarray(G).reshape(4, 4)
    for o in range(4):
        psi[quad[o]] = sum(G[o, l] * old[l] for l in range(4))


def _remap(psi, n, pos, src):
    N = 1 << n
    idx = np.arange(N)
    mask = 0
    for p in pos:
        mask |= 1 << p
    new = idx & ~mask
    for j in range(len(pos)):
        new |= ((idx >> pos[src[j]]) & 1) << pos[j]
    out = np.empty_like(psi)
    out[new] = psi
    return out


def _execute(plan, n, psi):
    passes = [[int(x) for x in r] for r in plan["passes"]]
    stages = [[int(x) for x in r] for r in plan["stages"]]
    for kind, index in ([int(x) for x in r] for r in plan["steps"]):
        if kind == 0:
            p = passes[index]
            n_stages, stage_begin, n_nt = p[0], p[1], p[2]
            pos, nt_pos = p[3:15], p[15:15 + n_nt]
            for s in range(stage_begin, stage_begin + n_stages):
                st = stages[s]
                reg, warp, ob, oe = st[0:4], st[4:7], st[7], st[8]

                def phys(src, bit):
                    return {CS_TILE: lambda: nt_pos[bit], CS_LANE: lambda: pos[bit],
                            CS_WARP: lambda: pos[warp[bit]], CS_REG: lambda: pos[reg[bit]]}[src]()

                for row in plan["tileops"][ob:oe]:
                    k, slot, csrc, cbit, dsrc, dbit, typ = (int(x) for x in row[:7])
                    m = _op([float(x) for x in row[7:]])
                    if k == TK_G2C:
                        continue
                    if k == TK_DIAG:
                        assert typ == F_D
                        _apply_diag(psi, n, phys(csrc, cbit), None if dsrc == CS_NONE else phys(dsrc, dbit), m["d"])
                    elif k == TK_G2:
                        assert typ == F_G2
                        _apply_2q(psi, n, phys(csrc, cbit), phys(dsrc, dbit), m["g"])
                    else:
                        t = pos[reg[slot]] if k == TK_REG else pos[slot]
                        if csrc == CS_NONE:
                            assert typ == F_G1
                            _apply_1q(psi, n, t, m["m0"])
                        else:
                            assert typ == F_G1C
                            _apply_1q(psi, n, t, m["m0"], m["m1"], phys(csrc, cbit))
        elif kind == 1:
            row = plan["plainops"][index]
            typ, t, c, a, b = (int(x) for x in row[:5])
            m = _op([float(x) for x in row[5:]])
            if typ == F_G1:
                _apply_1q(psi, n, t, m["m0"])
            elif typ == F_G1C:
                _apply_1q(psi, n, t, m["m0"], m["m1"], c)
            elif typ == F_D:
                _apply_diag(psi, n, a, None if b < 0 else b, m["d"])
            else:
                _apply_2q(psi, n, a, b, m["g"])
        elif kind == 2:
            r = [int(x) for x in plan["remaps"][index]]
            psi = _remap(psi, n, r[0:12], r[12:24])
        else:
            raise AssertionError("small-state step at n >= 12")
    return psi


CASES = {
    "gate_mix": (13, lambda: W.random_gate_mix(13, 300, seed=71), True, True),
    "gate_mix_unfused": (13, lambda: W.random_gate_mix(13, 200, seed=72), False, False),
    "diagonals": (13, lambda: W.random_gate_mix(13, 300, seed=73, two_q_fraction=0.6,
                                               names1=["RZ", "S", "T", "TDG", "U1", "RK", "Z", "H"],
                                               names2=["CZ", "CP"]), True, True),
    "layered": (14, lambda: W.layered_haar_cz(14, 10, seed=74), True, True),
    "qft_relabel": (14, lambda: W.qft_circuit(14), True, True),
    "swaps_dense": (13, lambda: W.random_gate_mix(13, 200, seed=75, two_q_fraction=0.5,
                                                 names2=["SWAP", "CNOT", "CZ"]), True, False),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tile_plan_reproduces_the_circuit(dump_exe, tmp_path, name):
    n, make, fuse, relabel = CASES[name]
    ops = make()
    plan = _plan(dump_exe, tmp_path, n, ops, fuse, relabel)
    assert plan["passes"]
    psi0 = W.random_state(n, W.rng(76))
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out = _execute(plan, n, psi0.copy())
    assert np.max(np.abs(out - ref)) < 1e-12


# ---------------------------------------------------------------- kernel images
# The forward tile pass as the library launches it: ops in their controlled-phase
# forms (TK_CP: a phase on the amplitudes whose two bits are 1, bit positions in
# the thread's context word) and runs of them packed (TK_RUN: per-thread entries,
# per-CTA jobs over tile bits, and host-built tables over (lane, warp) and over the
# 16 register indices).  Executing those images with numpy, in the meaning the
# kernel gives each field, must reproduce the oracle: this pins the packing (which
# factor goes to which table, job or entry list) on the CPU.
TK_CP, TK_RUN = 5, 6
CTX_ONE, CTX_LANE, CTX_WARP = 47, 48, 56


@pytest.fixture(scope="module")
def image_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2008_13490_gb300 import _build
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path_factory.mktemp("timage") / "tile_image_dump"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["g++", "-O1", "-std=c++17", os.path.join(ROOT, "tests", "tile_image_dump.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    return exe


def _images(exe, tmp_path, n, ops, fuse, relabel):
    import paper_2008_13490_gb300 as qs
    gin, out = tmp_path / "g.bin", tmp_path / "images.txt"
    qs.gates_array(ops).tofile(gin)
    subprocess.run([str(exe), str(gin), str(n), str(int(fuse)), str(int(relabel)), str(out)], check=True)
    lines = [l.split() for l in open(out).read().split("\n") if l.strip()]
    res = {"passes": [], "plainops": [], "remaps": []}
    i = 0
    assert lines[i][0] == "steps"
    res["steps"] = [tuple(int(x) for x in r) for r in lines[i + 1:i + 1 + int(lines[i][1])]]
    i += 1 + int(lines[i][1])
    while lines[i][0] == "pass":
        _, _, ns, nj, nt = lines[i]
        geo = [int(x) for x in lines[i + 1]]
        p = {"n_nt": geo[0], "pos": geo[1:13], "nt_pos": geo[13:13 + geo[0]], "stages": [], "jobs": [], "tabs": None}
        i += 2
        for _ in range(int(ns)):
            st = [int(x) for x in lines[i][1:]]
            stage = {"reg": st[0:4], "warp": st[4:7], "ops": []}
            i += 1
            while i < len(lines) and lines[i][0] in ("op", "run"):
                if lines[i][0] == "op":
                    r = lines[i]
                    ints = [int(x) for x in r[1:10]]
                    vals = np.asarray([float(x) for x in r[10:]])
                    c = vals[0::2] + 1j * vals[1::2]
                    stage["ops"].append(("op", ints, c[:4], c[4:8]))
                    i += 1
                else:
                    hdr = [int(x) for x in lines[i][1:]]
                    ents = [(complex(float(e[1]), float(e[2])), int(e[3]), int(e[4]), int(e[5]), int(e[6]))
                            for e in lines[i + 1:i + 1 + hdr[-1]]]
                    stage["ops"].append(("run", hdr, ents))
                    i += 1 + hdr[-1]
            p["stages"].append(stage)
        for _ in range(int(nj)):
            p["jobs"].append([int(x) for x in lines[i][1:]])
            i += 1
        p["tabs"] = np.asarray([complex(float(r[1]), float(r[2])) for r in lines[i:i + int(nt)]])
        i += int(nt)
        res["passes"].append(p)
    assert lines[i][0] == "plainops"
    res["plainops"] = lines[i + 1:i + 1 + int(lines[i][1])]
    i += 1 + int(lines[i][1])
    assert lines[i][0] == "remaps"
    res["remaps"] = lines[i + 1:i + 1 + int(lines[i][1])]
    return res


def _execute_images(img, n, psi):
    N = 1 << n
    J = np.arange(N)
    for kind, index in img["steps"]:
        if kind == 1:
            row = img["plainops"][index]
            typ, t, c, a, b = (int(x) for x in row[:5])
            m = _op([float(x) for x in row[5:]])
            if typ == F_G1:
                _apply_1q(psi, n, t, m["m0"])
            elif typ == F_G1C:
                _apply_1q(psi, n, t, m["m0"], m["m1"], c)
            elif typ == F_D:
                _apply_diag(psi, n, a, None if b < 0 else b, m["d"])
            else:
                _apply_2q(psi, n, a, b, m["g"])
            continue
        if kind == 2:
            r = [int(x) for x in img["remaps"][index]]
            psi = _remap(psi, n, r[0:12], r[12:24])
            continue
        assert kind == 0
        p = img["passes"][index]
        pos, nt_pos = p["pos"], p["nt_pos"]
        tile = np.zeros(N, dtype=np.int64)
        for j, q in enumerate(nt_pos):
            tile |= ((J >> q) & 1) << j
        lane = np.zeros(N, dtype=np.int64)
        for b in range(5):
            lane |= ((J >> pos[b]) & 1) << b
        jobs_by_op = {}
        for op, first, count, scalar in p["jobs"]:
            jobs_by_op.setdefault(op, []).append((first, count, scalar))
        for st in p["stages"]:
            reg, warpb = st["reg"], st["warp"]
            warp = np.zeros(N, dtype=np.int64)
            for b in range(3):
                warp |= ((J >> pos[warpb[b]]) & 1) << b
            rix = np.zeros(N, dtype=np.int64)
            for k in range(4):
                rix |= ((J >> pos[reg[k]]) & 1) << k
            ctx = tile | (1 << CTX_ONE) | (lane << CTX_LANE) | (warp << CTX_WARP)
            lw = warp * 32 + lane

            def cbit(x):   # bit of the context word at position x
                return (ctx >> x) & 1

            def phys(src, bit):
                return {CS_TILE: lambda: nt_pos[bit], CS_LANE: lambda: pos[bit],
                        CS_WARP: lambda: pos[warpb[bit]], CS_REG: lambda: pos[reg[bit]]}[src]()

            ops = st["ops"]
            k2 = 0
            while k2 < len(ops):
                rec = ops[k2]
                if rec[0] == "run":
                    hdr, ents = rec[1], rec[2]
                    opi, n_s, nf, umask, tmask, toff = hdr[0], hdr[1], hdr[2:6], hdr[7], hdr[8], hdr[9]
                    f = np.ones(N, dtype=np.complex128)
                    e = 0
                    for _ in range(n_s):   # residual: both context bits
                        ph, pa, pb, _, _ = ents[e]
                        f *= np.where((cbit(pa) & cbit(pb)) == 1, ph, 1)
                        e += 1
                    for k in range(4):     # residual: register slot k and a context bit
                        for _ in range(nf[k]):
                            ph, pa, _, _, _ = ents[e]
                            f *= np.where((((rix >> k) & 1) & cbit(pa)) == 1, ph, 1)
                            e += 1
                    jl = iter(jobs_by_op.get(opi, []))
                    for b in range(5):     # jobs: scalar (bit 0), then slots 0..3
                        if not (umask >> b) & 1:
                            continue
                        first, count, scalar = next(jl)
                        u = np.ones(N, dtype=np.complex128)
                        for ph, pa, pb, _, _ in ents[first:first + count]:
                            assert pa <= CTX_ONE and (not scalar or pb <= CTX_ONE)
                            on = (cbit(pa) & cbit(pb)) if scalar else cbit(pa)
                            u *= np.where(on == 1, ph, 1)
                        f *= u if b == 0 else np.where(((rix >> (b - 1)) & 1) == 1, u, 1)
                    t = toff
                    if tmask & 1:
                        f *= p["tabs"][t + lw]
                        t += 256
                    for k in range(4):
                        if (tmask >> (1 + k)) & 1:
                            f *= np.where(((rix >> k) & 1) == 1, p["tabs"][t + lw], 1)
                            t += 256
                    if tmask & 32:
                        f *= p["tabs"][t + rix]
                    psi *= f
                    k2 += 1
                    continue
                _, ints, m0, m1 = rec
                _, kind_, slot, csrc, cb, dsrc, db, pad0, pad1 = ints
                if kind_ == TK_CP:
                    ra, rb = csrc == CS_REG, dsrc == CS_REG
                    on_a = ((rix >> cb) & 1) if ra else cbit(pad0)
                    on_b = ((rix >> db) & 1) if rb else cbit(pad1)
                    psi *= np.where((on_a & on_b) == 1, m0[0], 1)
                elif kind_ == TK_DIAG:
                    _apply_diag(psi, n, phys(csrc, cb), None if dsrc == CS_NONE else phys(dsrc, db), m0)
                elif kind_ == TK_G2:
                    nxt = ops[k2 + 1]
                    g = np.concatenate([m0, m1, nxt[2], nxt[3]])
                    _apply_2q(psi, n, phys(csrc, cb), phys(dsrc, db), g)
                    k2 += 1
                else:
                    t = pos[reg[slot]] if kind_ == TK_REG else pos[slot]
                    if csrc == CS_NONE:
                        _apply_1q(psi, n, t, m0)
                    else:
                        _apply_1q(psi, n, t, m0, m1, phys(csrc, cb))
                k2 += 1
    return psi


IMAGE_CASES = {
    "qft": (14, lambda: W.qft_circuit(14), True, True),
    "diagonals": (14, lambda: W.random_gate_mix(14, 400, seed=81, two_q_fraction=0.7,
                                               names1=["RZ", "S", "T", "U1", "RK", "Z", "H"],
                                               names2=["CZ", "CP"]), True, True),
    "layered": (14, lambda: W.layered_haar_cz(14, 12, seed=82), True, True),
}


@pytest.mark.parametrize("name", list(IMAGE_CASES))
def test_tile_pass_images_reproduce_the_circuit(image_exe, tmp_path, name):
    n, make, fuse, relabel = IMAGE_CASES[name]
    ops = make()
    img = _images(image_exe, tmp_path, n, ops, fuse, relabel)
    runs = [r for p in img["passes"] for st in p["stages"] for r in st["ops"] if r[0] == "run"]
    if name != "layered":
        assert runs, "the case should pack controlled-phase runs"
    psi0 = W.random_state(n, W.rng(83))
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    out = _execute_images(img, n, psi0.copy())
    assert np.max(np.abs(out - ref)) < 1e-12


# Seed sweep: random circuits of several widths and gate mixes through the plan
# and through the kernel images (the fixed cases above pin the named structures;
# these reach other tile sets, stage splits and controlled-phase run layouts)
SWEEP = [(12, "phases"), (13, "mix"), (14, "swaps"), (15, "phases"), (16, "mix"), (13, "phases"),
         (14, "mix"), (12, "swaps"), (16, "phases"), (15, "swaps")]


def _sweep_ops(n, kind, seed):
    if kind == "phases":
        return W.random_gate_mix(n, 400, seed=seed, two_q_fraction=0.8,
                                 names1=["H", "RZ", "T", "RK", "U1"], names2=["CP", "CZ"])
    if kind == "swaps":
        return W.random_gate_mix(n, 250, seed=seed, two_q_fraction=0.5,
                                 names2=["SWAP", "CP", "CNOT", "MAT2"])
    return W.random_gate_mix(n, 300, seed=seed)


@pytest.mark.parametrize("case", range(len(SWEEP)))
def test_random_circuits_through_plan_and_images(dump_exe, image_exe, tmp_path, case):
    n, kind = SWEEP[case]
    ops = _sweep_ops(n, kind, 900 + case)
    psi0 = W.random_state(n, W.rng(950 + case))
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    for fuse, relabel in ((True, True), (True, False), (False, False)):
        plan = _plan(dump_exe, tmp_path, n, ops, fuse, relabel)
        assert np.max(np.abs(_execute(plan, n, psi0.copy()) - ref)) < 1e-12, (fuse, relabel)
        img = _images(image_exe, tmp_path, n, ops, fuse, relabel)
        assert np.max(np.abs(_execute_images(img, n, psi0.copy()) - ref)) < 1e-12, (fuse, relabel)


@pytest.mark.parametrize("limits", [(1,), (2,), (3, 12), (48, 6)])
def test_tight_pass_limits(dump_exe, tmp_path, limits):
    # small stage and op budgets per pass: ops (and one-qubit ops merged inside a
    # pass) that do not fit go back to later passes as the original ops, in order
    for case, (n, kind) in enumerate([(13, "mix"), (14, "phases"), (12, "swaps")]):
        ops = _sweep_ops(n, kind, 990 + case)
        psi0 = W.random_state(n, W.rng(995 + case))
        ref = SV.apply_circuit(psi0.copy(), n, ops)
        for fuse in (True, False):
            plan = _plan(dump_exe, tmp_path, n, ops, fuse, fuse, limits)
            for p in plan["passes"]:
                assert int(p[0]) <= limits[0]
            assert np.max(np.abs(_execute(plan, n, psi0.copy()) - ref)) < 1e-12, (limits, n, kind, fuse)


# ---------------------------------------------------------------- one-CTA op lists
# Circuits on fewer than 12 qubits (and the server's packed circuits) run their
# fused op list whole on one CTA, with one-qubit ops on a target merged across the
# ops between them: the list, applied with numpy in order, must give the oracle's
# state, and the merge must not lengthen it.
@pytest.fixture(scope="module")
def fused_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    from paper_2008_13490_gb300 import _build
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path_factory.mktemp("fused") / "fused_ops_dump"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["g++", "-O1", "-std=c++17", os.path.join(ROOT, "tests", "fused_ops_dump.cpp"),
                    "-I", os.path.join(ROOT, "paper_2008_13490_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", cuda_inc, "-o", str(exe), "-L", libdir, "-lqsim", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True, text=True)
    return exe


def _fused(exe, tmp_path, n, ops, merge):
    import paper_2008_13490_gb300 as qs
    gin, out = tmp_path / "g.bin", tmp_path / "fused.txt"
    qs.gates_array(ops).tofile(gin)
    subprocess.run([str(exe), str(gin), str(n), str(int(merge)), str(out)], check=True)
    lines = open(out).read().split("\n")
    head, cnt = lines[0].split()
    assert head == "ops"
    return [lines[1 + k].split() for k in range(int(cnt))]


def _run_fused(rows, n, psi):
    for row in rows:
        typ, t, c, a, b = (int(x) for x in row[:5])
        m = _op([float(x) for x in row[5:]])
        if typ == F_G1:
            _apply_1q(psi, n, t, m["m0"])
        elif typ == F_G1C:
            _apply_1q(psi, n, t, m["m0"], m["m1"], c)
        elif typ == F_D:
            _apply_diag(psi, n, a, None if b < 0 else b, m["d"])
        else:
            _apply_2q(psi, n, a, b, m["g"])
    return psi


SMALL = [(4, "mix"), (6, "phases"), (8, "swaps"), (10, "mix"), (11, "phases"), (10, "cnot"), (9, "layered")]


@pytest.mark.parametrize("case", range(len(SMALL)))
def test_merged_one_cta_op_lists(fused_exe, tmp_path, case):
    n, kind = SMALL[case]
    if kind == "cnot":
        ops = W.layered_haar_cnot(n, 20, seed=1001)
    elif kind == "layered":
        ops = W.layered_haar_cz(n, 12, seed=1002)
    else:
        ops = _sweep_ops(n, kind, 970 + case)
    psi0 = W.random_state(n, W.rng(975 + case))
    ref = SV.apply_circuit(psi0.copy(), n, ops)
    plain = _fused(fused_exe, tmp_path, n, ops, False)
    merged = _fused(fused_exe, tmp_path, n, ops, True)
    assert len(merged) <= len(plain)
    if kind in ("cnot", "layered"):
        assert len(merged) < 0.7 * len(plain)   # one-qubit layers ride on the two-qubit ops
    for rows in (plain, merged):
        assert np.max(np.abs(_run_fused(rows, n, psi0.copy()) - ref)) < 1e-12


# ---------------------------------------------------------------- plan structure
# What the tile kernel relies on in every pass, whichever tile set the planner
# chose: 12 distinct tile positions that include physical bits 0 and 1; per stage,
# 4 register bits and 3 warp bits that split local bits 5..11; lane and register
# slots in range; choice and diagonal bits with a source the kernel can read; the
# pass within the op and stage budgets; stages covering the pass's ops in order.
@pytest.mark.parametrize("case", range(len(SWEEP)))
def test_plan_structure(dump_exe, tmp_path, case):
    n, kind = SWEEP[case]
    ops = _sweep_ops(n, kind, 900 + case)
    for fuse, relabel in ((True, True), (False, False)):
        plan = _plan(dump_exe, tmp_path, n, ops, fuse, relabel)
        stages = [[int(x) for x in r] for r in plan["stages"]]
        kinds = [[int(x) for x in r[:7]] for r in plan["tileops"]]
        next_op = 0
        for p in plan["passes"]:
            n_st, st0, n_nt = (int(x) for x in p[:3])
            pos = [int(x) for x in p[3:15]]
            nt = [int(x) for x in p[15:15 + n_nt]]
            assert len(set(pos)) == 12 and {0, 1} <= set(pos) and sorted(pos) == pos
            assert sorted(pos + nt) == list(range(n))
            assert 1 <= n_st <= 48
            n_ops = 0
            for s in stages[st0:st0 + n_st]:
                reg, warp, b, e = s[0:4], s[4:7], s[7], s[8]
                assert sorted(reg + warp) == list(range(5, 12))
                assert b == next_op and e >= b
                next_op = e
                n_ops += e - b
                for kd, slot, csrc, cbit, dsrc, dbit, typ in kinds[b:e]:
                    if kd == TK_REG:
                        assert 0 <= slot < 4
                    elif kd == TK_LANE:
                        assert 0 <= slot < 5
                    for src, bit in ((csrc, cbit), (dsrc, dbit)):
                        assert src in (CS_NONE, CS_TILE, CS_LANE, CS_WARP, CS_REG)
                        limit = {CS_NONE: 1, CS_TILE: n_nt, CS_LANE: 5, CS_WARP: 3, CS_REG: 4}[src]
                        assert 0 <= bit < max(limit, 1)
            assert n_ops <= 352
        assert next_op == len(kinds)
