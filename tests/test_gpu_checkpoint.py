"""State checkpoints (sv_save / sv_load): bit-exact round trips, the file format
read back independently (header fields, amplitudes, checksum recomputed with
numpy), resuming a circuit, and the error paths."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _checksum(amp_bytes: bytes) -> int:
    # sum mod 2^64 of splitmix64_finaliser(w_i + (i + 1) * golden), the format's definition
    w = np.frombuffer(amp_bytes, dtype="<u8")
    with np.errstate(over="ignore"):
        z = w + (np.arange(len(w), dtype=np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
        return int(np.sum(z, dtype=np.uint64))


def _einval(qs, fn, *args):
    with pytest.raises(qs.QsimError) as e:
        fn(*args)
    assert e.value.status == qs.QS_EINVAL


def _state(qs, n, prec, seed):
    psi = W.random_state(n, W.rng(seed))
    psi = psi.astype(np.complex64 if prec == 0 else np.complex128)
    st = qs.State(n, prec)
    qs.sv_copy_in(st, psi)
    return st, psi


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [1, 11, 12, 20])
def test_round_trip_and_format(qs, tmp_path, n, prec):
    st, psi = _state(qs, n, prec, 900 + n)
    path = str(tmp_path / "psi.qsv")
    qs.sv_save(st, path)
    assert np.array_equal(qs.sv_copy_out(st), psi)          # saving leaves the state alone
    raw = open(path, "rb").read()
    assert raw[:8] == b"QSIMSV1\0"
    n_f, prec_f = np.frombuffer(raw[8:16], dtype="<u4")
    nbytes, csum = np.frombuffer(raw[16:32], dtype="<u8")
    assert (n_f, prec_f, nbytes) == (n, prec, psi.nbytes)
    assert raw[32:48] == bytes(16)
    body = raw[48:]
    assert len(body) == psi.nbytes
    assert np.array_equal(np.frombuffer(body, dtype=psi.dtype), psi)
    assert int(csum) == _checksum(body)
    qs.sv_set_basis(st, 0)
    qs.sv_load(st, path)
    assert np.array_equal(qs.sv_copy_out(st), psi)
    st.close()


def test_round_trip_several_chunks(qs, tmp_path):
    # 26 qubits complex64 = 512 MiB: eight 64 MiB chunks through the two pinned buffers
    n = 26
    st = qs.State(n, qs.QS_C64)
    qs.sv_apply_circuit(st, W.layered_haar_cz(n, 3, seed=910))
    ref = qs.sv_copy_out(st)
    path = str(tmp_path / "big.qsv")
    qs.sv_save(st, path)
    assert os.path.getsize(path) == 48 + ref.nbytes
    qs.sv_set_basis(st, 5)
    qs.sv_load(st, path)
    assert np.array_equal(qs.sv_copy_out(st), ref)
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_equals_uninterrupted(qs, tmp_path, prec):
    n = 14
    ops = W.layered_haar_cz(n, 10, seed=920)
    first, second = ops[: len(ops) // 2], ops[len(ops) // 2:]
    a = qs.State(n, prec)
    qs.sv_apply_circuit(a, first)
    qs.sv_apply_circuit(a, second)
    b = qs.State(n, prec)
    qs.sv_apply_circuit(b, first)
    path = str(tmp_path / "mid.qsv")
    qs.sv_save(b, path)
    b.close()
    c = qs.State(n, prec)
    qs.sv_load(c, path)
    qs.sv_apply_circuit(c, second)
    assert np.array_equal(qs.sv_copy_out(c), qs.sv_copy_out(a))
    a.close()
    c.close()


def test_errors(qs, tmp_path):
    n = 12
    st, psi = _state(qs, n, 0, 930)
    path = str(tmp_path / "ok.qsv")
    qs.sv_save(st, path)
    raw = open(path, "rb").read()
    # another size or precision: refused, state unchanged
    other = qs.State(n + 1, qs.QS_C64)
    _einval(qs, qs.sv_load, other, path)
    other.close()
    other = qs.State(n, qs.QS_C128)
    _einval(qs, qs.sv_load, other, path)
    other.close()
    # not a checkpoint / missing file: refused, state unchanged
    junk = str(tmp_path / "junk.qsv")
    open(junk, "wb").write(b"x" * 100)
    for bad in (junk, str(tmp_path / "missing.qsv")):
        _einval(qs, qs.sv_load, st, bad)
        assert np.array_equal(qs.sv_copy_out(st), psi)
    # a flipped amplitude byte or a truncated body: refused, state reset to |0...0>
    zero = np.zeros(1 << n, dtype=np.complex64)
    zero[0] = 1
    flipped = bytearray(raw)
    flipped[48 + 1000] ^= 0x10
    trunc = raw[: len(raw) - 8]
    for i, blob in enumerate((bytes(flipped), trunc)):
        p = str(tmp_path / f"bad{i}.qsv")
        open(p, "wb").write(blob)
        _einval(qs, qs.sv_load, st, p)
        assert np.array_equal(qs.sv_copy_out(st), zero)
        qs.sv_copy_in(st, psi)
    # unwritable path
    _einval(qs, qs.sv_save, st, str(tmp_path / "no_such_dir" / "x.qsv"))
    st.close()
