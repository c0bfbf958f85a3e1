"""Python binding of the qsim C ABI (include/qsim.h): argument marshalling only.

Every step of the computation runs in the CUDA library ``libqsim.so`` built
in-tree for sm_103a; there is no Python or CPU fallback.  PyTorch provides
device memory (its caching allocator backs the states) and CUDA streams.

Names follow the C ABI: :func:`sv_create`, :func:`sv_apply_circuit`,
:func:`sv_probs`, :func:`sv_loglik`, :func:`sv_grad`,
:func:`dm_apply_channels`, ...
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqsim.so")

QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EUNSUPPORTED = range(6)
QS_C64, QS_C128 = 0, 1
METHOD_TILED, METHOD_PLAIN, METHOD_BLOCKS_TF32, METHOD_BLOCKS_BF16, METHOD_AUTO = 0, 1, 2, 3, 4

KIND = {
    "I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8,
    "PX": 9, "MX": 10, "PY": 11, "MY": 12, "RX": 13, "RY": 14, "RZ": 15,
    "U1": 16, "U2": 17, "U3": 18, "RK": 19, "MAT1": 20,
    "CNOT": 32, "CZ": 33, "CP": 34, "SWAP": 35, "MAT2": 36,
}

# qs_gate (296 bytes)
GATE_DTYPE = np.dtype([("kind", "<i4"), ("q", "<i4", (2,)), ("reserved", "<i4"),
                       ("param", "<f8", (3,)), ("m", "<f8", (32,))])
assert GATE_DTYPE.itemsize == 296


class QsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"qsim status {status}: {msg}")
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [("gates_in", ctypes.c_int64), ("ops_fused", ctypes.c_int64),
                ("passes", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("bytes_moved", ctypes.c_double), ("flops", ctypes.c_double),
                ("upload_bytes", ctypes.c_int64), ("tile_launches", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double * 5), ("tile_flops", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


OPT_TIME_KERNELS = 1
DM_VALIDATE = 1


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_T), ("free", _FREE_T), ("ctx", ctypes.c_void_p)]


class DMBatch(ctypes.Structure):
    _fields_ = [("n_circuits", ctypes.c_int32), ("max_qubits", ctypes.c_int32),
                ("max_ops", ctypes.c_int32), ("n_ptm1", ctypes.c_int32),
                ("n_ptm2", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("nq", ctypes.c_void_p), ("op_off", ctypes.c_void_p), ("ops", ctypes.c_void_p),
                ("params", ctypes.c_void_p), ("out_off", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("ptm1", ctypes.c_void_p), ("ptm2", ctypes.c_void_p)]


class GstBatch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("count", ctypes.c_int32), ("r_max", ctypes.c_int32),
                ("n_ptm", ctypes.c_int32), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ptms", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("effects", ctypes.c_void_p), ("gate", ctypes.c_void_p), ("prep", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("small_max_qubits", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("persistent_ctas", ctypes.c_int32),
                ("mem_budget", ctypes.c_uint64), ("idle_ms", ctypes.c_int32),
                ("large_tiled", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("packed_launches", ctypes.c_int64), ("packed_circuits", ctypes.c_int64),
                ("large_circuits", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("circuits_per_s", ctypes.c_double), ("peak_bytes", ctypes.c_uint64),
                ("idle_timeouts", ctypes.c_int64)]


_lib = None


def load():
    """Load libqsim.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, u64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "sv_create": (i32, [i32, i32, ctypes.POINTER(_Allocator), vp, ctypes.POINTER(vp)]),
        "sv_wrap": (i32, [i32, i32, vp, ctypes.POINTER(_Allocator), vp, ctypes.POINTER(vp)]),
        "sv_destroy": (i32, [vp]),
        "sv_set_stream": (i32, [vp, vp]),
        "sv_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(vp)]),
        "sv_set_basis": (i32, [vp, u64]),
        "sv_copy_in": (i32, [vp, vp, i32]),
        "sv_copy_out": (i32, [vp, vp, i32]),
        "sv_apply_circuit": (i32, [vp, vp, sz, ctypes.POINTER(_Opts), ctypes.POINTER(_Stats)]),
        "sv_probs": (i32, [vp, vp, i32, u64, ctypes.POINTER(ctypes.c_double)]),
        "sv_probs_host": (i32, [vp, vp, i32, u64, ctypes.POINTER(ctypes.c_double)]),
        "sv_probs_host_async": (i32, [vp, vp, i32]),
        "sv_probs_wait": (i32, [vp]),
        "sv_loglik": (i32, [vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
        "sv_grad": (i32, [vp, vp, sz, vp, i32, i32, ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double)]),
        "dm_apply_channels": (i32, [ctypes.POINTER(DMBatch), vp, vp, vp, vp]),
        "qs_probs_noalloc": (i32, [vp, i32, i32, vp, i32, u64, ctypes.POINTER(ctypes.c_double), vp]),
        "sv_bloch": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
        "qs_ptm_check": (i32, [vp, i32, i32, ctypes.POINTER(i32)]),
        "dm_gst_series": (i32, [ctypes.POINTER(GstBatch), vp, vp]),
        "dm_code422_eval": (i32, [i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "dm_gst_power": (i32, [ctypes.POINTER(GstBatch), vp, vp, vp]),
        "sv_save": (i32, [vp, ctypes.c_char_p]),
        "sv_load": (i32, [vp, ctypes.c_char_p]),
        "qs_meas_error": (i32, [vp, i32, i32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), vp]),
        "qs_server_create": (i32, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
        "qs_server_submit": (i32, [vp, i32, vp, sz, u64, ctypes.POINTER(ctypes.c_int64)]),
        "qs_server_wait": (i32, [vp, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_double)]),
        "qs_server_stats_get": (i32, [vp, ctypes.POINTER(ServerStats)]),
        "qs_server_destroy": (i32, [vp]),
        "qs_server_inject_query_error": (i32, [vp, i32]),
        "qs_alu_peak": (i32, [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32),
                              ctypes.POINTER(ctypes.c_double), vp]),
        "qs_profile_begin": (i32, []),
        "qs_profile_end": (i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
        "qs_last_error": (ctypes.c_char_p, []),
        "qs_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return ["sv_create", "sv_wrap", "sv_destroy", "sv_set_stream", "sv_info", "sv_set_basis", "sv_copy_in",
            "sv_copy_out", "sv_apply_circuit", "sv_probs", "sv_probs_host", "sv_probs_host_async", "sv_probs_wait",
            "sv_loglik", "sv_grad",
            "dm_apply_channels", "qs_ptm_check", "qs_probs_noalloc", "sv_bloch", "qs_meas_error", "sv_save", "sv_load",
            "dm_gst_series", "dm_gst_power", "dm_code422_eval",
            "qs_profile_begin", "qs_profile_end", "qs_alu_peak",
            "qs_server_create", "qs_server_submit", "qs_server_wait", "qs_server_stats_get",
            "qs_server_destroy", "qs_server_inject_query_error", "qs_last_error", "qs_version"]


class Server:
    """Continuous-batching circuit server (native scheduler thread; see qsim.h)."""

    def __init__(self, prec: int = QS_C64, small_max_qubits: int = 0, max_inflight: int = 0,
                 persistent_ctas: int = 0, mem_budget: int = 0, idle_ms: int = 0,
                 large_tiled: bool = False):
        lib = load()
        _torch()
        cfg = ServerConfig(prec, small_max_qubits, max_inflight, persistent_ctas, mem_budget, idle_ms,
                           1 if large_tiled else 0)
        h = ctypes.c_void_p()
        _check(lib.qs_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._masks = {}

    def submit(self, n: int, gates, marg_mask: int = 0) -> int:
        arr = gates if isinstance(gates, np.ndarray) else gates_array(gates)
        arr = np.ascontiguousarray(arr, dtype=GATE_DTYPE)
        t = ctypes.c_int64()
        _check(load().qs_server_submit(self.handle, int(n), arr.ctypes.data, len(arr),
                                       int(marg_mask), ctypes.byref(t)))
        k = bin(marg_mask).count("1") if marg_mask else n
        self._masks[t.value] = k
        return t.value

    def wait(self, ticket: int):
        """Returns (marginal probabilities as float64 numpy, latency_ms)."""
        k = self._masks.pop(ticket)
        out = np.empty(1 << k, dtype=np.float64)
        lat = ctypes.c_double()
        _check(load().qs_server_wait(self.handle, int(ticket), out.ctypes.data, ctypes.byref(lat)))
        return out, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().qs_server_stats_get(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().qs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_inject_query_error(srv: Server, cuda_error: int):
    """Testing hook: the server's next completion query reports ``cuda_error``."""
    _check(load().qs_server_inject_query_error(srv.handle, int(cuda_error)))


def ptm_check(ptms, n: int):
    """qs_ptm_check on host PTMs (array of shape (count, 4^n, 4^n) or (4^n, 4^n)).

    Returns -1 when every matrix is trace preserving and completely positive,
    else raises QsimError naming the first failing index."""
    a = np.ascontiguousarray(np.asarray(ptms, dtype=np.float64))
    D = 4 ** n
    a = a.reshape(-1, D, D)
    bad = ctypes.c_int()
    _check(load().qs_ptm_check(a.ctypes.data, int(n), int(a.shape[0]), ctypes.byref(bad)))
    return bad.value


def qs_probs_noalloc(amps_ptr: int, n: int, prec: int, out=None, fp64: bool = False,
                     marg_mask: int = 0, want_norm: bool = True, stream=None):
    """Probabilities of a caller-owned device amplitude buffer, with no device
    allocation inside the library (for callers that may not allocate).
    ``out`` must be a preallocated device tensor; returns (out, norm)."""
    norm = ctypes.c_double()
    _check(load().qs_probs_noalloc(int(amps_ptr), int(n), int(prec),
                                   out.data_ptr() if out is not None else None, 1 if fp64 else 0,
                                   int(marg_mask), ctypes.byref(norm) if want_norm else None,
                                   _stream_ptr(stream)))
    return out, (norm.value if want_norm else None)


def alu_peak(kind: int, stream=None) -> dict:
    """Measured FP32 (kind 0, packed FP32x2 FMA) or FP64 (kind 1) peak of this GPU."""
    f = ctypes.c_double()
    sms = ctypes.c_int()
    ms = ctypes.c_double()
    _check(load().qs_alu_peak(int(kind), ctypes.byref(f), ctypes.byref(sms), ctypes.byref(ms),
                              _stream_ptr(stream)))
    return {"tflops": f.value / 1e12, "sm_count": sms.value, "ms": ms.value}


def qs_profile_begin():
    _check(load().qs_profile_begin())


def qs_profile_end():
    """Returns ({kind: ms}, {kind: launches}) for kinds tile, plain, remap, small, block."""
    ms = (ctypes.c_double * 5)()
    cnt = (ctypes.c_int64 * 5)()
    _check(load().qs_profile_end(ms, cnt))
    kinds = ("tile", "plain", "remap", "small", "block")
    return dict(zip(kinds, list(ms))), dict(zip(kinds, list(cnt)))


def _check(status: int):
    if status != QS_OK:
        raise QsimError(status, load().qs_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("qsim needs a CUDA device")
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


# ---------------------------------------------------------------- allocator
def _make_torch_allocator():
    torch = _torch()

    @_ALLOC_T
    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          stream or 0))
        except Exception:   # out of memory -> NULL -> QS_ENOMEM
            return None

    @_FREE_T
    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = _Allocator(_alloc, _free, None)
    a._keep = (_alloc, _free)
    return a


_TORCH_ALLOC = None


def torch_allocator():
    global _TORCH_ALLOC
    if _TORCH_ALLOC is None:
        _TORCH_ALLOC = _make_torch_allocator()
    return _TORCH_ALLOC


# ---------------------------------------------------------------- gates
def gates_array(ops) -> np.ndarray:
    """Gate records ``(name, qubits, params, matrix)`` -> qs_gate array."""
    arr = np.zeros(len(ops), dtype=GATE_DTYPE)
    for i, (name, qubits, params, mat) in enumerate(ops):
        arr[i]["kind"] = KIND[name]
        arr[i]["q"][: len(qubits)] = qubits
        if params:
            arr[i]["param"][: len(params)] = params
        if mat is not None:
            m = np.asarray(mat, dtype=np.complex128).reshape(-1)
            flat = np.empty(2 * m.size)
            flat[0::2] = m.real
            flat[1::2] = m.imag
            arr[i]["m"][: flat.size] = flat
    return arr


# ---------------------------------------------------------------- state vector
class State:
    """Owns a qs_state_t.  Device memory comes from PyTorch's caching allocator."""

    def __init__(self, n: int, prec: int = QS_C64, stream=None, use_torch_allocator: bool = True):
        lib = load()
        _torch()
        self.n = n
        self.prec = prec
        h = ctypes.c_void_p()
        alloc = ctypes.byref(torch_allocator()) if use_torch_allocator else None
        _check(lib.sv_create(n, prec, alloc, _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().sv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def amp_dtype(self):
        return np.complex64 if self.prec == QS_C64 else np.complex128

    def device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(load().sv_info(self.handle, None, None, ctypes.byref(p)))
        return int(p.value)


def sv_create(n: int, prec: int = QS_C64, stream=None) -> State:
    return State(n, prec, stream)


class WrappedState(State):
    """A state over a caller-owned device tensor (sv_wrap): the library updates the
    tensor in place and never frees it; keep the tensor alive while this lives."""

    def __init__(self, tensor, stream=None):   # noqa: super().__init__ is not called on purpose
        lib = load()
        torch = _torch()
        if not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("a contiguous CUDA tensor is required")
        if tensor.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("complex64 or complex128 amplitudes are required")
        N = tensor.numel()
        n = N.bit_length() - 1
        if N != 1 << n:
            raise ValueError("the tensor must hold 2^n amplitudes")
        self.n = n
        self.prec = QS_C64 if tensor.dtype == torch.complex64 else QS_C128
        self.tensor = tensor
        h = ctypes.c_void_p()
        _check(lib.sv_wrap(n, self.prec, tensor.data_ptr(), ctypes.byref(torch_allocator()),
                           _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h


def sv_wrap(tensor, stream=None) -> WrappedState:
    return WrappedState(tensor, stream)


def sv_destroy(st: State):
    st.close()


def sv_set_stream(st: State, stream):
    _check(load().sv_set_stream(st.handle, _stream_ptr(stream)))


def sv_set_basis(st: State, J: int):
    _check(load().sv_set_basis(st.handle, int(J)))


def sv_copy_in(st: State, amps):
    """amps: numpy array (host) or torch tensor (device) of 2^n complex values."""
    torch = _torch()
    if isinstance(amps, torch.Tensor):
        t = amps.contiguous()
        _check(load().sv_copy_in(st.handle, t.data_ptr(), 1 if t.is_cuda else 0))
        return
    a = np.ascontiguousarray(amps, dtype=st.amp_dtype)
    _check(load().sv_copy_in(st.handle, a.ctypes.data, 0))


def sv_copy_out(st: State, out=None):
    """Returns a host numpy array, or fills a torch device tensor ``out``."""
    torch = _torch()
    if out is not None and isinstance(out, torch.Tensor):
        _check(load().sv_copy_out(st.handle, out.data_ptr(), 1 if out.is_cuda else 0))
        return out
    a = np.empty(1 << st.n, dtype=st.amp_dtype)
    _check(load().sv_copy_out(st.handle, a.ctypes.data, 0))
    return a


def sv_apply_circuit(st: State, gates, method: int = METHOD_AUTO, time_kernels: bool = False) -> dict:
    arr = gates if isinstance(gates, np.ndarray) else gates_array(gates)
    arr = np.ascontiguousarray(arr, dtype=GATE_DTYPE)
    opts = _Opts(method, OPT_TIME_KERNELS if time_kernels else 0)
    stats = _Stats()
    _check(load().sv_apply_circuit(st.handle, arr.ctypes.data, len(arr), ctypes.byref(opts),
                                   ctypes.byref(stats)))
    out = {k: getattr(stats, k) for k, _ in _Stats._fields_}
    out["kernel_ms"] = list(stats.kernel_ms)
    return out


def sv_probs(st: State, out=None, fp64: bool = False, marg_mask: int = 0, want_norm: bool = True):
    """Born-rule probabilities into the device tensor ``out`` (or a new one).

    Returns (out, norm) with norm = sum_J p_J accumulated in fp64 (None if
    want_norm is False, which keeps the call asynchronous)."""
    torch = _torch()
    k = bin(marg_mask).count("1") if marg_mask else st.n
    if out is None:
        out = torch.empty(1 << k, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    norm = ctypes.c_double()
    _check(load().sv_probs(st.handle, out.data_ptr(), 1 if fp64 else 0, int(marg_mask),
                           ctypes.byref(norm) if want_norm else None))
    return out, (norm.value if want_norm else None)


def sv_probs_host(st: State, out=None, fp64: bool = False, marg_mask: int = 0, want_norm: bool = False):
    """Born-rule probabilities into a HOST buffer through the C ABI (a numpy array,
    or a pinned CPU torch tensor ``out``).  Returns (out, norm or None); synchronises."""
    k = bin(marg_mask).count("1") if marg_mask else st.n
    if out is None:
        out = np.empty(1 << k, dtype=np.float64 if fp64 else np.float32)
    ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
    norm = ctypes.c_double()
    _check(load().sv_probs_host(st.handle, ptr, 1 if fp64 else 0, int(marg_mask),
                                ctypes.byref(norm) if want_norm else None))
    return out, (norm.value if want_norm else None)


def sv_probs_host_async(st: State, out, fp64: bool = False):
    """The full Born-rule distribution into a HOST buffer ``out`` (a numpy array, or a
    pinned CPU torch tensor; 2^n float32, or float64 with ``fp64``) without waiting
    for the copy: ``out`` holds it once ``sv_probs_wait(st)`` has returned.  Returns out."""
    ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
    _check(load().sv_probs_host_async(st.handle, ptr, 1 if fp64 else 0))
    return out


def sv_probs_wait(st: State):
    """Waits for the host copies queued on the state by sv_probs_host_async."""
    _check(load().sv_probs_wait(st.handle))


def _gst_batch(n, ptms, rho, effects, gate, prep, r_max=0, validate=False):
    """qs_gst_batch over device tensors: ptms (n_ptm, 4^n, 4^n) float64, rho (4^n,),
    effects (2^n, 4^n), gate (count,) int32, prep (count, 8) int32 (-1 = end)."""
    b = GstBatch(int(n), int(gate.numel()), int(r_max), int(ptms.shape[0]),
                 DM_VALIDATE if validate else 0, 0, ptms.data_ptr(),
                 rho.data_ptr(), effects.data_ptr(), gate.data_ptr(), prep.data_ptr())
    return b


def gst_series(n, ptms, rho, effects, gate, prep, r_max, out=None, stream=None, validate=False):
    """p_J(r) = <<E_J| G_s^r G_prep |rho>> for r = 1..r_max: (count, r_max, 2^n) float32."""
    torch = _torch()
    b = _gst_batch(n, ptms, rho, effects, gate, prep, r_max, validate)
    if out is None:
        out = torch.empty((b.count, r_max, 1 << n), dtype=torch.float32, device="cuda")
    _check(load().dm_gst_series(ctypes.byref(b), out.data_ptr(), _stream_ptr(stream)))
    return out


def gst_power(n, ptms, rho, effects, gate, prep, reps, out=None, stream=None, validate=False):
    """p_J = <<E_J| G_s^reps G_prep |rho>> by repeated squaring: (count, 2^n) float64."""
    torch = _torch()
    b = _gst_batch(n, ptms, rho, effects, gate, prep, validate=validate)
    if out is None:
        out = torch.empty((b.count, 1 << n), dtype=torch.float64, device="cuda")
    _check(load().dm_gst_power(ctypes.byref(b), reps.data_ptr(), out.data_ptr(), _stream_ptr(stream)))
    return out


def code422_eval(enc, bare, ideal, stream=None):
    """[[4,2,2]] evaluation from device float tensors enc (C, 32), bare (C, 4), ideal (C, 4):
    returns (p_enc (C, 4), ratio (C,), d_bare (C,), d_enc (C,))."""
    torch = _torch()
    C = int(enc.shape[0])
    p_enc = torch.empty((C, 4), dtype=torch.float32, device="cuda")
    ratio, d_bare, d_enc = (torch.empty(C, dtype=torch.float32, device="cuda") for _ in range(3))
    _check(load().dm_code422_eval(C, enc.data_ptr(), bare.data_ptr(), ideal.data_ptr(), p_enc.data_ptr(),
                                  ratio.data_ptr(), d_bare.data_ptr(), d_enc.data_ptr(), _stream_ptr(stream)))
    return p_enc, ratio, d_bare, d_enc


def sv_save(st: State, path: str) -> None:
    """Binary checkpoint of the state (see qsim.h for the format)."""
    _check(load().sv_save(st.handle, os.fsencode(path)))


def sv_load(st: State, path: str) -> None:
    """Resume from a checkpoint written for the same n and precision."""
    _check(load().sv_load(st.handle, os.fsencode(path)))


def sv_bloch(st: State) -> np.ndarray:
    """Bloch vectors of every qubit: (n, 3) float64 array, row q = (<X_q>, <Y_q>, <Z_q>)."""
    r = np.zeros(3 * st.n, dtype=np.float64)
    _check(load().sv_bloch(st.handle, r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return r.reshape(st.n, 3)


def meas_error(probs, e01, e10=None, stream=None):
    """Measurement-error model in place on a device probability tensor of 2^n
    float32/float64 values; e01, e10: per-qubit misread rates (scalars or n values;
    e10 defaults to e01).  Returns probs."""
    torch = _torch()
    N = probs.numel()
    n = N.bit_length() - 1
    if N != 1 << n or n < 1:
        raise ValueError("probs must hold 2^n values, n >= 1")
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(e01, dtype=np.float64), (n,)))
    b = None if e10 is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(e10, dtype=np.float64), (n,)))
    dbl = ctypes.POINTER(ctypes.c_double)
    _check(load().qs_meas_error(probs.data_ptr(), n, 1 if probs.dtype == torch.float64 else 0,
                                a.ctypes.data_as(dbl), None if b is None else b.ctypes.data_as(dbl),
                                _stream_ptr(stream)))
    return probs


def sv_loglik(st: State, counts) -> tuple[float, int]:
    """counts: device uint32/int32 tensor of 2^n outcome counts."""
    out = ctypes.c_double()
    clamped = ctypes.c_int64()
    _check(load().sv_loglik(st.handle, counts.data_ptr(), ctypes.byref(out), ctypes.byref(clamped)))
    return out.value, clamped.value


def sv_grad(st: State, gates, weights, mode: int = 0, checkpoint_every: int = 0):
    """Adjoint gradient; weights: device float64 tensor (weights or counts).

    Returns (loss, dtheta[n_gates, 3])."""
    arr = gates if isinstance(gates, np.ndarray) else gates_array(gates)
    arr = np.ascontiguousarray(arr, dtype=GATE_DTYPE)
    g = np.zeros((len(arr), 3), dtype=np.float64)
    loss = ctypes.c_double()
    _check(load().sv_grad(st.handle, arr.ctypes.data, len(arr), weights.data_ptr(), int(mode),
                          int(checkpoint_every),
                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(loss)))
    return loss.value, g


# ---------------------------------------------------------------- density matrices
def dm_apply_channels(nq, op_off, ops, params, out_off, counts=None, ptm1=None, ptm2=None,
                      probs=None, loglik=None, grad=None, max_qubits=6, max_ops=None, stream=None,
                      validate=False):
    """All arrays are torch device tensors (see qs_dm_batch in include/qsim.h).

    ops: int32 [rows, 4] (code, q0, q1, aux).  max_ops defaults to the longest
    circuit (computed from op_off on the host)."""
    b = DMBatch()
    b.n_circuits = int(nq.numel())
    b.max_qubits = int(max_qubits)
    if max_ops is None:
        oo = op_off.cpu().numpy() if hasattr(op_off, "cpu") else np.asarray(op_off)
        max_ops = int(np.max(np.diff(oo))) if len(oo) > 1 else 0
    b.max_ops = int(max_ops)
    b.n_ptm1 = int(ptm1.shape[0]) if ptm1 is not None else 0
    b.n_ptm2 = int(ptm2.shape[0]) if ptm2 is not None else 0
    b.flags = DM_VALIDATE if validate else 0
    ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
    b.nq, b.op_off, b.ops, b.params, b.out_off = (ptr(nq), ptr(op_off), ptr(ops), ptr(params),
                                                   ptr(out_off))
    b.counts, b.ptm1, b.ptm2 = ptr(counts), ptr(ptm1), ptr(ptm2)
    _check(load().dm_apply_channels(ctypes.byref(b), ptr(probs), ptr(loglik), ptr(grad),
                                    _stream_ptr(stream)))


class NoisyBatchDevice:
    """Device copy of a ``workloads.NoisyBatch`` (inputs resident in HBM)."""

    def __init__(self, batch, counts=True):
        torch = _torch()
        dev = "cuda"
        self.size = batch.size
        self.nq = torch.tensor(batch.nq.astype(np.int32), device=dev)
        self.op_off = torch.tensor(batch.op_off.astype(np.int64), device=dev)
        ops4 = np.full((batch.ops.shape[0], 4), 0, dtype=np.int32)
        ops4[:, :3] = batch.ops
        self.ops = torch.tensor(ops4, device=dev)
        self.params = torch.tensor(batch.params.astype(np.float64), device=dev)
        self.out_off = torch.tensor(batch.cnt_off.astype(np.int64), device=dev)
        self.counts = (torch.tensor(batch.counts.astype(np.int32), device=dev)
                       if counts and batch.counts is not None else None)
        self.max_qubits = int(batch.nq.max()) if batch.size else 1
        self.max_ops = int(np.max(np.diff(batch.op_off))) if batch.size else 0
        self.n_out = int(batch.cnt_off[-1])

    def run(self, probs=True, loglik=True, grad=False, stream=None):
        torch = _torch()
        p = torch.empty(self.n_out, dtype=torch.float32, device="cuda") if probs else None
        ll = torch.empty(self.size, dtype=torch.float64, device="cuda") if loglik else None
        g = torch.empty((self.size, 4), dtype=torch.float64, device="cuda") if grad else None
        dm_apply_channels(self.nq, self.op_off, self.ops, self.params, self.out_off,
                          counts=self.counts, probs=p, loglik=ll, grad=g,
                          max_qubits=self.max_qubits, max_ops=self.max_ops, stream=stream)
        return p, ll, g


def version() -> str:
    return load().qs_version().decode()
