"""GB300 (sm_103a) exact (min,+) products and the 2-domination power chain.

A thin ctypes binding over ``libminplus.so`` (the C ABI in ``include/minplus.h``).
Every function here only marshals arguments: tensors become raw device
pointers, the current torch stream becomes the ``cudaStream_t``, and every step
of the computation runs in the library's CUDA kernels.  There is no CPU or
PyTorch fallback: if the library is not built, every call raises.

Names follow the C ABI.  Notation: path order ``n`` (matrix size
N = |C_n|, Table 1 of arXiv 2409.17688) and cycle length ``m``; the paper
writes the cylinder as P_m x C_n with the letters swapped.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

INF16 = 0x7FFF
INF8 = 0xFF
MP_I16 = 0
MP_U8 = 1

STATUS = {0: "MP_OK", -1: "MP_EINVAL", -2: "MP_EALIAS", -3: "MP_ENOMEM", -4: "MP_ERANGE",
          -5: "MP_ECUDA", -6: "MP_ETIMEOUT", -7: "MP_EBUSY", -8: "MP_ENOTREADY", -9: "MP_EIO",
          -10: "MP_ECHECK"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libminplus.so")
_lib = None


class MinplusError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code


class mp_problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("Z", ctypes.c_void_p),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
                ("ldx", ctypes.c_int64), ("ldy", ctypes.c_int64), ("ldz", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def lib() -> ctypes.CDLL:
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "mp_transfer_size": (I64, [I]),
        "mp_transfer_circuit_info": (I, [I, P, I]),
        "mp_transfer_words": (I64, [I, P, I64]),
        "mp_build_transfer_matrix": (I, [I, P, I64, P, P]),
        "mp_minplus_mul": (I, [P, P, P, I64, I64, I64, I64, I64, I64, I, P]),
        "mp_minplus_power_sequence": (I, [P, I64, I, P, P, P]),
        "mp_transfer_power_sequence": (I, [I, I, P, P, P]),
        "mp_gamma2_cylinder": (I, [I, I64, P]),
        "mp_gamma2_squaring": (I, [I, I64, P]),
        "mp_inject_circuit_timeout": (I, [I, P]),
        "mp_powers_save": (I, [ctypes.c_char_p, I, I, I64, P, P]),
        "mp_powers_info": (I, [ctypes.c_char_p, P, I]),
        "mp_powers_load": (I, [ctypes.c_char_p, P, I64, P]),
        "mp_transfer_power_sequence_from": (I, [I, I, P, I, P, P, P]),
        "mp_gamma2_table": (I, [I, I, P]),
        "mp_transfer_power_sequences": (I, [P, I, I, P, P]),
        "mp_gamma2_tables": (I, [P, I, I, P]),
        "mp_diag_min": (I, [P, I64, I64, P, P]),
        "mp_diff_const": (I, [P, P, I64, P, P]),
        "mp_transfer_recurrence": (I, [I, I, P]),
        "mp_transfer_recurrence_stream": (I, [I, I, I, P]),
        "mp_min_trace": (I, [P, P, I64, I64, I64, P, P]),
        "mp_minplus_mul_batched": (I, [P, I, I, P]),
        "mp_batch_prepare": (I, [P, I, P]),
        "mp_batch_run": (I, [P, I, P]),
        "mp_batch_destroy": (I, [P]),
        "mp_autotune": (I, [P]),
        "mp_tuning_set": (I, [P]),
        "mp_tuning_get": (I, [P]),
        "mp_server_create": (I, [ctypes.c_size_t, I, I64, I64, P]),
        "mp_server_submit": (I, [P, I, I64, P]),
        "mp_server_replay": (I, [P, P, P, P, I64, P]),
        "mp_server_poll": (I, [P, ctypes.c_uint64, P]),
        "mp_server_cancel": (I, [P, ctypes.c_uint64]),
        "mp_server_latency": (I, [P, ctypes.c_uint64, P, P]),
        "mp_server_stats": (I, [P, P]),
        "mp_server_destroy": (I, [P]),
        "mp_dpx_peak": (I, [I, I64, P]),
        "mp_device_status": (I, []),
        "mp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int) -> int:
    if status < 0:
        msg = lib().mp_last_error()
        raise MinplusError(int(status), msg.decode() if msg else "")
    return status


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda, "expected a CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ words / A

def mp_transfer_circuit_info(n: int) -> dict:
    """The reuse circuit of A(D_n)'s sparse step on the current device."""
    import numpy as np
    info = np.zeros(6, dtype=np.int64)
    k = _check(lib().mp_transfer_circuit_info(int(n), ctypes.c_void_p(info.ctypes.data), 6))
    keys = ("width", "levels", "reads", "cover_reads", "nnz", "N")
    return {key: int(info[i]) for i, key in enumerate(keys[:k])}


def mp_transfer_size(n: int) -> int:
    """N = |C_n|, the number of correct n-words."""
    return _check(lib().mp_transfer_size(int(n)))


def mp_transfer_words(n: int) -> np.ndarray:
    """Correct n-words, packed 2 bits per letter, lexicographic order (host)."""
    N = mp_transfer_size(n)
    out = np.zeros(N, dtype=np.uint32)
    _check(lib().mp_transfer_words(int(n), out.ctypes.data, N))
    return out


def mp_build_transfer_matrix(n: int, A=None, words: bool = False, stream=None):
    """A(D_n) on the current CUDA device (int16, INF = 0x7FFF)."""
    import torch
    N = mp_transfer_size(n)
    if A is None:
        A = torch.empty((N, N), dtype=torch.int16, device="cuda")
    assert A.dtype == torch.int16 and A.dim() == 2 and A.shape[0] >= N and A.stride(1) == 1
    W = torch.empty(N, dtype=torch.int32, device=A.device) if words else None
    _check(lib().mp_build_transfer_matrix(int(n), _dev(A), A.stride(0),
                                          _dev(W) if words else None, _stream(stream)))
    return (A, W) if words else A


# --------------------------------------------------------------- products

def _ld(t) -> int:
    """Leading dimension (elements) of a row-major 2-D tensor; an empty
    tensor reports stride 0, so its row length stands in."""
    return int(t.stride(0)) if t.numel() else max(int(t.shape[1]), 1)


def mp_minplus_mul(X, Y, Z=None, stream=None):
    """Z = X (x) Y, exact and saturating; int16 (INF 0x7FFF) or uint8 (INF 255)."""
    import torch
    assert X.dtype == Y.dtype and X.dim() == 2 and Y.dim() == 2 and X.shape[1] == Y.shape[0]
    assert X.stride(1) == 1 and Y.stride(1) == 1
    dtype = {torch.int16: MP_I16, torch.uint8: MP_U8}[X.dtype]
    M, K = X.shape
    N = Y.shape[1]
    if Z is None:
        Z = torch.empty((M, N), dtype=X.dtype, device=X.device)
    assert Z.dtype == X.dtype and Z.stride(1) == 1
    _check(lib().mp_minplus_mul(_dev(X), _dev(Y), _dev(Z), M, N, K, _ld(X), _ld(Y), _ld(Z),
                                dtype, _stream(stream)))
    return Z


def mp_minplus_mul_batched(problems, mode: int = 0, stream=None):
    """problems: list of (X, Y, Z) CUDA tensors; mode 0 persistent, 1 per-product."""
    import torch
    arr = (mp_problem * len(problems))()
    for i, (X, Y, Z) in enumerate(problems):
        dtype = {torch.int16: MP_I16, torch.uint8: MP_U8}[X.dtype]
        arr[i] = mp_problem(X.data_ptr(), Y.data_ptr(), Z.data_ptr(), X.shape[0], Y.shape[1],
                            X.shape[1], _ld(X), _ld(Y), _ld(Z), dtype, 0)
    _check(lib().mp_minplus_mul_batched(ctypes.cast(arr, ctypes.c_void_p), len(problems),
                                        int(mode), _stream(stream)))


class Batch:
    """A prepared batch of products (mp_batch_prepare); run() is graph-capturable."""

    def __init__(self, problems):
        import torch
        self._keep = list(problems)
        arr = (mp_problem * len(problems))()
        for i, (X, Y, Z) in enumerate(problems):
            dtype = {torch.int16: MP_I16, torch.uint8: MP_U8}[X.dtype]
            arr[i] = mp_problem(X.data_ptr(), Y.data_ptr(), Z.data_ptr(), X.shape[0], Y.shape[1],
                                X.shape[1], _ld(X), _ld(Y), _ld(Z), dtype, 0)
        h = ctypes.c_void_p()
        _check(lib().mp_batch_prepare(ctypes.cast(arr, ctypes.c_void_p), len(problems),
                                      ctypes.byref(h)))
        self._h = h

    def run(self, mode: int = 0, stream=None):
        _check(lib().mp_batch_run(self._h, int(mode), _stream(stream)))

    def close(self):
        if self._h:
            lib().mp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_autotune() -> np.ndarray:
    """Times both tile shapes per size class on this device and installs the
    faster; returns the int32[2][6] table (row 0 int16, row 1 uint8)."""
    t = np.zeros((2, 6), dtype=np.int32)
    _check(lib().mp_autotune(t.ctypes.data))
    return t


def mp_tuning_get() -> np.ndarray:
    t = np.zeros((2, 6), dtype=np.int32)
    _check(lib().mp_tuning_get(t.ctypes.data))
    return t


def mp_tuning_set(table) -> None:
    t = np.ascontiguousarray(table, dtype=np.int32).reshape(2, 6)
    _check(lib().mp_tuning_set(t.ctypes.data))


def save_tuning(path: str) -> None:
    """Writes the current table to a JSON cache keyed by the GPU's name."""
    import json

    import torch
    key = torch.cuda.get_device_name()
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = mp_tuning_get().tolist()
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load_tuning(path: str) -> bool:
    """Installs the cached table for this GPU, if the cache has one."""
    import json

    import torch
    if not os.path.exists(path):
        return False
    with open(path) as f:
        data = json.load(f)
    t = data.get(torch.cuda.get_device_name())
    if t is None:
        return False
    mp_tuning_set(t)
    return True


# ------------------------------------------------------------ power chains

def mp_minplus_power_sequence(A, k_max: int, keep_powers: bool = True, stream=None):
    """Powers A^1..A^k_max of a square int16 CUDA matrix and g[k-1] = min diag A^k."""
    import torch
    N = A.shape[0]
    assert A.dtype == torch.int16 and A.shape == (N, N) and A.is_contiguous()
    P = torch.empty((k_max, N, N), dtype=torch.int16, device=A.device) if keep_powers else None
    g = torch.empty(k_max, dtype=torch.int32, device=A.device)
    _check(lib().mp_minplus_power_sequence(_dev(A), N, int(k_max), _dev(P) if keep_powers else None,
                                           _dev(g), _stream(stream)))
    return P, g


def mp_transfer_power_sequence(n: int, k_max: int, keep_powers: bool = True, stream=None):
    """Powers of A(D_n) built on the device from n, and their diagonal minima."""
    import torch
    N = mp_transfer_size(n)
    P = torch.empty((k_max, N, N), dtype=torch.int16, device="cuda") if keep_powers else None
    g = torch.empty(k_max, dtype=torch.int32, device="cuda")
    _check(lib().mp_transfer_power_sequence(int(n), int(k_max), _dev(P) if keep_powers else None,
                                            _dev(g), _stream(stream)))
    return P, g


def mp_transfer_power_sequence_from(n: int, k0: int, P_k0, k_max: int, keep_powers: bool = True,
                                    stream=None):
    """Algorithm 2 resumed from P_k0 = A(D_n)^k0 (a CUDA int16 N x N tensor):
    returns (A^(k0+1)..A^k_max or None, their diagonal minima)."""
    import torch
    N = mp_transfer_size(n)
    assert P_k0.dtype == torch.int16 and tuple(P_k0.shape) == (N, N) and P_k0.is_contiguous()
    steps = int(k_max) - int(k0)
    P = torch.empty((steps, N, N), dtype=torch.int16, device=P_k0.device) if keep_powers else None
    g = torch.empty(max(steps, 0), dtype=torch.int32, device=P_k0.device)
    _check(lib().mp_transfer_power_sequence_from(int(n), int(k0), _dev(P_k0), int(k_max),
                                                 _dev(P) if keep_powers else None, _dev(g),
                                                 _stream(stream)))
    return P, g


def mp_powers_save(path: str, n: int, k0: int, powers, stream=None) -> None:
    """Checkpoint powers[j] = A(D_n)^(k0 + j) (CUDA int16 [count, N, N]) to a file."""
    import torch
    assert powers.dtype == torch.int16 and powers.is_contiguous() and powers.dim() == 3
    _check(lib().mp_powers_save(os.fsencode(path), int(n), int(k0), int(powers.shape[0]), _dev(powers),
                                _stream(stream)))


def mp_powers_info(path: str) -> dict:
    """Header of a powers checkpoint: n, N, k0, count (host only)."""
    info = np.zeros(4, dtype=np.int64)
    _check(lib().mp_powers_info(os.fsencode(path), info.ctypes.data, 4))
    return dict(zip(["n", "N", "k0", "count"], (int(x) for x in info)))


def mp_powers_load(path: str, stream=None):
    """The stored powers as a CUDA int16 [count, N, N] tensor, with the header."""
    import torch
    h = mp_powers_info(path)
    P = torch.empty((h["count"], h["N"], h["N"]), dtype=torch.int16, device="cuda")
    _check(lib().mp_powers_load(os.fsencode(path), _dev(P), int(h["count"]), _stream(stream)))
    return P, h


def mp_gamma2_cylinder(n: int, m: int) -> int:
    """gamma_2(P_n x C_m), synchronous."""
    out = ctypes.c_int64(0)
    _check(lib().mp_gamma2_cylinder(int(n), int(m), ctypes.byref(out)))
    return int(out.value)


def mp_gamma2_squaring(n: int, m: int) -> int:
    """gamma_2(P_n x C_m) by repeated squaring and a min-trace, synchronous."""
    out = ctypes.c_int64(0)
    _check(lib().mp_gamma2_squaring(int(n), int(m), ctypes.byref(out)))
    return int(out.value)


def mp_gamma2_table(n: int, k_max: int) -> np.ndarray:
    """gamma_2(P_n x C_m) for m = 0..k_max (entries m < 3 are -1), synchronous."""
    out = np.zeros(k_max + 1, dtype=np.int64)
    _check(lib().mp_gamma2_table(int(n), int(k_max), out.ctypes.data))
    return out


def mp_transfer_power_sequences(ns, k_max: int, stream=None):
    """min diag A^k, k = 1..k_max, of several path orders at once (device
    int32 [len(ns), k_max]); the chains run side by side on library streams."""
    import torch
    ns_arr = (ctypes.c_int * len(ns))(*[int(n) for n in ns])
    g = torch.empty((len(ns), int(k_max)), dtype=torch.int32, device="cuda")
    _check(lib().mp_transfer_power_sequences(ns_arr, len(ns), int(k_max), _dev(g),
                                             _stream(stream)))
    return g


def mp_gamma2_tables(ns, k_max: int) -> np.ndarray:
    """gamma_2 tables of several path orders, [len(ns), k_max + 1], synchronous."""
    ns_arr = (ctypes.c_int * len(ns))(*[int(n) for n in ns])
    out = np.zeros((len(ns), int(k_max) + 1), dtype=np.int64)
    _check(lib().mp_gamma2_tables(ns_arr, len(ns), int(k_max), out.ctypes.data))
    return out


# -------------------------------------------------------------- reductions

def mp_diff_const(X, Y, stream=None):
    """(min, max, inf_mismatch, any_finite) of X - Y over both-finite entries."""
    import torch
    out = torch.empty(4, dtype=torch.int32, device=X.device)
    _check(lib().mp_diff_const(_dev(X), _dev(Y), X.numel(), _dev(out), _stream(stream)))
    return out


def mp_transfer_recurrence(n: int, K: int = 50):
    """Algorithms 3 and 4 on the device: (r0, a, b, n0) for A(D_n) over K powers."""
    out = np.zeros(4, dtype=np.int32)
    _check(lib().mp_transfer_recurrence(int(n), int(K), out.ctypes.data))
    return tuple(int(v) for v in out)


def mp_transfer_recurrence_stream(n: int, k_limit: int = 64, ring: int = 20):
    """Streaming recurrence detection: (n0, a, b, k) with only `ring` powers kept."""
    out = np.zeros(4, dtype=np.int32)
    _check(lib().mp_transfer_recurrence_stream(int(n), int(k_limit), int(ring), out.ctypes.data))
    return tuple(int(v) for v in out)


def mp_diag_min(P, stream=None):
    import torch
    out = torch.empty(1, dtype=torch.int32, device=P.device)
    _check(lib().mp_diag_min(_dev(P), P.shape[0], P.stride(0), _dev(out), _stream(stream)))
    return out


def mp_min_trace(X, Y, stream=None):
    import torch
    out = torch.empty(1, dtype=torch.int32, device=X.device)
    _check(lib().mp_min_trace(_dev(X), _dev(Y), X.shape[0], X.stride(0), Y.stride(0), _dev(out),
                              _stream(stream)))
    return out


# ----------------------------------------------------------------- serving

class Server:
    """A gamma_2(n, m) server (mp_server_*): submit() returns tickets, poll()
    returns the value or None while pending."""

    def __init__(self, hbm_budget: int, max_batch: int = 256, max_m: int = 2000,
                 max_tickets: int = 1 << 16):
        h = ctypes.c_void_p()
        _check(lib().mp_server_create(int(hbm_budget), int(max_batch), int(max_m),
                                      int(max_tickets), ctypes.byref(h)))
        self._h = h

    def submit(self, n: int, m: int) -> int:
        t = ctypes.c_uint64(0)
        _check(lib().mp_server_submit(self._h, int(n), int(m), ctypes.byref(t)))
        return int(t.value)

    def replay(self, ns, ms, offsets=None):
        """Native load generator: submit query i at offsets[i] seconds (or at once)."""
        ns = np.ascontiguousarray(ns, dtype=np.int32)
        ms = np.ascontiguousarray(ms, dtype=np.int64)
        tk = np.zeros(len(ns), dtype=np.uint64)
        off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.float64)
        _check(lib().mp_server_replay(self._h, ns.ctypes.data, ms.ctypes.data,
                                      None if off is None else off.ctypes.data, len(ns),
                                      tk.ctypes.data))
        return tk

    def poll(self, ticket: int):
        v = ctypes.c_int64(0)
        rc = lib().mp_server_poll(self._h, int(ticket), ctypes.byref(v))
        if rc == -8:
            return None
        _check(rc)
        return int(v.value)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        import time
        t0 = time.perf_counter()
        while True:
            v = self.poll(ticket)
            if v is not None:
                return v
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"ticket {ticket} not answered in {timeout_s} s")
            time.sleep(0.0002)

    def cancel(self, ticket: int) -> None:
        _check(lib().mp_server_cancel(self._h, int(ticket)))

    def latency(self, ticket: int):
        a, b = ctypes.c_double(0), ctypes.c_double(0)
        rc = lib().mp_server_latency(self._h, int(ticket), ctypes.byref(a), ctypes.byref(b))
        if rc == -8:
            return None
        _check(rc)
        return float(a.value), float(b.value)

    def stats(self) -> dict:
        out = np.zeros(8, dtype=np.int64)
        _check(lib().mp_server_stats(self._h, out.ctypes.data))
        keys = ["submitted", "completed", "failed", "cancelled", "batches", "builds",
                "evictions", "resident_bytes"]
        return dict(zip(keys, (int(v) for v in out)))

    def close(self):
        if self._h:
            lib().mp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- misc

def mp_dpx_peak(variant: int = 0, iters: int = 1 << 16) -> float:
    out = ctypes.c_double(0.0)
    _check(lib().mp_dpx_peak(int(variant), int(iters), ctypes.byref(out)))
    return float(out.value)


def mp_device_status() -> int:
    return _check(lib().mp_device_status())


def mp_inject_circuit_timeout(n: int, stream=None) -> None:
    """Failure injection: one circuit step of A(D_n) whose bounded device
    wait runs out; the next mp_device_status() reports MP_ETIMEOUT."""
    _check(lib().mp_inject_circuit_timeout(int(n), _stream(stream)))


def mp_last_error() -> str:
    m = lib().mp_last_error()
    return m.decode() if m else ""
