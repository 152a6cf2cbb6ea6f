"""Plain CPU oracle for the 2-domination transfer-matrix method (arXiv 2409.17688).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it, and the two share no source.

The arithmetic lives in ``oracle.c`` (plain C, compiled with gcc by
:func:`build`); this module only marshals numpy arrays into it.  Every function
is the plain definition from the paper:

* :func:`enumerate_words`  -- correct n-words (Section 2.2), lexicographic order
* :func:`build_transfer`   -- A(D_n), Algorithm 1
* :func:`minplus_mul`      -- the (min,+) product (Section 1), int32 accumulate
* :func:`power_sequence`   -- Algorithm 2, with min-diagonal readout (Theorem 2)
* :func:`power_rows`       -- rows of the chain via row_k = row_{k-1} (x) A
* :func:`recurrence_search`, :func:`min_recurrence` -- Algorithms 3 and 4
* :func:`gamma2`           -- gamma_2(P_n x C_m) = min diag A^m (Theorem 2)

INF is 0x7FFF for int16 and 255 for uint8, with saturating semantics.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

INF16 = 0x7FFF
INF8 = 0xFF

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so with gcc (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = [cc, "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    lib.or_enumerate_words.argtypes = [I, P, I64]
    lib.or_enumerate_words.restype = I64
    lib.or_can_follow.argtypes = [P, P, I]
    lib.or_can_follow.restype = I
    lib.or_build_transfer.argtypes = [I, P, I64]
    lib.or_build_transfer.restype = I64
    for f in (lib.or_minplus_mul_i16, lib.or_minplus_mul_u8):
        f.argtypes = [P, P, P, I64, I64, I64, I64, I64, I64, I]
        f.restype = None
    lib.or_diag_min.argtypes = [P, I64, I64]
    lib.or_diag_min.restype = ctypes.c_int32
    lib.or_power_sequence.argtypes = [P, I64, I, P, P, I, I]
    lib.or_power_sequence.restype = I
    lib.or_power_rows.argtypes = [P, I64, P, I64, I, P, I]
    lib.or_power_rows.restype = I
    lib.or_transfer_power_rows.argtypes = [I, P, I64, I, P, I]
    lib.or_transfer_power_rows.restype = I64
    lib.or_diff_is_constant.argtypes = [P, P, I64, P]
    lib.or_diff_is_constant.restype = I
    lib.or_recurrence_search.argtypes = [P, I64, I, P, P, P]
    lib.or_recurrence_search.restype = I
    lib.or_min_recurrence.argtypes = [P, I64, I, I, ctypes.c_int32]
    lib.or_min_recurrence.restype = I
    lib.or_have_openmp.argtypes = []
    lib.or_have_openmp.restype = I
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def have_openmp() -> bool:
    return bool(_load().or_have_openmp())


def transfer_size(n: int) -> int:
    """|C_n|, the number of correct n-words (Table 1 rows)."""
    N = _load().or_enumerate_words(int(n), None, 0)
    if N < 0:
        raise ValueError(f"bad path order {n}")
    return int(N)


def enumerate_words(n: int) -> np.ndarray:
    """Correct n-words as an (N, n) uint8 array of letters, lexicographic order."""
    N = transfer_size(n)
    out = np.zeros((N, n), dtype=np.uint8)
    _load().or_enumerate_words(int(n), _ptr(out), N)
    return out


def can_follow(q, p) -> bool:
    """The arc rule of Section 2.2: may column word p follow column word q?"""
    q = np.ascontiguousarray(q, dtype=np.uint8)
    p = np.ascontiguousarray(p, dtype=np.uint8)
    assert q.shape == p.shape and q.ndim == 1
    return bool(_load().or_can_follow(_ptr(q), _ptr(p), q.shape[0]))


def build_transfer(n: int) -> np.ndarray:
    """A(D_n) by Algorithm 1: (N, N) int16, INF16 off the arcs."""
    N = transfer_size(n)
    A = np.empty((N, N), dtype=np.int16)
    r = _load().or_build_transfer(int(n), _ptr(A), N)
    if r != N:
        raise RuntimeError("oracle transfer build failed")
    return A


def minplus_mul(X: np.ndarray, Y: np.ndarray, threads: int = 1) -> np.ndarray:
    """Z = min(INF, X (x) Y) for int16 (INF 0x7FFF) or uint8 (INF 255) inputs."""
    X = np.ascontiguousarray(X)
    Y = np.ascontiguousarray(Y)
    assert X.dtype == Y.dtype and X.ndim == 2 and Y.ndim == 2 and X.shape[1] == Y.shape[0]
    M, K = X.shape
    N = Y.shape[1]
    Z = np.empty((M, N), dtype=X.dtype)
    if X.dtype == np.int16:
        f = _load().or_minplus_mul_i16
    elif X.dtype == np.uint8:
        f = _load().or_minplus_mul_u8
    else:
        raise TypeError("int16 or uint8 only")
    f(_ptr(X), _ptr(Y), _ptr(Z), M, N, K, K, N, N, int(threads))
    return Z


def diag_min(P: np.ndarray) -> int:
    P = np.ascontiguousarray(P, dtype=np.int16)
    return int(_load().or_diag_min(_ptr(P), P.shape[0], P.shape[1]))


def power_sequence(A: np.ndarray, kmax: int, keep_powers: bool = True,
                   left_mul: bool = True, threads: int = 1):
    """Algorithm 2.  Returns (powers or None, gdiag) with powers[k-1] = A^k and
    gdiag[k-1] = min diag A^k.  left_mul selects A (x) A^{k-1} (the paper's
    order, cost N*nnz(A) per step here) versus A^{k-1} (x) A."""
    A = np.ascontiguousarray(A, dtype=np.int16)
    N = A.shape[0]
    powers = np.empty((kmax, N, N), dtype=np.int16) if keep_powers else None
    g = np.empty(kmax, dtype=np.int32)
    r = _load().or_power_sequence(_ptr(A), N, int(kmax),
                                  _ptr(powers) if keep_powers else None,
                                  _ptr(g), int(bool(left_mul)), int(threads))
    if r != 0:
        raise MemoryError("oracle power sequence failed")
    return powers, g


def power_rows(A: np.ndarray, rows, kmax: int, threads: int = 1) -> np.ndarray:
    """Rows `rows` of A^1..A^kmax: out[t, k-1, :] = (A^k)[rows[t], :]."""
    A = np.ascontiguousarray(A, dtype=np.int16)
    N = A.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.shape[0], kmax, N), dtype=np.int16)
    r = _load().or_power_rows(_ptr(A), N, _ptr(rows), rows.shape[0], int(kmax),
                              _ptr(out), int(threads))
    if r != 0:
        raise MemoryError("oracle power rows failed")
    return out


def transfer_power_rows(n: int, rows, kmax: int, threads: int = 1) -> np.ndarray:
    """Rows `rows` of A(D_n)^1..A(D_n)^kmax without forming A (its finite
    entries listed from the word rule): out[t, k-1, :] = (A^k)[rows[t], :]."""
    N = transfer_size(n)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.shape[0], kmax, N), dtype=np.int16)
    r = _load().or_transfer_power_rows(int(n), _ptr(rows), rows.shape[0], int(kmax), _ptr(out),
                                       int(threads))
    if r != N:
        raise MemoryError("oracle transfer power rows failed")
    return out


def diff_is_constant(Pi: np.ndarray, Pj: np.ndarray):
    """(True, b) when Pi - Pj is the constant b with equal INF patterns."""
    Pi = np.ascontiguousarray(Pi, dtype=np.int16)
    Pj = np.ascontiguousarray(Pj, dtype=np.int16)
    b = np.zeros(1, dtype=np.int32)
    ok = _load().or_diff_is_constant(_ptr(Pi), _ptr(Pj), Pi.shape[0], _ptr(b))
    return bool(ok), int(b[0])


def recurrence_search(powers: np.ndarray):
    """Algorithm 3 over powers[k-1] = A^k, k = 1..K.  Returns (r0, a, b) or None."""
    powers = np.ascontiguousarray(powers, dtype=np.int16)
    K, N, _ = powers.shape
    r0 = np.zeros(1, np.int32)
    a = np.zeros(1, np.int32)
    b = np.zeros(1, np.int32)
    ok = _load().or_recurrence_search(_ptr(powers), N, K, _ptr(r0), _ptr(a), _ptr(b))
    return (int(r0[0]), int(a[0]), int(b[0])) if ok else None


def min_recurrence(powers: np.ndarray, r0: int, a: int, b: int) -> int:
    """Algorithm 4: the least n0 with A^{n+a} = b + A^n for all n >= n0."""
    powers = np.ascontiguousarray(powers, dtype=np.int16)
    return int(_load().or_min_recurrence(_ptr(powers), powers.shape[1], r0, a, b))


def gamma2(n: int, m: int, threads: int = 1) -> int:
    """gamma_2(P_n x C_m) = min_i (A^m)_ii (Theorem 2), m >= 3."""
    if m < 3:
        raise ValueError("the cycle C_m needs m >= 3")
    A = build_transfer(n)
    _, g = power_sequence(A, m, keep_powers=False, left_mul=True, threads=threads)
    return int(g[m - 1])


def gamma2_range(n: int, m_max: int, threads: int = 1) -> np.ndarray:
    """gamma_2(P_n x C_m) for m = 0..m_max (entries m < 3 are -1)."""
    A = build_transfer(n)
    _, g = power_sequence(A, m_max, keep_powers=False, left_mul=True, threads=threads)
    out = np.full(m_max + 1, -1, dtype=np.int64)
    out[3:] = g[2:]
    return out
