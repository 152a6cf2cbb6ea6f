"""CPU-side checks of the C ABI: the library loads, exports every symbol
include/minplus.h declares, and its host-only word enumeration (Section 2.2,
Table 1) matches the oracle.  No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mp():
    import paper_2409_17688_gb300 as mp
    from paper_2409_17688_gb300 import _build
    _build.build_library()
    mp.lib()
    return mp


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "minplus.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(mp):
    names = declared_symbols()
    assert "mp_minplus_mul" in names and "mp_transfer_power_sequence" in names
    L = ctypes.CDLL(mp.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name


def test_transfer_size_matches_oracle(mp):
    for n in range(1, 14):
        assert mp.mp_transfer_size(n) == oracle.transfer_size(n)


def test_transfer_words_match_oracle_order(mp):
    for n in range(1, 10):
        W = oracle.enumerate_words(n)
        packed = np.zeros(len(W), dtype=np.uint64)
        for i in range(n):
            packed = (packed << np.uint64(2)) | W[:, i].astype(np.uint64)
        got = mp.mp_transfer_words(n).astype(np.uint64)
        assert np.array_equal(got, packed), n
        assert np.all(np.diff(got.astype(np.int64)) > 0)


def test_invalid_path_order_rejected(mp):
    for n in (0, -3, 17):
        with pytest.raises(mp.MinplusError) as e:
            mp.mp_transfer_size(n)
        assert e.value.code == -1
        assert "path order" in mp.mp_last_error()


def test_circuit_info_rejects_bad_arguments_before_any_cuda_call(mp):
    info = np.zeros(6, dtype=np.int64)
    for n in (0, 17):
        assert mp.lib().mp_transfer_circuit_info(n, ctypes.c_void_p(info.ctypes.data), 6) == -1
    assert mp.lib().mp_transfer_circuit_info(5, None, 6) == -1
    assert mp.lib().mp_transfer_circuit_info(5, ctypes.c_void_p(info.ctypes.data), -1) == -1
    assert not info.any()


_NOALLOC_REJECT = r"""
import ctypes, sys
L = ctypes.CDLL(sys.argv[1])
f = L.mp_minplus_mul_noalloc
P, I64 = ctypes.c_void_p, ctypes.c_int64
f.restype = ctypes.c_int
f.argtypes = [P, P, P, I64, I64, I64, I64, I64, I64, ctypes.c_int, P]
L.mp_last_error.restype = ctypes.c_char_p
big = 200_000  # ceil(200000/128)^2 * 2 mask bytes > 1 MiB
X = 1 << 32    # never dereferenced: the size check comes first
rc = f(X, X + (1 << 40), X + (1 << 41), big, big, big, big, big, big, 0, None)
print(rc, L.mp_last_error().decode())
# a single row against a 2^30 x 2^30 operand: 2^46 mask bytes
K = N = 1 << 30
rc2 = f(X, X + (1 << 40), X + (1 << 33), 1, N, K, K, N, N, 0, None)
print(rc2, L.mp_last_error().decode())
"""


def test_noalloc_rejects_sizes_beyond_its_scratch(mp):
    """The no-allocation product refuses problems whose masks exceed its fixed
    scratch before any CUDA call.  Run with no visible device, so a
    regression of the check would fail with MP_ECUDA and launch nothing."""
    import subprocess
    import sys
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _NOALLOC_REJECT, mp.LIB_PATH], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    rc, msg = lines[0].split(" ", 1)
    assert int(rc) == -1 and "mask bytes" in msg
    rc2, msg2 = lines[1].split(" ", 1)
    assert int(rc2) == -1 and "mask bytes" in msg2


def _fnv1a_words(words):
    h = 1469598103934665603
    for w in words:
        for b in range(4):
            h ^= (int(w) >> (8 * b)) & 0xFF
            h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _checkpoint_bytes(n, k0, count, words, version=1, magic=b"MPPOWERS", extra=0):
    import struct
    N = len(words)
    head = struct.pack("<8sIIiiqqiIQQ", magic, version, 64, n, k0, N, count, 0x7FFF, 1,
                       _fnv1a_words(words), 0)
    assert len(head) == 64
    return head + bytes(2 * count * N * N + extra)


def test_powers_checkpoint_header_is_checked_on_the_host(mp, tmp_path):
    """A powers checkpoint names its path order, first exponent, count, INF
    code and word order, and carries a hash of the word list; the library
    reads it back and refuses files that are not its checkpoints, that were
    written with another word list or version, or whose size does not match
    the header.  Host only: no CUDA call."""
    n = 4
    words = mp.mp_transfer_words(n)
    good = tmp_path / "good.mpp"
    good.write_bytes(_checkpoint_bytes(n, 7, 3, words))
    assert mp.mp_powers_info(str(good)) == {"n": n, "N": len(words), "k0": 7, "count": 3}
    bad = {
        "magic": _checkpoint_bytes(n, 7, 3, words, magic=b"NOTPOWER"),
        "version": _checkpoint_bytes(n, 7, 3, words, version=2),
        "words": _checkpoint_bytes(n, 7, 3, list(words[::-1])),
        "short": _checkpoint_bytes(n, 7, 3, words)[:-2],
        "long": _checkpoint_bytes(n, 7, 3, words, extra=2),
        "header": _checkpoint_bytes(n, 7, 3, words)[:40],
    }
    for name, blob in bad.items():
        f = tmp_path / f"{name}.mpp"
        f.write_bytes(blob)
        with pytest.raises(mp.MinplusError) as e:
            mp.mp_powers_info(str(f))
        assert e.value.code == -9, name
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_powers_info(str(tmp_path / "missing.mpp"))
    assert e.value.code == -9


def test_command_line_lists_its_commands():
    """The package's command line (python -m paper_2409_17688_gb300) parses
    without a GPU and names its commands."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-m", "paper_2409_17688_gb300", "--help"], cwd=ROOT,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    for cmd in ("gamma2", "table", "recurrence", "circuit", "product", "save", "autotune"):
        assert cmd in r.stdout


def test_bounds_checked_build_compiles_and_exports_everything():
    """The -DMP_CHECK variant of the library builds (nvcc cross-compiles it
    without a GPU) and exports every entry point the header declares."""
    from paper_2409_17688_gb300 import _build
    lib = _build.build_library(check=True)
    L = ctypes.CDLL(lib)
    for name in declared_symbols():
        assert hasattr(L, name), name
