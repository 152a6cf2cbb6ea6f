"""The bounds-checked build (-DMP_CHECK).

In that build the circuit kernels check every shared- and global-memory
index they compute (image rows, chunk columns, circuit slices and entries,
caller rows, staged columns); an index outside its buffer latches MP_ECHECK
in the device status word and is replaced by 0, so the access stays in
bounds.  These tests build it and run the chain forms through it: every
result must equal the regular library's (itself compared with the oracle by
the parity tests) and no check may fire.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[2])
import paper_2409_17688_gb300 as mp
mp.LIB_PATH = sys.argv[1]
import run_cases
out = run_cases.run(mp)
out["status"] = np.array([mp.mp_device_status()])
np.savez(sys.argv[3], **out)
"""

_CASES = r'''
import numpy as np


def run(mp):
    """The chain forms of the library: side-by-side gamma_2 tables (the
    multi-chain launch on 16-column chunks), full powers through the narrow
    chain and its mirror copy (8- and 16-column chunks), one chain alone,
    and the global circuit (n = 10)."""
    out = {}
    out["tables"] = np.asarray(mp.mp_gamma2_tables([6, 7, 8, 9], 40))
    for n, k in ((5, 16), (7, 12), (9, 6)):
        P, g = mp.mp_transfer_power_sequence(n, k)
        out[f"P{n}"] = P.cpu().numpy()
        out[f"g{n}"] = g.cpu().numpy()
    _, g9 = mp.mp_transfer_power_sequence(9, 30, keep_powers=False)
    out["g9narrow"] = g9.cpu().numpy()
    _, g10 = mp.mp_transfer_power_sequence(10, 6, keep_powers=False)
    out["g10"] = g10.cpu().numpy()
    return out
'''


@pytest.fixture(scope="module")
def mp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_17688_gb300 as mp
    mp.lib()
    return mp


@pytest.mark.gpu
def test_bounds_checked_build_matches_and_catches_nothing(mp, tmp_path):
    from paper_2409_17688_gb300 import _build
    lib = _build.build_library(check=True)
    (tmp_path / "run_cases.py").write_text(_CASES)
    res = tmp_path / "check.npz"
    env = dict(os.environ, PYTHONPATH=str(tmp_path) + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", _CHILD, lib, ROOT, str(res)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(res)
    assert int(got["status"][0]) == 0, "a bounds check fired"
    sys.path.insert(0, str(tmp_path))
    try:
        import run_cases
        want = run_cases.run(mp)
    finally:
        sys.path.remove(str(tmp_path))
    assert mp.mp_device_status() == 0
    for key, val in want.items():
        assert np.array_equal(got[key], val), key
