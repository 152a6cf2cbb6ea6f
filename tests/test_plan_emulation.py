"""Host logic of the sparse transfer step: the plan (row groups, stages,
clusters, membership-mask segments, task dealing, unit schedules) is built by
the library's own host code and its semantics are carried out on the CPU by
tests/plan_emulation.cu; every power must equal the oracle's."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def emu():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="planemu")
    exe = os.path.join(d, "plan_emulation")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           os.path.join(HERE, "plan_emulation.cu"),
           os.path.join(ROOT, "paper_2409_17688_gb300", "csrc", "transfer.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


# (n, k, max cluster size, buffer rows): the small buffers force multi-stage
# groups (a row's gathered rows spread over several stages)
CASES = [(1, 12, 3, 648), (3, 20, 3, 648), (5, 10, 3, 648), (5, 10, 4, 648), (6, 8, 1, 648),
         (6, 8, 3, 648), (6, 6, 4, 40), (7, 5, 3, 648), (7, 4, 3, 100), (8, 3, 3, 120)]


@pytest.mark.parametrize("n,k,cl,cap", CASES)
def test_plan_semantics_match_oracle(emu, n, k, cl, cap):
    r = subprocess.run([emu, str(n), str(k), str(cl), str(cap)], capture_output=True)
    assert r.returncode == 0, r.stderr.decode()
    groups, stages = (int(w) for w in r.stderr.decode().split()[1:4:2])
    if cap < 648 and n >= 6:
        assert stages > groups  # the small buffer did split groups into stages
    N = oracle.transfer_size(n)
    got = np.frombuffer(r.stdout, dtype=np.int16).reshape(k, N, N)
    want, _ = oracle.power_sequence(oracle.build_transfer(n), k, threads=os.cpu_count() or 1)
    assert np.array_equal(got, want)
