"""Host logic of the reuse circuit of the sparse transfer step: the circuit
(greedy covers of each row's arcs by the arcs of other rows, levels, slices)
is built by the library's own host code and its semantics are carried out on
the CPU by tests/circuit_emulation.cu; every power must equal the oracle's."""
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
    d = tempfile.mkdtemp(prefix="circemu")
    exe = os.path.join(d, "circuit_emulation")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           os.path.join(HERE, "circuit_emulation.cu"),
           os.path.join(ROOT, "paper_2409_17688_gb300", "csrc", "transfer.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


# (n, k)
CASES = [(1, 6), (2, 8), (3, 20), (4, 12), (5, 10), (6, 8), (7, 5)]


@pytest.mark.parametrize("n,k", CASES)
def test_circuit_semantics_match_oracle(emu, n, k):
    r = subprocess.run([emu, str(n), str(k)], capture_output=True)
    assert r.returncode == 0, (r.returncode, r.stderr.decode())
    stats = r.stderr.decode().split()
    reads, nnz = int(stats[5]), int(stats[9])
    assert reads <= nnz  # a cover never reads more rows than the arcs
    N = oracle.transfer_size(n)
    got = np.frombuffer(r.stdout, dtype=np.int16).reshape(k, N, N)
    want, _ = oracle.power_sequence(oracle.build_transfer(n), k, threads=os.cpu_count() or 1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,k", [(3, 20), (5, 12), (6, 9), (7, 4)])
def test_chain_image_bookkeeping_matches_oracle(emu, n, k):
    """The chain kernel's shared-memory image: result rows from Nh, reads at
    (index + sh) mod 2Nh, labels added in place, regions swapped per step."""
    r = subprocess.run([emu, str(n), str(k), "image"], capture_output=True)
    assert r.returncode == 0, (r.returncode, r.stderr.decode())
    N = oracle.transfer_size(n)
    got = np.frombuffer(r.stdout, dtype=np.int16).reshape(k, N, N)
    want, _ = oracle.power_sequence(oracle.build_transfer(n), k, threads=os.cpu_count() or 1)
    assert np.array_equal(got, want)


def test_circuit_reads_far_fewer_rows_than_arcs(emu):
    # the arc rule nests successor sets: at n = 7 the covers read under a
    # fifth of the arcs
    r = subprocess.run([emu, "7", "2"], capture_output=True)
    assert r.returncode == 0, r.stderr.decode()
    stats = r.stderr.decode().split()
    reads, cover, nnz = int(stats[5]), int(stats[7]), int(stats[9])
    assert cover > 0 and reads * 5 < nnz


@pytest.fixture(scope="module")
def gemu():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="gcircemu")
    exe = os.path.join(d, "gcircuit_emulation")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           os.path.join(HERE, "gcircuit_emulation.cu"),
           os.path.join(ROOT, "paper_2409_17688_gb300", "csrc", "transfer.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("n,k,lanes", [(1, 6, 4), (2, 9, 8), (3, 20, 32), (4, 12, 4), (5, 10, 16),
                                       (6, 8, 8), (7, 5, 4)])
def test_global_circuit_semantics_match_oracle(gemu, n, k, lanes):
    """The global-memory circuit (path orders past shared memory): covers
    from the arc rule (a 0 or 1 of the source word turned into a 2 keeps the
    successors with a 0 there), warp tasks of 32 / lanes rows, entries that
    carry their row's label, rows in the chain's internal order; every power
    equals the oracle's."""
    r = subprocess.run([gemu, str(n), str(k), str(lanes)], capture_output=True)
    assert r.returncode == 0, (r.returncode, r.stderr.decode())
    stats = r.stderr.decode().split()
    reads, nnz = int(stats[5]), int(stats[9])
    assert reads <= nnz
    N = oracle.transfer_size(n)
    got = np.frombuffer(r.stdout, dtype=np.int16).reshape(k, N, N)
    want, _ = oracle.power_sequence(oracle.build_transfer(n), k, threads=os.cpu_count() or 1)
    assert np.array_equal(got, want)


def test_global_circuit_covers_read_few_arcs(gemu):
    # the rule's subsets alone already cover most arcs at n = 7
    r = subprocess.run([gemu, "7", "2", "8"], capture_output=True)
    assert r.returncode == 0, r.stderr.decode()
    stats = r.stderr.decode().split()
    reads, cover, nnz = int(stats[5]), int(stats[7]), int(stats[9])
    assert cover > 0 and reads * 4 < nnz
