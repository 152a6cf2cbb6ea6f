"""GPU parity: the CUDA path against the CPU oracle, bit-exact.

Every comparison is integer equality: every entry of every power, every
product and every gamma_2.  Inputs come from paper_2409_17688_gb300.synth
(seeded) or from the paper's construction; expected values only from oracle/.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2409_17688_gb300 import synth

pytestmark = pytest.mark.gpu

INF = oracle.INF16
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def mp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_17688_gb300 as mp
    mp.lib()
    return mp


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


_ORACLE_G = {}


def oracle_gdiag(n, kmax):
    """min diag A(D_n)^k for k = 1..kmax from the oracle's chain (Algorithm 2
    and Theorem 2), computed once per path order in this module."""
    have = _ORACLE_G.get(n)
    if have is None or have.shape[0] < kmax:
        _, have = oracle.power_sequence(oracle.build_transfer(n), kmax, keep_powers=False,
                                        threads=THREADS)
        _ORACLE_G[n] = have
    return have[:kmax]


# Table 4's (n0, a, b) and Table 5's alpha pattern: gamma_2 = ceil(b m / a) +
# alpha for m >= n0 (Section 4), alpha = 1 exactly for m mod a in the set
CLOSED_FORM = {6: (19, 11, 28, {5, 9}), 7: (23, 18, 53, {1, 2, 4, 5}), 8: (25, 3, 10, set()),
               9: (22, 3, 11, set())}


def closed_form(n, m):
    n0, a, b, ones = CLOSED_FORM[n]
    assert m >= n0
    return -(-b * m // a) + (1 if m % a in ones else 0)


# ------------------------------------------------------------- a1/a2: A(D_n)

@pytest.mark.parametrize("n", list(range(1, 11)))
def test_transfer_matrix(mp, torch, n):
    A, W = mp.mp_build_transfer_matrix(n, words=True)
    torch.cuda.synchronize()
    assert np.array_equal(host(A), oracle.build_transfer(n))
    assert np.array_equal(host(W).astype(np.uint32), mp.mp_transfer_words(n))


def test_transfer_matrix_leading_dimension(mp, torch):
    N = mp.mp_transfer_size(5)
    buf = torch.full((N, N + 13), 77, dtype=torch.int16, device="cuda")
    mp.mp_build_transfer_matrix(5, A=buf)
    torch.cuda.synchronize()
    h = host(buf)
    assert np.array_equal(h[:, :N], oracle.build_transfer(5))
    assert np.all(h[:, N:] == 77)


# ----------------------------------------------------- a5: dense products

SHAPES = [(1, 1, 1), (7, 13, 5), (33, 1, 17), (128, 128, 128), (130, 257, 129),
          (257, 131, 300), (300, 300, 300), (64, 1000, 40), (5, 3000, 7)]


@pytest.mark.parametrize("dtype", [np.int16, np.uint8])
@pytest.mark.parametrize("shape", SHAPES)
def test_minplus_mul_random(mp, torch, dtype, shape):
    M, K, N = shape
    seed = M * 7919 + K * 31 + N
    X = synth.block_inf_matrix(M, K, seed, dtype, inf_frac=0.3, block=32)
    Y = synth.entry_inf_matrix(K, N, seed + 1, dtype, inf_frac=0.2)
    Z = mp.mp_minplus_mul(to_dev(torch, X), to_dev(torch, Y))
    torch.cuda.synchronize()
    assert np.array_equal(host(Z), oracle.minplus_mul(X, Y, threads=THREADS))


@pytest.mark.parametrize("dtype", [np.int16, np.uint8])
def test_minplus_mul_special_values(mp, torch, dtype):
    inf = INF if dtype == np.int16 else 255
    rng = np.random.default_rng(2)
    M, K, N = 150, 260, 140
    # all INF, no INF, near-INF values (saturation), single INF entries
    cases = [np.full((M, K), inf, dtype), rng.integers(0, 5, (M, K)).astype(dtype),
             rng.integers(inf - 3, inf + 1, (M, K)).astype(dtype)]
    Ys = [rng.integers(0, 30, (K, N)).astype(dtype), np.full((K, N), inf, dtype),
          rng.integers(inf - 3, inf + 1, (K, N)).astype(dtype)]
    for X in cases:
        for Y in Ys:
            Z = mp.mp_minplus_mul(to_dev(torch, X), to_dev(torch, Y))
            torch.cuda.synchronize()
            assert np.array_equal(host(Z), oracle.minplus_mul(X, Y))


def test_minplus_mul_whole_inf_blocks(mp, torch):
    """128-aligned all-INF blocks exercise the block-skip path."""
    X = synth.block_inf_matrix(384, 512, 5, np.int16, inf_frac=0.5)
    Y = synth.block_inf_matrix(512, 256, 6, np.int16, inf_frac=0.5)
    Z = mp.mp_minplus_mul(to_dev(torch, X), to_dev(torch, Y))
    torch.cuda.synchronize()
    assert np.array_equal(host(Z), oracle.minplus_mul(X, Y, threads=THREADS))


def test_minplus_mul_strided_and_k0(mp, torch):
    X = synth.entry_inf_matrix(40, 70, 9, np.int16)
    Y = synth.entry_inf_matrix(70, 50, 10, np.int16)
    Xb = torch.zeros((40, 77), dtype=torch.int16, device="cuda")
    Xb[:, :70] = to_dev(torch, X)
    Zb = torch.full((40, 61), 5, dtype=torch.int16, device="cuda")
    mp.mp_minplus_mul(Xb[:, :70], to_dev(torch, Y), Zb[:, :50])
    torch.cuda.synchronize()
    h = host(Zb)
    assert np.array_equal(h[:, :50], oracle.minplus_mul(X, Y))
    assert np.all(h[:, 50:] == 5)
    Z0 = mp.mp_minplus_mul(torch.zeros((4, 0), dtype=torch.int16, device="cuda"),
                           torch.zeros((0, 6), dtype=torch.int16, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(host(Z0) == INF)


def test_minplus_mul_alias_rejected(mp, torch):
    X = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
    Y = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_minplus_mul(X, Y, X)
    assert e.value.code == -2


@pytest.mark.parametrize("dtype", [np.int16, np.uint8])
def test_minplus_mul_8192_sampled(mp, torch, dtype):
    """The N = 8192 product with 40% INF 128-blocks, checked on sampled rows
    and columns (each computed by the oracle on its own)."""
    N = 8192
    X = synth.block_inf_matrix(N, N, 1, dtype, inf_frac=0.4)
    Y = synth.block_inf_matrix(N, N, 2, dtype, inf_frac=0.4)
    Z = host(mp.mp_minplus_mul(to_dev(torch, X), to_dev(torch, Y)))
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, N - 1], rng.choice(N, 14, replace=False)])
    cols = np.concatenate([[0, N - 1], rng.choice(N, 6, replace=False)])
    for i in rows:
        assert np.array_equal(Z[i:i + 1], oracle.minplus_mul(X[i:i + 1], Y, threads=THREADS)), i
    for j in cols:
        assert np.array_equal(Z[:, j:j + 1], oracle.minplus_mul(X, Y[:, j:j + 1], threads=THREADS)), j


# ------------------------------------------------- a3/a4: the power chain

@pytest.mark.parametrize("n,kmax", [(1, 40), (2, 60), (3, 30), (4, 50), (5, 80), (6, 200), (7, 200)])
def test_transfer_chain_every_power(mp, torch, n, kmax):
    """Every entry of every power and every min-diagonal, bit-exact."""
    P, g = mp.mp_transfer_power_sequence(n, kmax)
    torch.cuda.synchronize()
    A = oracle.build_transfer(n)
    Po, go = oracle.power_sequence(A, kmax, left_mul=True, threads=THREADS)
    assert np.array_equal(host(g), go)
    Ph = host(P)
    for k in range(kmax):
        assert np.array_equal(Ph[k], Po[k]), k + 1


def test_transfer_chain_graph_replay(mp, torch):
    """The same chain into the same buffers runs directly, then is captured
    into a CUDA graph, then replayed; every run gives the oracle's powers."""
    import ctypes
    n, kmax = 6, 40
    N = mp.mp_transfer_size(n)
    P = torch.empty((kmax, N, N), dtype=torch.int16, device="cuda")
    g = torch.empty(kmax, dtype=torch.int32, device="cuda")
    Po, go = oracle.power_sequence(oracle.build_transfer(n), kmax, threads=THREADS)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for rep in range(4):
        P.fill_(0)
        g.fill_(-1)
        mp._check(mp.lib().mp_transfer_power_sequence(n, kmax, ctypes.c_void_p(P.data_ptr()),
                                                      ctypes.c_void_p(g.data_ptr()), s))
        torch.cuda.synchronize()
        assert np.array_equal(host(P), Po), rep
        assert np.array_equal(host(g), go), rep


@pytest.mark.parametrize("n,kmax", [(1, 2), (2, 3), (4, 2), (6, 1), (7, 3), (8, 2)])
def test_full_powers_short_chains(mp, torch, n, kmax):
    """Full powers for the shortest chains, where the mirrored form stages a
    single power or none (k_max = 1 takes A itself): every entry against the
    oracle, on odd and even N."""
    P, g = mp.mp_transfer_power_sequence(n, kmax)
    torch.cuda.synchronize()
    Po, go = oracle.power_sequence(oracle.build_transfer(n), kmax, threads=THREADS)
    assert np.array_equal(host(P), Po)
    assert np.array_equal(host(g), go)
    assert mp.mp_device_status() == 0


@pytest.mark.parametrize("n", [8, 9])
def test_transfer_chain_sampled_rows(mp, torch, n):
    """n = 8, 9 with k_max = 200: every power on sampled rows (the oracle's own
    row chain), every min-diagonal (the oracle's chain, the diagonals of the
    GPU powers themselves and Section 4's closed form), and Table 4's
    whole-matrix identity A^{n0+a} = b + A^{n0} on the GPU powers."""
    kmax = 200
    P, g = mp.mp_transfer_power_sequence(n, kmax)
    torch.cuda.synchronize()
    A = oracle.build_transfer(n)
    N = A.shape[0]
    rng = np.random.default_rng(n)
    rows = np.unique(np.concatenate([[0, N - 1], rng.choice(N, 62, replace=False)]))
    R = oracle.power_rows(A, rows, kmax, threads=THREADS)
    for t, i in enumerate(rows):
        got = host(P[:, i, :])
        assert np.array_equal(got, R[t]), i
    # every min-diagonal to k = 200 against the oracle's chain, and against
    # the diagonals of the GPU's own powers
    gh = host(g)
    assert np.array_equal(gh, oracle_gdiag(n, kmax))
    diag = torch.diagonal(P, dim1=1, dim2=2).min(dim=1).values.to(torch.int32)
    assert np.array_equal(host(diag), gh)
    # Section 4's closed form for every m from n0 to k_max
    for m in range(CLOSED_FORM[n][0], kmax + 1):
        assert int(gh[m - 1]) == closed_form(n, m), m
    n0, a, b = {8: (25, 3, 10), 9: (22, 3, 11)}[n]
    lhs = P[n0 + a - 1].to(torch.int32)
    rhs = P[n0 - 1].to(torch.int32) + b
    assert bool(torch.equal(lhs, rhs))
    # Lemma 1: the relation propagates to every later power
    assert bool(torch.equal(P[kmax - 1].to(torch.int32), P[kmax - 1 - a].to(torch.int32) + b))


_GATHER_PLAN_SCRIPT = r"""
import sys
import numpy as np
import torch
import paper_2409_17688_gb300 as mp
out = sys.argv[1]
P, g = mp.mp_transfer_power_sequence(6, 40)
_, g9 = mp.mp_transfer_power_sequence(9, 60, keep_powers=False)
torch.cuda.synchronize()
np.savez(out, P=P.cpu().numpy(), g=g.cpu().numpy(), g9=g9.cpu().numpy())
"""


def test_gather_plan_steps_without_circuit(mp, torch, tmp_path):
    """With MP_SPARSE_CIRCUIT=0 the transfer steps run on the gather plan
    (the cluster kernel) instead of the reuse circuit; a full chain and a
    mirror-column chain still give the oracle's powers and diagonals."""
    import subprocess
    import sys
    out = str(tmp_path / "gather.npz")
    env = dict(os.environ, MP_SPARSE_CIRCUIT="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _GATHER_PLAN_SCRIPT, out], env=env, cwd=root,
                       capture_output=True, timeout=600)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    got = np.load(out)
    Po, go = oracle.power_sequence(oracle.build_transfer(6), 40, threads=THREADS)
    assert np.array_equal(got["P"], Po) and np.array_equal(got["g"], go)
    _, g9 = oracle.power_sequence(oracle.build_transfer(9), 60, keep_powers=False, threads=THREADS)
    assert np.array_equal(got["g9"], g9)


def test_circuit_info(mp):
    """Path orders whose column chunk fits shared memory (n <= 9) run on the
    reuse circuit in shared memory (8-column chunks), larger ones on the
    circuit in global memory (chunks of 32 to 256 columns); both read far
    fewer rows than the arcs.  At n = 3 no cover pays for the level it adds:
    every row is read directly."""
    for n in (3, 6, 9):
        c = mp.mp_transfer_circuit_info(n)
        A = oracle.build_transfer(n)
        assert c["N"] == A.shape[0] and c["nnz"] == int((A < INF).sum())
        assert c["width"] == 8 and c["levels"] >= 1
        assert 0 <= c["cover_reads"] < c["reads"] <= c["nnz"]
        assert (c["cover_reads"] > 0) == (n > 3)
    assert mp.mp_transfer_circuit_info(9)["reads"] * 10 < mp.mp_transfer_circuit_info(9)["nnz"]
    c10 = mp.mp_transfer_circuit_info(10)
    assert c10["width"] in (32, 64, 128, 256) and c10["levels"] >= 1
    assert 0 < c10["cover_reads"] < c10["reads"] and c10["reads"] * 10 < c10["nnz"]


def _large_order_rows(mp, torch, n, kmax, nsample):
    """Powers A^1..A^kmax of a large path order on the GPU, checked on
    sampled rows (first, last and drawn ones) against the oracle's rows,
    which it lists from the word rule without forming A."""
    P, _ = mp.mp_transfer_power_sequence(n, kmax)
    torch.cuda.synchronize()
    N = P.shape[1]
    rng = np.random.default_rng(n)
    rows = np.unique(np.concatenate([[0, N - 1], rng.choice(N, nsample, replace=False)]))
    want = oracle.transfer_power_rows(n, rows, kmax, threads=THREADS)
    for t, i in enumerate(rows):
        assert np.array_equal(host(P[:, i, :]), want[t]), (n, i)
    del P
    torch.cuda.empty_cache()


def test_path_order_12_sampled_rows(mp, torch):
    """n = 12 (N = 52929, 5.6 GB per power): six powers, bit-exact on
    sampled rows against the oracle."""
    N = mp.mp_transfer_size(12)
    free, _ = torch.cuda.mem_get_info()
    if 8 * N * N * 2 * 1.1 > free:
        pytest.skip("not enough device memory for six powers")
    _large_order_rows(mp, torch, 12, 6, 6)


def test_path_order_13_sampled_rows(mp, torch):
    """n = 13 (N = 131562, 34.6 GB per power), the largest path order whose
    powers fit one GPU: four powers (138 GB) bit-exact on sampled rows
    against the oracle.  Skipped only where the device has too little free
    memory."""
    torch.cuda.empty_cache()
    N = mp.mp_transfer_size(13)
    free, _ = torch.cuda.mem_get_info()
    if 6 * N * N * 2 * 1.05 > free:
        pytest.skip("not enough device memory for four powers and the chain buffers")
    _large_order_rows(mp, torch, 13, 4, 4)


@pytest.mark.parametrize("n,kmax,cut", [(6, 40, 17), (9, 30, 12), (10, 12, 5)])
def test_checkpoint_and_resume(mp, torch, tmp_path, n, kmax, cut):
    """Checkpoint and resume (the paper keeps its powers on disk): powers
    A^(cut-2)..A^cut saved, read back bit for bit, and the chain resumed from
    the last of them equals the uninterrupted chain, powers and diagonal
    minima, on the reuse circuit (n = 6, 9) and the gather plan (n = 10), in
    full and mirror-column form; the diagonals equal the oracle's."""
    P, g = mp.mp_transfer_power_sequence(n, kmax)
    torch.cuda.synchronize()
    path = str(tmp_path / f"powers{n}.mpp")
    mp.mp_powers_save(path, n, cut - 2, P[cut - 3:cut])
    assert mp.mp_powers_info(path) == {"n": n, "N": P.shape[1], "k0": cut - 2, "count": 3}
    L, h = mp.mp_powers_load(path)
    torch.cuda.synchronize()
    assert torch.equal(L, P[cut - 3:cut])
    R, gr = mp.mp_transfer_power_sequence_from(n, cut, L[-1].contiguous(), kmax)
    _, gn = mp.mp_transfer_power_sequence_from(n, cut, L[-1].contiguous(), kmax, keep_powers=False)
    torch.cuda.synchronize()
    assert torch.equal(R, P[cut:]), n
    assert torch.equal(gr, g[cut:]) and torch.equal(gn, g[cut:]), n
    if n <= 9:
        assert np.array_equal(host(gn), oracle_gdiag(n, kmax)[cut:]), n
    del P, R, L
    torch.cuda.empty_cache()


def test_power_sequence_generic_matches_transfer(mp, torch):
    """The generic entry point on the dense A(D_n) (it detects the
    column-constant labels) agrees with the transfer chain and the oracle."""
    n, kmax = 6, 40
    A = mp.mp_build_transfer_matrix(n)
    P, g = mp.mp_minplus_power_sequence(A, kmax)
    P2, g2 = mp.mp_transfer_power_sequence(n, kmax)
    torch.cuda.synchronize()
    Po, go = oracle.power_sequence(oracle.build_transfer(n), kmax, threads=THREADS)
    assert np.array_equal(host(P), Po) and np.array_equal(host(g), go)
    assert torch.equal(P, P2) and torch.equal(g, g2)


@pytest.mark.parametrize("N,density,seed", [(50, 0.1, 1), (300, 0.05, 2), (700, 0.02, 3),
                                            (129, 0.2, 4)])
def test_power_sequence_sparse_general(mp, torch, N, density, seed):
    """A sparse A with arbitrary labels (per-entry add-min path)."""
    A = synth.entry_inf_matrix(N, N, seed, np.int16, inf_frac=1 - density, lo=0, hi=9)
    kmax = 12
    P, g = mp.mp_minplus_power_sequence(to_dev(torch, A), kmax)
    torch.cuda.synchronize()
    Po, go = oracle.power_sequence(A, kmax, threads=THREADS)
    assert np.array_equal(host(P), Po)
    assert np.array_equal(host(g), go)


def test_power_sequence_dense(mp, torch):
    A = synth.entry_inf_matrix(200, 200, 8, np.int16, inf_frac=0.3, lo=0, hi=9)
    P, g = mp.mp_minplus_power_sequence(to_dev(torch, A), 6)
    torch.cuda.synchronize()
    Po, go = oracle.power_sequence(A, 6, threads=THREADS)
    assert np.array_equal(host(P), Po) and np.array_equal(host(g), go)


def test_power_sequence_without_powers(mp, torch):
    _, g = mp.mp_transfer_power_sequence(7, 120, keep_powers=False)
    torch.cuda.synchronize()
    _, go = oracle.power_sequence(oracle.build_transfer(7), 120, keep_powers=False, threads=THREADS)
    assert np.array_equal(host(g), go)


# ------------------------------------------------------------ K3, a6

def test_diag_min_and_min_trace(mp, torch):
    rng = np.random.default_rng(12)
    for N in (1, 31, 33, 100, 257):
        X = synth.entry_inf_matrix(N, N, N, np.int16, inf_frac=0.3)
        Y = synth.entry_inf_matrix(N, N, N + 1, np.int16, inf_frac=0.3)
        d = mp.mp_diag_min(to_dev(torch, X))
        t = mp.mp_min_trace(to_dev(torch, X), to_dev(torch, Y))
        torch.cuda.synchronize()
        assert int(host(d)[0]) == oracle.diag_min(X)
        assert int(host(t)[0]) == oracle.diag_min(oracle.minplus_mul(X, Y))


@pytest.mark.parametrize("n,m", [(1, 3), (1, 101), (2, 7), (3, 12), (4, 5), (5, 37), (6, 64),
                                 (7, 100), (7, 257), (8, 49), (9, 40)])
def test_gamma2_cylinder(mp, n, m):
    assert mp.mp_gamma2_cylinder(n, m) == oracle.gamma2(n, m, threads=THREADS)


def test_gamma2_cylinder_large_m_uses_recurrence_identity(mp):
    """Large m, answered through the cached recurrence (Theorem 3), against
    Table 4/5's closed form: gamma_2 = ceil(b m / a) + alpha for m >= n0
    (Section 4)."""
    import math
    cases = {3: (6, 8, set()), 8: (3, 10, set()), 9: (3, 11, set())}
    for n, (a, b, ones) in cases.items():
        for m in (500, 1000, 1024, 2000):
            want = math.ceil(b * m / a) + (1 if (m % a) in ones else 0)
            assert mp.mp_gamma2_cylinder(n, m) == want, (n, m)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 6, 7, 8])
def test_gamma2_squaring(mp, n):
    """Repeated squaring with the min-trace (Theorem 2, Lemma 1's power
    algebra) against the oracle's chain: powers of two, which take the
    square-only branch, and cycle lengths with several set bits."""
    ms = [3, 4, 5, 8, 16, 32, 37, 63, 64, 100]
    g = oracle_gdiag(n, max(ms))
    for m in ms:
        assert mp.mp_gamma2_squaring(n, m) == int(g[m - 1]), (n, m)


def test_gamma2_squaring_large_orders(mp):
    """n = 9 and 10 by squaring (dense N^3 products on N = 3447 and 8568)
    against Section 4's closed form (n = 9) and the recurrence (n = 10)."""
    for m in (64, 101):
        assert mp.mp_gamma2_squaring(9, m) == closed_form(9, m), m
    assert mp.mp_gamma2_squaring(10, 99) == mp.mp_gamma2_cylinder(10, 99)
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_gamma2_squaring(3, 2)
    assert e.value.code == -1
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_gamma2_squaring(10, 4000)
    assert e.value.code == -4


def test_gamma2_cylinder_errors(mp):
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_gamma2_cylinder(3, 2)
    assert e.value.code == -1
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_gamma2_cylinder(0, 10)
    assert e.value.code == -1
    # a table past the int16 range is refused rather than saturated
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_gamma2_table(10, 4000)
    assert e.value.code == -4


# ------------------------------------------------- NEXT f1: recurrence

def test_diff_const_kernel(mp, torch):
    rng = np.random.default_rng(21)
    for N in (1, 7, 130, 513):
        X = synth.entry_inf_matrix(N, N, N, np.int16, inf_frac=0.2)
        cases = [np.where(X < INF, X + 5, INF).astype(np.int16),           # constant shift
                 np.where(X < INF, X + rng.integers(0, 2, X.shape), INF).astype(np.int16),
                 np.full_like(X, INF), X.copy()]
        cases[3].flat[0] = INF if cases[3].flat[0] != INF else 3          # INF pattern differs
        for Y in cases:
            d = host(mp.mp_diff_const(to_dev(torch, Y), to_dev(torch, X)))
            ok, b = oracle.diff_is_constant(Y, X)
            got = bool(d[2] == 0 and d[3] == 1 and d[0] == d[1])
            assert got == ok, N
            if ok:
                assert d[0] == b


T3 = {2: (48, 2, 2), 3: (44, 6, 8), 4: (42, 8, 14), 5: (43, 7, 15), 6: (39, 11, 28),
      7: (32, 18, 53), 8: (47, 3, 10), 9: (47, 3, 11), 10: (47, 3, 12), 11: (47, 3, 13)}
T4_N0 = {2: 4, 3: 7, 4: 9, 5: 31, 6: 19, 7: 23, 8: 25, 9: 22, 10: 21, 11: 24}


@pytest.mark.parametrize("n", list(range(2, 12)))
def test_recurrence_tables_3_4(mp, torch, n):
    """Algorithms 3 and 4 on the device over K = 50 powers reproduce the
    paper's Table 3 (r0, a, b) and Table 4 (n0), n = 2..11 (n = 10, 11 are
    pinned by the paper's printed values alone)."""
    N = mp.mp_transfer_size(n)
    free, _ = torch.cuda.mem_get_info()
    if 50 * N * N * 2 * 1.2 > free:
        pytest.skip("not enough device memory for 50 powers")
    r0, a, b, n0 = mp.mp_transfer_recurrence(n, 50)
    assert (r0, a, b) == T3[n]
    assert n0 == T4_N0[n]


@pytest.mark.parametrize("n", [3, 5, 7, 9, 11, 12])
def test_recurrence_streaming_table_4(mp, torch, n):
    """The ring-buffer form finds Table 4's (n0, a, b) keeping only 20
    powers; for n = 12 (N = 52929, 5.6 GB per power) that is the paper's
    printed row, which its own GPU reached only through 50 stored powers."""
    T4 = {3: (7, 6, 8), 5: (31, 7, 15), 7: (23, 18, 53), 9: (22, 3, 11), 11: (24, 3, 13),
          12: (26, 3, 14)}
    N = mp.mp_transfer_size(n)
    free, _ = torch.cuda.mem_get_info()
    if 23 * N * N * 2 * 1.1 > free:
        pytest.skip("not enough device memory for the ring")
    n0, a, b, k = mp.mp_transfer_recurrence_stream(n, 64, 20)
    assert (n0, a, b) == T4[n]
    assert k == n0 + a


def test_recurrence_stream_twice_with_large_ring(mp, torch):
    """Two streaming detections back to back whose ring takes most of the
    free memory: the first call's buffers go back to the device's memory pool
    and must not make the second call's memory check fail."""
    N = mp.mp_transfer_size(12)
    free, _ = torch.cuda.mem_get_info()
    R = int(free / (N * N * 2))  # narrow ring slots: a little over half of that
    if R < 4:
        pytest.skip("not enough device memory")
    for _ in range(2):
        n0, a, b, k = mp.mp_transfer_recurrence_stream(12, 40, R)
        assert (n0, a, b) == (26, 3, 14)


def test_column_blocks_match_the_whole_width(mp, torch):
    """Chains whose buffers do not fit run over blocks of columns (column
    chunks of a power depend only on the same chunks of the previous power).
    With most of the device memory held elsewhere, the gamma_2 table and the
    ring detection of n = 12 run in blocks and give the whole-width table and
    Table 4's (n0, a, b) = (26, 3, 14)."""
    want = mp.mp_gamma2_table(12, 40)
    assert mp.mp_transfer_recurrence_stream(12, 40, 8)[:3] == (26, 3, 14)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 12e9:
        pytest.skip("not enough device memory to set aside")
    hold = torch.empty(int(free - 4e9), dtype=torch.uint8, device="cuda")
    try:
        got = mp.mp_gamma2_table(12, 40)
        rec = mp.mp_transfer_recurrence_stream(12, 40, 8)
    finally:
        del hold
        torch.cuda.empty_cache()
    assert np.array_equal(got, want)
    assert rec[:3] == (26, 3, 14) and rec[3] == 29


def test_path_order_14(mp, torch):
    """Path order 14 (N = 327006, about 4.7e8 arcs; the two mirror-column
    chain buffers alone would take 214 GB), beyond the paper's reach: the
    chain and the ring detection run over column blocks.  Pins are the
    paper's statements: the C_5 formula 2n + 2 = 30 for even n (Section 4),
    the conjecture gamma_2 = (n + 2) m / 3 = 16 m / 3 for m = 0 mod 3
    (Section 5) and so the period's slope b / a = 16 / 3; Theorem 3 carries
    them to m = 3000.  Skipped only where the device has too little memory."""
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 120e9:
        pytest.skip("not enough free device memory for path order 14")
    n0, a, b, k = mp.mp_transfer_recurrence_stream(14, 48, 4)
    assert a > 0 and k == n0 + a
    assert 3 * b == 16 * a
    assert mp.mp_gamma2_cylinder(14, 5) == 30
    for m in range(3, 3001, 3):
        assert mp.mp_gamma2_cylinder(14, m) == 16 * m // 3, m


def test_path_order_13_conjecture(mp, torch):
    """Path order 13 (N = 131562, 34.6 GB per power), which the paper could
    not fit: the ring-buffer detector keeps four powers and the two chain
    buffers (about 208 GB).  Pins are the paper's statements: its conjecture
    (Section 5) gamma_2(P_n x C_m) = (n + 2) m / 3 for n >= 8 and m = 0 mod 3,
    the C_5 formula 2n + 1 for odd n (Section 4), and so the period's slope
    b / a = (n + 2) / 3.  About a minute; skipped only where the device has
    too little free memory."""
    torch.cuda.empty_cache()
    try:
        n0, a, b, k = mp.mp_transfer_recurrence_stream(13, 64, 4)
    except mp.MinplusError as e:
        if e.code == -3:
            pytest.skip("not enough free device memory for four powers of N = 131562")
        raise
    assert a > 0 and k == n0 + a
    assert 3 * b == 15 * a
    assert mp.mp_gamma2_cylinder(13, 5) == 27
    for m in range(3, 3001, 3):
        assert mp.mp_gamma2_cylinder(13, m) == 5 * m, m


def test_gamma2_any_m_by_recurrence(mp):
    """Theorem 3 answers every m, past the int16 range too: the closed form
    of Section 4 with Table 5's alpha, m from n0 to 10^5."""
    import math
    alpha_ones = {2: (2, set()), 3: (6, set()), 4: (8, {4, 5}), 5: (7, set()), 6: (11, {5, 9}),
                  7: (18, {1, 2, 4, 5}), 8: (3, set()), 9: (3, set()), 10: (3, {1, 2}),
                  11: (3, {2})}
    for n in range(2, 12):
        a, ones = alpha_ones[n]
        b = T3[n][2]
        for m in [T4_N0[n], T4_N0[n] + 1, 97, 1000, 4001, 33333, 100000]:
            want = math.ceil(b * m / a) + (1 if (m % a) in ones else 0)
            assert mp.mp_gamma2_cylinder(n, m) == want, (n, m)


# ------------------------------------------------------------------ a7

@pytest.mark.parametrize("mode", [0, 1])
def test_batched_matches_single(mp, torch, mode):
    sizes = [64, 100, 129, 300, 517, 77, 1000]
    probs, want = [], []
    for i, N in enumerate(sizes):
        dt = np.int16 if i % 3 else np.uint8
        X = synth.block_inf_matrix(N, N, 100 + i, dt, inf_frac=0.3)
        Y = synth.block_inf_matrix(N, N, 200 + i, dt, inf_frac=0.3)
        Xd, Yd = to_dev(torch, X), to_dev(torch, Y)
        Zd = torch.empty_like(Xd)
        probs.append((Xd, Yd, Zd))
        want.append(oracle.minplus_mul(X, Y, threads=THREADS))
    mp.mp_minplus_mul_batched(probs, mode=mode)
    torch.cuda.synchronize()
    for (_, _, Zd), w in zip(probs, want):
        assert np.array_equal(host(Zd), w)


def test_batched_empty_and_rectangular(mp, torch):
    """Degenerate and rectangular products in one persistent launch: M = 0
    (nothing written), K = 0 (all INF), 1 x 1, and non-square shapes that
    leave ragged tiles in every dimension; an empty batch is a no-op."""
    mp.mp_minplus_mul_batched([])
    shapes = [(0, 5, 7, np.int16), (6, 0, 9, np.int16), (1, 1, 1, np.uint8),
              (130, 70, 300, np.int16), (257, 129, 65, np.uint8), (64, 1000, 3, np.int16)]
    probs, want = [], []
    for i, (M, K, N, dt) in enumerate(shapes):
        X = synth.entry_inf_matrix(M, K, 300 + i, dt, inf_frac=0.2)
        Y = synth.entry_inf_matrix(K, N, 400 + i, dt, inf_frac=0.2)
        Zd = torch.full((M, N), 7, dtype=torch.int16 if dt == np.int16 else torch.uint8,
                        device="cuda")
        probs.append((to_dev(torch, X), to_dev(torch, Y), Zd))
        want.append(oracle.minplus_mul(X, Y, threads=THREADS) if M and N else None)
    for mode in (0, 1):
        for _, _, Zd in probs:
            Zd.fill_(7)
        mp.mp_minplus_mul_batched(probs, mode=mode)
        torch.cuda.synchronize()
        for (_, _, Zd), w in zip(probs, want):
            if w is not None:
                assert np.array_equal(host(Zd), w), (mode, Zd.shape)
    assert np.all(host(probs[1][2]) == INF)  # K = 0: every entry is an empty minimum


@pytest.mark.slow
def test_batched_full_workload_sampled(mp, torch):
    """The bench's batched workload at full size (96 square products, N
    log-uniform in [64, 8192], 30% INF 128-blocks, the same seeds), run the
    way it is timed: autotuned tile table, one persistent launch captured in
    a CUDA graph and replayed.  Three rows of every product (first, last and
    one drawn) equal the oracle's product of those rows with Y."""
    sizes = synth.batch_sizes(96, 64, 8192, seed=7)
    probs, hosts = [], []
    for i, N in enumerate(sizes):
        X = synth.block_inf_matrix(N, N, 1000 + 2 * i, np.int16, inf_frac=0.3)
        Y = synth.block_inf_matrix(N, N, 1001 + 2 * i, np.int16, inf_frac=0.3)
        Xd = to_dev(torch, X)
        probs.append((Xd, to_dev(torch, Y), torch.full_like(Xd, 5)))
        hosts.append((X, Y))
    mp.mp_autotune()
    batch = mp.Batch(probs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.run(0)
    torch.cuda.synchronize()
    for _, _, Zd in probs:
        Zd.fill_(5)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.run(0, stream=s)
    g.replay()
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(99))
    for (X, Y), (_, _, Zd) in zip(hosts, probs):
        N = X.shape[0]
        rows = sorted({0, N - 1, int(rng.integers(0, N))})
        got = host(Zd[rows])
        for j, r in enumerate(rows):
            assert np.array_equal(got[j], oracle.minplus_mul(X[r:r + 1], Y, threads=THREADS)[0]), (N, r)
    del batch


def test_batched_alias_rejected(mp, torch):
    X = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
    Z = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_minplus_mul_batched([(X, X, Z), (Z, X, X.clone())])
    assert e.value.code == -2


@pytest.mark.parametrize("shape_cfg", [0, 1])
@pytest.mark.parametrize("dtype", [np.int16, np.uint8])
def test_each_tile_shape(mp, torch, shape_cfg, dtype):
    """Both tile shapes (128x128 and 64x64) on ragged sizes, forced for every
    size class through the tuning table."""
    saved = mp.mp_tuning_get()
    try:
        mp.mp_tuning_set(np.full((2, 6), shape_cfg, dtype=np.int32))
        for M, K, N in [(1, 1, 1), (63, 65, 64), (130, 257, 129), (300, 200, 517)]:
            X = synth.block_inf_matrix(M, K, M + K, dtype, inf_frac=0.3, block=64)
            Y = synth.entry_inf_matrix(K, N, N + K, dtype, inf_frac=0.2)
            Z = mp.mp_minplus_mul(to_dev(torch, X), to_dev(torch, Y))
            torch.cuda.synchronize()
            assert np.array_equal(host(Z), oracle.minplus_mul(X, Y, threads=THREADS)), (M, K, N)
    finally:
        mp.mp_tuning_set(saved)


def test_batch_graph_replay(mp, torch):
    """A prepared batch captured in a CUDA graph: every replay, in both modes,
    gives the oracle's products; operands changed between replays are seen."""
    sizes = [64, 100, 129, 200, 517, 1000, 70]
    Xs, Ys, Zs, probs = [], [], [], []
    for i, N in enumerate(sizes):
        X = synth.block_inf_matrix(N, N, 300 + i, np.int16, inf_frac=0.3)
        Y = synth.block_inf_matrix(N, N, 400 + i, np.int16, inf_frac=0.3)
        Xs.append(to_dev(torch, X)); Ys.append(to_dev(torch, Y)); Zs.append(torch.empty_like(Xs[-1]))
        probs.append((Xs[-1], Ys[-1], Zs[-1]))
    b = mp.Batch(probs)
    for mode in (0, 1):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b.run(mode)  # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.run(mode, stream=s)
        for rep in range(2):
            for i, N in enumerate(sizes):  # new operand values, same buffers
                Xs[i].copy_(to_dev(torch, synth.block_inf_matrix(N, N, 500 + 10 * rep + i, np.int16, inf_frac=0.3)))
                Zs[i].fill_(1)
            g.replay()
            torch.cuda.synchronize()
            for i in range(len(sizes)):
                assert np.array_equal(host(Zs[i]), oracle.minplus_mul(host(Xs[i]), host(Ys[i]), threads=THREADS))
    b.close()


def test_autotune_installs_a_valid_table(mp):
    saved = mp.mp_tuning_get()
    try:
        t = mp.mp_autotune()
        assert t.shape == (2, 6) and set(np.unique(t)) <= {0, 1}
        assert np.array_equal(mp.mp_tuning_get(), t)
    finally:
        mp.mp_tuning_set(saved)


# ----------------------------------------------- failures made on the host

def test_allocation_failures_are_reported(mp, torch):
    """Requests that cannot fit the device come back as MP_ENOMEM, checked
    before any kernel runs; the context stays usable afterwards."""
    free, _ = torch.cuda.mem_get_info()
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_transfer_recurrence(12, 200)  # 200 powers of 5.6 GB
    assert e.value.code in (-3, -4)
    with pytest.raises(mp.MinplusError) as e:
        # more ring slots than even one column chunk per slot can hold (twice
        # over: the library's memory pool may keep a reserve that the free
        # figure above does not count)
        mp.mp_transfer_recurrence_stream(12, 60, 2 * int(free // (52929 * 128)) + 8)
    assert e.value.code == -3
    # a server whose budget cannot hold the path order refuses it
    srv = mp.Server(hbm_budget=1 << 20, max_batch=8, max_m=100)
    t = srv.submit(8, 50)
    with pytest.raises(mp.MinplusError) as e:
        srv.wait(t)
    assert e.value.code == -3
    srv.close()
    # the device still works
    assert mp.mp_gamma2_cylinder(4, 5) == 10
    assert mp.mp_device_status() == 0


# --------------------------------------------------------------- misc

def test_dpx_peak_positive(mp):
    """K6: DPX rates (terms/s) and the shared-memory load rate (bytes/s) are
    measured; every one is above 1e12 on a GB300."""
    for v in (0, 1, 2, 3):
        assert mp.mp_dpx_peak(v, 4096) > 1e12


def test_command_line(mp, capsys, tmp_path):
    """The command line answers through the library: gamma_2(P_3 x C_12) = 16
    (ceil(4m/3)) by the chain and by repeated squaring, and a checkpoint it
    writes reads back."""
    import json
    from paper_2409_17688_gb300.__main__ import main
    for extra in ([], ["--squaring"]):
        assert main(["gamma2", "--n", "3", "--m", "12", *extra]) == 0
        assert json.loads(capsys.readouterr().out)["gamma2"] == 16
    path = str(tmp_path / "p.mpp")
    assert main(["save", "--n", "4", "--kmax", "5", "--out", path]) == 0
    out = json.loads(capsys.readouterr().out)
    assert (out["n"], out["k0"], out["count"]) == (4, 1, 5)


def test_device_status_clean(mp):
    assert mp.mp_device_status() == 0


def test_bounded_wait_runs_out_and_reports(mp, torch):
    """The circuit kernel's wait for its copies is bounded: a step whose wait
    expects bytes that never arrive gives up (about two seconds), latches
    MP_ETIMEOUT and returns; the status is read once and cleared, and the
    device computes correctly afterwards.  No fault, trap or hang."""
    assert mp.mp_device_status() == 0
    mp.mp_inject_circuit_timeout(3)
    assert mp.lib().mp_device_status() == -6
    assert mp.mp_device_status() == 0
    _, g = mp.mp_transfer_power_sequence(3, 30, keep_powers=False)
    torch.cuda.synchronize()
    assert np.array_equal(host(g), oracle_gdiag(3, 30))
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_inject_circuit_timeout(10)  # no circuit for N = 8568
    assert e.value.code == -1


def test_gamma2_table(mp):
    for n in (2, 5, 8):
        t = mp.mp_gamma2_table(n, 60)
        assert np.array_equal(t, oracle.gamma2_range(n, 60, threads=THREADS))


def test_several_chains_side_by_side(mp, torch):
    """Chains of several path orders run side by side on library streams give
    the same min-diagonal sequences as one at a time, and the oracle's for
    the small orders; the synchronous tables equal the per-order tables."""
    ns = [9, 3, 6, 1, 8, 7]
    g = mp.mp_transfer_power_sequences(ns, 60)
    torch.cuda.synchronize()
    for i, n in enumerate(ns):
        _, gi = mp.mp_transfer_power_sequence(n, 60, keep_powers=False)
        torch.cuda.synchronize()
        assert torch.equal(g[i], gi), n
        if n <= 6:
            _, go = oracle.power_sequence(oracle.build_transfer(n), 60, keep_powers=False,
                                          threads=THREADS)
            assert np.array_equal(host(g[i]), go), n
    t = mp.mp_gamma2_tables([6, 7, 8, 9], 200)
    for i, n in enumerate([6, 7, 8, 9]):
        assert np.array_equal(t[i], mp.mp_gamma2_table(n, 200)), n
    assert mp.mp_gamma2_tables([], 10).shape == (0, 11)
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_transfer_power_sequences([5, 5], 10)
    assert e.value.code == -1
    with pytest.raises(mp.MinplusError) as e:
        mp.mp_gamma2_tables([5, 12], 3000)  # 12 * 3000 reaches the INF code
    assert e.value.code == -4


def test_gamma2_tables_of_the_timed_workload(mp, torch):
    """The exact call the benchmark times: the gamma_2 tables of n = 6, 7, 8,
    9 to k_max = 200 side by side (mirror-column chains on the reuse
    circuit), every entry against the oracle's chain and, from n0 on, against
    Section 4's closed form with Table 5's alpha."""
    ns, kmax = [6, 7, 8, 9], 200
    t = mp.mp_gamma2_tables(ns, kmax)
    for i, n in enumerate(ns):
        want = np.full(kmax + 1, -1, dtype=np.int64)
        want[3:] = oracle_gdiag(n, kmax)[2:]
        assert np.array_equal(t[i], want), n
        for m in range(CLOSED_FORM[n][0], kmax + 1):
            assert int(t[i][m]) == closed_form(n, m), (n, m)
    # twice more: the second call is captured into graphs, the third replays them
    for _ in range(2):
        assert np.array_equal(mp.mp_gamma2_tables(ns, kmax), t)


def test_side_by_side_chains_mixing_both_circuits(mp, torch):
    """Chains on the shared-memory circuit run in one launch; a set that also
    holds a path order on the global circuit (n = 10) runs on library streams
    instead.  Both give the one-at-a-time minimum diagonals, and the oracle's
    for the small orders."""
    for ns in ([10, 6, 3], [9, 8, 7, 6, 5, 4, 3, 2]):
        g = mp.mp_transfer_power_sequences(ns, 50)
        torch.cuda.synchronize()
        for i, n in enumerate(ns):
            _, gi = mp.mp_transfer_power_sequence(n, 50, keep_powers=False)
            torch.cuda.synchronize()
            assert torch.equal(g[i], gi), (ns, n)
            if n <= 7:
                assert np.array_equal(host(g[i]), oracle_gdiag(n, 50)), (ns, n)


def test_several_chains_in_a_cuda_graph(mp, torch):
    """The side-by-side chains can be captured into a CUDA graph (the library
    streams join the capture through the fork and join events) and replayed;
    every replay gives the one-at-a-time sequences."""
    ns = [8, 6, 7]
    want = [mp.mp_transfer_power_sequence(n, 40, keep_powers=False)[1] for n in ns]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.empty((len(ns), 40), dtype=torch.int32, device="cuda")
    ns_arr = (ctypes.c_int * len(ns))(*ns)
    L = mp.lib()

    def run():
        mp._check(L.mp_transfer_power_sequences(ns_arr, len(ns), 40, ctypes.c_void_p(g.data_ptr()),
                                                ctypes.c_void_p(s.cuda_stream)))

    with torch.cuda.stream(s):
        run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        run()
    for _ in range(2):
        g.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        for i in range(len(ns)):
            assert torch.equal(g[i], want[i]), ns[i]


@pytest.mark.parametrize("n", [2, 5, 7, 8, 9])
def test_mirror_columns_chain_matches_full(mp, torch, n):
    """Without powers to write, the chain keeps one column of every mirror
    pair of words (the reversal symmetry of A(D_n)); its min-diagonals equal
    those of the full chain, which writes every power, and the oracle's, for
    every k up to 200."""
    kmax = 200
    _, g_narrow = mp.mp_transfer_power_sequence(n, kmax, keep_powers=False)
    P, g_full = mp.mp_transfer_power_sequence(n, kmax, keep_powers=True)
    torch.cuda.synchronize()
    assert torch.equal(g_narrow, g_full), n
    assert np.array_equal(host(g_narrow), oracle_gdiag(n, kmax)), n
    # the symmetry itself, on the full powers: P_k[R q][R c] = P_k[q][c]
    words = [int(w) for w in mp.mp_transfer_words(n)]
    index = {w: i for i, w in enumerate(words)}
    R = [index[sum(((w >> (2 * j)) & 3) << (2 * (n - 1 - j)) for j in range(n))] for w in words]
    Rt = torch.tensor(R, device="cuda")
    for k in (1, 7, 80, 200):
        Pk = P[k - 1]
        assert torch.equal(Pk[Rt][:, Rt], Pk), (n, k)


def test_threads_share_the_plan_caches(mp, torch):
    """Host threads asking for the same path orders at once (both chain
    kinds, plans built on first use) get the single-thread results."""
    import threading
    want = {n: mp.mp_gamma2_table(n, 60) for n in (4, 5, 6, 7)}
    results, errors = {}, []

    def work(i):
        try:
            torch.cuda.set_device(0)
            n = 4 + i % 4
            results[i] = mp.mp_gamma2_table(n, 60)
            P, g = mp.mp_transfer_power_sequence(n, 20)
            # this thread's stream only: a device-wide synchronisation would
            # also reach another thread's chain while it is being captured
            # into a graph (the library then runs that chain directly)
            torch.cuda.current_stream().synchronize()
            results[(i, "g")] = (n, host(g))
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i in range(8):
        n = 4 + i % 4
        assert np.array_equal(results[i], want[n]), n
        n2, g = results[(i, "g")]
        assert np.array_equal(g[2:], want[n2][3:21]), n2

