"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each compares it with a
printed table of the paper, a closed form stated there, an exhaustive search
from the graph definition, Carre's walk characterisation (Theorem 1), a library
shortest-path routine, or an algebraic identity of the tropical semiring.
"""
import ctypes
import itertools
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from conftest import read_golden

INF = oracle.INF16

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- Table 1

def test_table1_row_counts():
    """Table 1: |C_n| for path orders 2..13 (Section 3)."""
    for n, N, _, _ in read_golden("table1_sizes.txt"):
        assert oracle.transfer_size(int(n)) == int(N), n


def test_table1_memory_column():
    """Table 1 memory column = N^2 * 2 bytes in binary units.  n = 7 is
    printed as 0.69 MB, a misprint of 0.59 MiB."""
    scale = {"KB": 2 ** 10, "MB": 2 ** 20, "GB": 2 ** 30}
    for n, N, mem, unit in read_golden("table1_sizes.txt"):
        got = int(N) ** 2 * 2 / scale[unit]
        if int(n) == 7:
            assert abs(got - 0.59) < 0.01
            continue
        assert abs(got - float(mem)) <= 0.025 * float(mem) + 0.006, (n, got, mem)


# ------------------------------------------------------- words and arcs

def test_words_are_lexicographic_and_distinct():
    for n in range(1, 8):
        W = oracle.enumerate_words(n)
        codes = [int("".join(map(str, w)), 3) for w in W]
        assert codes == sorted(set(codes))


def test_path_order_one_matrix_by_hand():
    """n = 1: words 0, 1, 2.  From the three bullets of Section 2.2: p = 0
    may follow anything; p = 1 needs two zeros among {q} and never can;
    p = 2 needs exactly one zero, i.e. q = 0.  Labels: zeros of p."""
    A = oracle.build_transfer(1)
    expect = np.array([[1, INF, 0], [1, INF, INF], [1, INF, INF]], dtype=np.int16)
    assert np.array_equal(A, expect)


def test_arc_labels_are_zero_counts_of_target():
    """The label of arc (q, p) depends only on p (Section 2.2)."""
    for n in (2, 3, 4, 5):
        A = oracle.build_transfer(n)
        W = oracle.enumerate_words(n)
        for j in range(A.shape[1]):
            col = A[:, j]
            fin = col[col < INF]
            assert np.all(fin == np.sum(W[j] == 0))


# ------------------------------------------------------ brute force pins

@pytest.fixture(scope="module")
def brute():
    src = os.path.join(HERE, "brute_gamma2.c")
    d = tempfile.mkdtemp(prefix="brute")
    so = os.path.join(d, "brute.so")
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.brute_gamma2.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.brute_gamma2.restype = ctypes.c_int
    return lib.brute_gamma2


def test_exhaustive_subset_search(brute):
    """gamma_2 from the oracle's chain equals exhaustive search over vertex
    subsets of P_n x C_m for every cylinder with n*m <= 24."""
    for n in range(1, 9):
        A = oracle.build_transfer(n)
        mmax = 24 // n
        if mmax < 3:
            continue
        _, g = oracle.power_sequence(A, mmax, keep_powers=False)
        for m in range(3, mmax + 1):
            assert g[m - 1] == brute(n, m), (n, m)


def test_example1_p4_c5(brute):
    """Example 1: a 2-dominating set of P_4 x C_5 with 10 vertices exists;
    exhaustive search shows none is smaller."""
    g = oracle.gamma2(4, 5)
    assert g <= 10
    assert g == brute(4, 5) == 10


def _subset_pair_gamma2(n, mmax):
    """gamma_2(P_n x C_m), m = 3..mmax, from a second transfer construction
    that shares nothing with the paper's words: a state is the pair
    (D_prev, D_cur) of column subsets in the dominating set, a step to
    (D_cur, D_next) is allowed when every vertex of the current column outside
    D_cur has at least two neighbours in D (up and down in D_cur, left in
    D_prev, right in D_next), and it costs |D_next|.  A 2-dominating set of
    the cylinder is a closed walk of m steps, so gamma_2 is the least diagonal
    entry of the m-th (min,+) power."""
    S = 1 << n
    big = 1 << 20
    pop = np.array([bin(d).count("1") for d in range(S)], dtype=np.int64)
    cover_ok = np.zeros((S, S, S), dtype=bool)  # [prev, cur, next]
    for prev, cur, nxt in itertools.product(range(S), repeat=3):
        ok = True
        for r in range(n):
            if cur >> r & 1:
                continue
            cnt = (prev >> r & 1) + (nxt >> r & 1)
            cnt += (r > 0 and cur >> (r - 1) & 1) + (r < n - 1 and cur >> (r + 1) & 1)
            if cnt < 2:
                ok = False
                break
        cover_ok[prev, cur, nxt] = ok
    B = np.full((S * S, S * S), big, dtype=np.int64)
    for prev, cur, nxt in zip(*np.nonzero(cover_ok)):
        B[prev * S + cur, cur * S + nxt] = pop[nxt]
    out, P = {}, B.copy()
    for m in range(2, mmax + 1):
        P = np.min(P[:, :, None] + B[None, :, :], axis=1) if S <= 8 else \
            np.stack([np.min(P[i][:, None] + B, axis=0) for i in range(S * S)])
        np.minimum(P, big, out=P)
        if m >= 3:
            out[m] = int(P.diagonal().min())
    return out


@pytest.mark.parametrize("n,mmax", [(1, 12), (2, 12), (3, 12), (4, 10), (5, 6)])
def test_subset_pair_construction(n, mmax):
    """The oracle's gamma_2 (the paper's correct words and arc rules, Section
    2.2, with Theorem 2) equals the subset-pair transfer construction."""
    want = _subset_pair_gamma2(n, mmax)
    got = oracle.gamma2_range(n, mmax)
    for m in range(3, mmax + 1):
        assert got[m] == want[m], (n, m)


def test_cycle_closed_form():
    """Path order 1 is the cycle C_m, whose 2-domination number is ceil(m/2)."""
    g = oracle.gamma2_range(1, 60)
    for m in range(3, 61):
        assert g[m] == (m + 1) // 2


# --------------------------------------------------------- Tables 3, 4, 5

def _powers(n, K=50, threads=None):
    A = oracle.build_transfer(n)
    P, g = oracle.power_sequence(A, K, keep_powers=True, left_mul=True,
                                 threads=threads or os.cpu_count() or 1)
    return A, P, g


T3 = {int(r[0]): tuple(map(int, r[1:])) for r in read_golden("table3_recurrence.txt")}
T4 = {int(r[0]): tuple(map(int, r[1:])) for r in read_golden("table4_values.txt")}
T5 = {int(r[0]): (int(r[1]), set() if r[2] == "-" else set(map(int, r[2].split(","))))
      for r in read_golden("table5_alpha.txt")}


def _alpha(n, m):
    a, ones = T5[n]
    k = m % a
    if n == 7 and m < 19:
        return 0
    return 1 if k in ones else 0


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_tables_3_4_5(n):
    """Algorithm 3 over K = 50 powers reproduces Table 3, Algorithm 4
    reproduces Table 4 (so A^{n+a} = b + A^n entrywise for n >= n0), and
    the closed form of Section 4 with Table 5's alpha holds for n0 <= m <= 50."""
    _, P, g = _powers(n)
    r = oracle.recurrence_search(P)
    assert r == T3[n]
    r0, a, b = r
    n0 = oracle.min_recurrence(P, r0, a, b)
    assert (n0, a, b) == T4[n]
    for m in range(n0, 51):
        assert g[m - 1] == math.ceil(b * m / a) + _alpha(n, m), (n, m)


@pytest.mark.slow
def test_tables_3_4_path_order_9():
    test_tables_3_4_5(9)


def test_c5_formula():
    """Section 4 quotes gamma_2(C_5 x P_n) = 2n+2 for even n > 2 and 2n+1
    for n = 2 or odd n."""
    for n in range(2, 10):
        want = 2 * n + 2 if (n % 2 == 0 and n > 2) else 2 * n + 1
        assert oracle.gamma2(n, 5, threads=os.cpu_count() or 1) == want, n


def test_mod3_formula_path_8():
    """Section 4: for 8 <= n <= 12 and m = 0 (mod 3), gamma_2 = (n+2) m / 3."""
    A = oracle.build_transfer(8)
    _, g = oracle.power_sequence(A, 48, keep_powers=False, threads=os.cpu_count() or 1)
    for m in range(3, 49, 3):
        assert g[m - 1] == 10 * m // 3, m


def test_powers_dense_from_third():
    """Section 3: the powers have no infinite entry from the third one on."""
    for n in range(2, 8):
        A = oracle.build_transfer(n)
        P, _ = oracle.power_sequence(A, 4)
        assert np.all(P[2] < INF) and np.all(P[3] < INF)
        assert np.any(A == INF)


def test_operand_order_bit_identical():
    """Algorithm 2 multiplies A (x) A^{k-1}; the chain here also uses
    A^{k-1} (x) A.  Associativity makes both the same matrix."""
    for n in range(2, 7):
        A = oracle.build_transfer(n)
        P1, g1 = oracle.power_sequence(A, 24, left_mul=True)
        P2, g2 = oracle.power_sequence(A, 24, left_mul=False)
        assert np.array_equal(P1, P2) and np.array_equal(g1, g2)


def test_power_rows_match_full_chain():
    for n in (4, 6):
        A = oracle.build_transfer(n)
        P, _ = oracle.power_sequence(A, 20)
        rows = np.array([0, 3, A.shape[0] - 1])
        R = oracle.power_rows(A, rows, 20)
        for t, i in enumerate(rows):
            assert np.array_equal(R[t], P[:, i, :])


# ------------------------------------------------ (min,+) product pins

def _rand(rng, shape, inf_frac, hi=31, dtype=np.int16, inf=INF):
    X = rng.integers(0, hi + 1, size=shape).astype(dtype)
    X[rng.random(shape) < inf_frac] = inf
    return X


def test_transfer_power_rows_match_dense():
    """The oracle's rows of A(D_n)^k listed straight from the word rule (for
    path orders whose N x N matrix does not fit the host) equal the rows of
    the dense oracle chain, for every row of n <= 6 and sampled rows of 7, 8."""
    for n in range(1, 9):
        A = oracle.build_transfer(n)
        N = A.shape[0]
        rows = np.arange(N) if N <= 225 else np.array(sorted({0, N // 3, N // 2, N - 1}))
        got = oracle.transfer_power_rows(n, rows, 10, threads=os.cpu_count() or 1)
        want = oracle.power_rows(A, rows, 10, threads=os.cpu_count() or 1)
        assert np.array_equal(got, want), n


def test_carre_walks():
    """Theorem 1: (A^k)_ij is the least label over walks of length k from
    i to j (INF when there is none).  Brute force over all walks."""
    rng = np.random.default_rng(5)
    for N in (3, 4, 5):
        A = _rand(rng, (N, N), 0.35, hi=9)
        P, _ = oracle.power_sequence(A, 4, left_mul=True)
        for k in range(1, 5):
            for i in range(N):
                for j in range(N):
                    best = INF
                    for mid in itertools.product(range(N), repeat=k - 1):
                        path = (i,) + mid + (j,)
                        w = [int(A[path[t], path[t + 1]]) for t in range(k)]
                        if all(x < INF for x in w):
                            best = min(best, sum(w))
                    assert P[k - 1, i, j] == best, (N, k, i, j)


def test_shortest_path_closure():
    """With a zero diagonal, the (N-1)-th (min,+) power of a nonnegative
    weight matrix is the all-pairs shortest-path matrix (scipy's routine)."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(9)
    for N in (7, 12):
        # weights >= 1: scipy's dense input reads a 0 off the diagonal as "no edge"
        W = np.where(rng.random((N, N)) < 0.6, INF, rng.integers(1, 21, (N, N))).astype(np.int16)
        np.fill_diagonal(W, 0)
        P, _ = oracle.power_sequence(W, N - 1, keep_powers=True)
        dense = np.where(W < INF, W.astype(float), np.inf)
        D = csgraph.shortest_path(dense, method="FW", directed=True)
        want = np.where(np.isinf(D), INF, D).astype(np.int16)
        assert np.array_equal(P[N - 2], want)
        # the same closure in uint8 (INF = 255), weights small enough not to saturate
        W8 = np.where(W < INF, W, 255).astype(np.uint8)
        Z = W8.copy()
        for _ in range(N - 2):
            Z = oracle.minplus_mul(Z, W8)
        assert np.array_equal(Z, np.where(want == INF, 255, want).astype(np.uint8))


def test_tropical_identities():
    rng = np.random.default_rng(11)
    for (M, K, L, N) in [(5, 7, 3, 6), (16, 9, 13, 4), (1, 1, 1, 1)]:
        X = _rand(rng, (M, K), 0.3)
        Y = _rand(rng, (K, L), 0.3)
        Z = _rand(rng, (L, N), 0.3)
        # associativity
        assert np.array_equal(oracle.minplus_mul(oracle.minplus_mul(X, Y), Z),
                              oracle.minplus_mul(X, oracle.minplus_mul(Y, Z)))
        # tropical identity: 0 on the diagonal, INF elsewhere
        I = np.full((K, K), INF, np.int16)
        np.fill_diagonal(I, 0)
        assert np.array_equal(oracle.minplus_mul(X, I), X)
        # an all-INF row of X gives an all-INF row; an INF column of Y likewise
        X2 = X.copy(); X2[0, :] = INF
        assert np.all(oracle.minplus_mul(X2, Y)[0] == INF)
        Y2 = Y.copy(); Y2[:, 0] = INF
        assert np.all(oracle.minplus_mul(X, Y2)[:, 0] == INF)
        # monotone: raising entries of X never lowers the product
        X3 = np.minimum(X.astype(np.int32) + rng.integers(0, 3, X.shape), INF).astype(np.int16)
        assert np.all(oracle.minplus_mul(X3, Y) >= oracle.minplus_mul(X, Y))
        # scalar (x) matrix: adding c to X adds c to every finite entry
        Xc = np.where(X < INF, X + 3, INF).astype(np.int16)
        P0, Pc = oracle.minplus_mul(X, Y), oracle.minplus_mul(Xc, Y)
        assert np.array_equal(np.where(P0 < INF, P0 + 3, INF), Pc)


def test_power_additivity():
    """A^a (x) A^b = A^{a+b} (Lemma 1's algebra) on a transfer matrix."""
    A = oracle.build_transfer(5)
    P, _ = oracle.power_sequence(A, 12)
    for a, b in [(1, 1), (2, 3), (5, 7), (4, 4)]:
        assert np.array_equal(oracle.minplus_mul(P[a - 1], P[b - 1]), P[a + b - 1])


def test_saturation_at_inf():
    """Sums at or above the INF code clamp to INF (the saturating reading)."""
    X = np.array([[INF - 1, 5]], dtype=np.int16)
    Y = np.array([[1], [INF - 3]], dtype=np.int16)
    assert oracle.minplus_mul(X, Y)[0, 0] == INF
    Y2 = np.array([[0], [INF - 3]], dtype=np.int16)
    assert oracle.minplus_mul(X, Y2)[0, 0] == INF - 1
    X8 = np.array([[200, 254]], dtype=np.uint8)
    Y8 = np.array([[100], [0]], dtype=np.uint8)
    assert oracle.minplus_mul(X8, Y8)[0, 0] == 254
    Y8b = np.array([[60], [1]], dtype=np.uint8)
    assert oracle.minplus_mul(X8, Y8b)[0, 0] == 255


def test_uint8_agrees_with_int16_below_saturation():
    """Both INF encodings give the same product when nothing saturates."""
    rng = np.random.default_rng(3)
    X = _rand(rng, (33, 40), 0.3)
    Y = _rand(rng, (40, 29), 0.3)
    Z16 = oracle.minplus_mul(X, Y)
    to8 = lambda M: np.where(M == INF, 255, M).astype(np.uint8)
    Z8 = oracle.minplus_mul(to8(X), to8(Y))
    assert np.array_equal(Z8, to8(Z16))


def test_threads_do_not_change_results():
    rng = np.random.default_rng(4)
    X = _rand(rng, (70, 50), 0.3)
    Y = _rand(rng, (50, 60), 0.3)
    assert np.array_equal(oracle.minplus_mul(X, Y, threads=1),
                          oracle.minplus_mul(X, Y, threads=4))
