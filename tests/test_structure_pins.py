"""Structural facts the GPU path relies on, pinned on the oracle (CPU).

* Reading every word backwards is an automorphism of A(D_n) (Section 2.2's
  rules are mirror images of each other: the forbidden windows 020, 111,
  211/112, 212 and the start/end rules 11, 12 / 11, 21), hence of every
  power.  The mirror-column chains keep one column of every pair {c, R c};
  the server's traces read one row of every pair {i, R i}.
* When the successors of q' are a subset of those of q, row q' of any
  product A (x) X bounds row q from above (a minimum over fewer terms with
  the same labels): the reuse circuit of the transfer step computes rows
  from such contained rows.
"""
import os

import numpy as np
import pytest

import oracle

INF = oracle.INF16
THREADS = os.cpu_count() or 1


def reversal(n):
    """The permutation of the words' indices that reads each word backwards."""
    W = oracle.enumerate_words(n)
    index = {w.tobytes(): i for i, w in enumerate(W)}
    perm = np.array([index[w[::-1].tobytes()] for w in W], dtype=np.int64)
    return perm


@pytest.mark.parametrize("n", list(range(1, 9)))
def test_reversal_is_an_automorphism(n):
    perm = reversal(n)
    assert np.array_equal(perm[perm], np.arange(perm.size))  # an involution
    A = oracle.build_transfer(n)
    assert np.array_equal(A[np.ix_(perm, perm)], A)


@pytest.mark.parametrize("n,kmax", [(4, 30), (6, 12)])
def test_powers_keep_the_reversal_symmetry(n, kmax):
    perm = reversal(n)
    P, g = oracle.power_sequence(oracle.build_transfer(n), kmax, threads=THREADS)
    for k in range(kmax):
        assert np.array_equal(P[k][np.ix_(perm, perm)], P[k]), k + 1
        # so the minimum diagonal is reached on the columns c <= R c alone
        d = np.diagonal(P[k]).astype(np.int64)
        keep = np.arange(perm.size) <= perm
        assert d[keep].min() == g[k]


def test_trace_terms_pair_up():
    """min over (i, l) of X[i][l] + Y[l][i] equals the same minimum over the
    rows i <= R i only (X, Y powers of A(D_n))."""
    n = 5
    perm = reversal(n)
    P, _ = oracle.power_sequence(oracle.build_transfer(n), 12, threads=THREADS)
    for a, b in [(3, 7), (5, 11), (1, 12)]:
        T = P[a - 1].astype(np.int64) + P[b - 1].astype(np.int64).T  # T[i][l]
        assert np.array_equal(T[np.ix_(perm, perm)], T)
        keep = np.arange(perm.size) <= perm
        assert T[keep].min() == T.min()


def test_nested_successor_sets_bound_rows():
    n = 6
    A = oracle.build_transfer(n)
    fin = A < INF
    N = A.shape[0]
    inter = fin.astype(np.int64) @ fin.T.astype(np.int64)
    size = fin.sum(1)
    sub = inter == size[None, :]  # sub[q, q']: Out(q') within Out(q)
    np.fill_diagonal(sub, False)
    # nearly every row contains another row's successors
    assert sub.any(axis=1).mean() > 0.95
    rng = np.random.default_rng(6)
    X = rng.integers(0, 40, size=(N, 17)).astype(np.int16)
    R = oracle.minplus_mul(A, X).astype(np.int64)
    qs, qps = np.nonzero(sub)
    assert (R[qs] <= R[qps]).all()
    # a row is the minimum of a few contained rows and of only the arcs they
    # leave uncovered (contained rows picked greedily by what they cover)
    reads = 0
    for q in range(N):
        left = fin[q].copy()
        parts = []
        for _ in range(8):
            cand = np.nonzero(sub[q])[0]
            if cand.size == 0:
                break
            gain = (fin[cand] & left).sum(1)
            if gain.max() < 2:
                break
            c = cand[gain.argmax()]
            parts.append(R[c])
            left &= ~fin[c]
        direct = np.where(left[:, None], A[q][:, None].astype(np.int64) + X.astype(np.int64), 10**9).min(0)
        assert np.array_equal(np.minimum.reduce(parts + [direct]), np.minimum(R[q], INF)), q
        reads += len(parts) + int(left.sum())
    assert reads * 3 < int(fin.sum())  # far fewer row reads than arcs
