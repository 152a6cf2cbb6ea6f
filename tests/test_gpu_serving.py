"""The gamma_2 server: continuous batching, admission by footprint, refusals.

Every answer equals the oracle's gamma_2 (small cases) or the same query
answered alone by a fresh server; admission, eviction, refusal, queue overflow
and cancellation are driven from the host.
"""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def mp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_17688_gb300 as mp
    mp.lib()
    return mp


def footprint(mp, n, max_m):
    B = int(np.ceil(np.sqrt(max_m)))
    T = max(2, -(-max_m // B))
    N = mp.mp_transfer_size(n)
    return (B + T) * ((N * N + 7) // 8 * 8) * 2


def test_mixed_queries_match_oracle_and_alone(mp):
    rng = np.random.default_rng(3)
    qs = [(int(rng.integers(1, 8)), int(rng.integers(3, 120))) for _ in range(300)]
    srv = mp.Server(hbm_budget=8 << 30, max_batch=64, max_m=120)
    tickets = [srv.submit(n, m) for n, m in qs]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(qs) and st["failed"] == 0
    tables = {n: oracle.gamma2_range(n, 120, threads=THREADS) for n in range(1, 8)}
    for (n, m), g in zip(qs, got):
        assert g == tables[n][m], (n, m)
    # the native load generator submits the same stream again
    srv2 = mp.Server(hbm_budget=8 << 30, max_batch=64, max_m=120)
    tk = srv2.replay([q[0] for q in qs], [q[1] for q in qs], np.linspace(0, 0.05, len(qs)))
    assert [srv2.wait(int(t)) for t in tk] == got
    srv2.close()
    # the same queries answered one at a time by a fresh server
    solo = mp.Server(hbm_budget=8 << 30, max_batch=64, max_m=120)
    for (n, m), g in list(zip(qs, got))[:40]:
        assert solo.wait(solo.submit(n, m)) == g
    solo.close()


def test_large_m_matches_recurrence(mp):
    """m up to 2000 for path orders up to 9, against Theorem 3 (computed by
    the library's recurrence path, itself pinned to Tables 3/4)."""
    srv = mp.Server(hbm_budget=16 << 30, max_batch=128, max_m=2000)
    qs = [(n, m) for n in (2, 5, 8, 9) for m in (3, 77, 500, 1999, 2000)]
    ts = [srv.submit(n, m) for n, m in qs]
    for (n, m), t in zip(qs, ts):
        assert srv.wait(t) == mp.mp_gamma2_cylinder(n, m), (n, m)
    srv.close()


def test_admission_evicts_and_stays_correct(mp):
    """A budget that holds path order 8 with 6 but not with 7 forces evictions;
    answers stay exact."""
    budget = footprint(mp, 8, 200) + footprint(mp, 6, 200) + footprint(mp, 7, 200) // 2
    srv = mp.Server(hbm_budget=budget, max_batch=32, max_m=200)
    want = {n: oracle.gamma2_range(n, 200, threads=THREADS) for n in (6, 7, 8)}
    for rnd in range(3):
        for n in (8, 7, 6, 8):
            m = 37 + 11 * rnd + n
            assert srv.wait(srv.submit(n, m)) == want[n][m]
    st = srv.stats()
    srv.close()
    assert st["evictions"] >= 1 and st["resident_bytes"] <= budget


def test_refusals_overflow_and_cancel(mp):
    small = footprint(mp, 5, 100)
    srv = mp.Server(hbm_budget=small, max_batch=8, max_m=100, max_tickets=6)
    t_big = srv.submit(9, 50)  # footprint far above the budget
    with pytest.raises(mp.MinplusError) as e:
        srv.wait(t_big)
    assert e.value.code == -3
    with pytest.raises(mp.MinplusError) as e:
        srv.submit(4, 2)
    assert e.value.code == -1
    with pytest.raises(mp.MinplusError) as e:
        srv.submit(4, 101)
    assert e.value.code == -1
    ts = [srv.submit(3, 10 + i) for i in range(5)]  # fills the six-ticket table
    with pytest.raises(mp.MinplusError) as e:
        srv.submit(3, 50)
    assert e.value.code == -7
    for i, t in enumerate(ts):
        assert srv.wait(t) == -(-4 * (10 + i) // 3)
    srv.close()
    # cancellation of a query waiting for its path order to be built
    srv = mp.Server(hbm_budget=16 << 30, max_batch=8, max_m=2000)
    t = srv.submit(9, 1000)
    srv.cancel(t)
    with pytest.raises(mp.MinplusError):
        srv.wait(t, timeout_s=30)
    assert srv.stats()["cancelled"] == 1
    srv.close()
