"""The sparse samplers' shared-memory layout (moq_plan_gather_layout, host only): a valid slot
permutation and per-row gather orders, determinism, its shared-memory pass counts against an
independent recount of the bank model and a hand-counted cycle, and the reduction it buys on
random regular graphs."""
import numpy as np
import pytest

from paper_2604_26477_b300 import workloads as wl


@pytest.fixture(scope="module")
def M():
    from paper_2604_26477_b300 import moqaia
    return moqaia


def _rb(n):
    # replicas per block with the fullest warps among blocks of about 256 threads
    best, rb = -1.0, 1
    for c in range(1, max(1, min(32, 256 // n)) + 1):
        util = n * c / (32.0 * -(-(n * c) // 32))
        if util > best + 0.01:
            best, rb = util, c
    return rb


def _rows(n, ei, ej):
    nb = [[] for _ in range(n)]
    for a, b in zip(ei.tolist(), ej.tolist()):
        nb[a].append(b)
        nb[b].append(a)
    return [sorted(r) for r in nb]


def _passes(n, slot_spin, rows):
    """8-byte (per half-warp, words modulo 16) and 4-byte (per warp, modulo 32) passes of one
    gather step: distinct words per bank, the largest count, summed over cells and rounds."""
    rb = _rb(n)
    spin_slot = np.empty(n, np.int64)
    spin_slot[np.asarray(slot_spin)] = np.arange(n)
    D = max(len(r) for r in rows)
    T = n * rb
    p8 = p4 = 0
    for d in range(D):
        words = []
        for t in range(T):
            s, lp = divmod(t, rb)
            i = int(slot_spin[s])
            c = rows[i][d] if d < len(rows[i]) else i
            words.append(int(spin_slot[c]) * rb + lp)
        for size, banks in ((16, 16), (32, 32)):
            for t0 in range(0, T, size):
                u = set(words[t0:t0 + size])
                cnt = np.bincount([w % banks for w in u], minlength=banks)
                if size == 16:
                    p8 += int(cnt.max())
                else:
                    p4 += int(cnt.max())
    return p8, p4


def _column_layout(n, rows):
    deg = np.array([len(r) for r in rows])
    return sorted(range(n), key=lambda i: -deg[i])  # stable: decreasing degree


def _check_valid(n, ei, ej, slot, gather):
    rows = _rows(n, ei, ej)
    assert sorted(slot.tolist()) == list(range(n))
    p = 0
    out = []
    for i in range(n):
        r = gather[p:p + len(rows[i])].tolist()
        assert sorted(r) == rows[i]
        out.append(r)
        p += len(rows[i])
    return rows, out


def test_cycle_pass_counts_by_hand(M):
    # cycle of 32, one replica per block slot: the column layout reads i-1 then i+1 (spin 0: 1
    # then 31, spin 31: 0 then 30). 8-byte: in round 0 the second half-warp reads words 16 and 0
    # (bank 0), in round 1 the first reads 31 and 15 (bank 15): 1 + 2 + 2 + 1 passes. 4-byte: the
    # warp's words are distinct modulo 32 in both rounds (1 + 1)
    n = 32
    ei = np.arange(n, dtype=np.int32)
    ej = (ei + 1) % n
    a, b = np.minimum(ei, ej), np.maximum(ei, ej)
    slot, gather, passes = M.moq_plan_gather_layout(n, a, b)
    assert passes[0] == 6 and passes[1] == 2
    rows, chosen = _check_valid(n, a, b, slot, gather)
    assert _passes(n, _column_layout(n, rows), rows) == (6, 2)
    assert tuple(passes[2:]) == _passes(n, slot, chosen)
    assert 4 * passes[2] + passes[3] <= 4 * 6 + 2
    assert passes[2] >= 2 * 2 and passes[3] >= 2  # one pass per cell and round at best


@pytest.mark.parametrize("src", [wl.heavy_hex_like(1001, K=4), wl.random_regular(64, 5, K=3), wl.random_regular(300, 5, K=3),
                                 wl.random_regular(200, 6, K=3, d=4), wl.random_graph(150, 0.02, 4, K=3)],
                         ids=["heavyhex42", "reg3_64", "reg3_300", "reg4_200", "gnp150_deg0to8"])
def test_layout_valid_deterministic_and_counted(M, src):
    n = src.n
    slot, gather, passes = M.moq_plan_gather_layout(n, src.ei, src.ej)
    rows, chosen = _check_valid(n, src.ei, src.ej, slot, gather)
    slot2, gather2, passes2 = M.moq_plan_gather_layout(n, src.ei, src.ej)
    assert np.array_equal(slot, slot2) and np.array_equal(gather, gather2) and np.array_equal(passes, passes2)
    assert tuple(passes[:2]) == _passes(n, _column_layout(n, rows), rows)
    assert tuple(passes[2:]) == _passes(n, slot, chosen)
    assert 4 * passes[2] + passes[3] <= 4 * passes[0] + passes[1]


def test_layout_cuts_passes_on_large_random_graphs(M):
    # column order: 18.4 8-byte passes per warp and step at n = 1024 (3 rounds); the layout
    # removes well over a quarter of the 8-byte and 4-byte passes
    for n, seed in ((1024, 5), (700, 6)):
        src = wl.random_regular(n, seed, K=3)
        _, _, p = M.moq_plan_gather_layout(n, src.ei, src.ej)
        assert p[2] <= 0.72 * p[0] and p[3] <= 0.72 * p[1], p


def test_layout_rejects_what_the_samplers_do_not_take(M):
    star = (np.zeros(9, np.int32), np.arange(1, 10, dtype=np.int32))  # degree 9
    with pytest.raises(M.MoqError) as e:
        M.moq_plan_gather_layout(10, *star)
    assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    big = wl.random_regular(1026, 1, K=3)
    with pytest.raises(M.MoqError):
        M.moq_plan_gather_layout(1026, big.ei, big.ej)
    with pytest.raises(M.MoqError):
        M.moq_plan_gather_layout(4, np.array([0, 0], np.int32), np.array([1, 1], np.int32))  # repeated edge


def test_longer_search_on_regular_graphs(M, monkeypatch):
    # MOQ_SB_LAYOUT_EFFORT = 1000: the transversal search on a random 3-regular graph (one replica
    # per slot) is valid, deterministic, counted as the bank model counts it, and removes a good
    # part of the 8-byte passes the default planner leaves
    src = wl.random_regular(1024, 5, K=3)
    _, _, base = M.moq_plan_gather_layout(src.n, src.ei, src.ej)
    monkeypatch.setenv("MOQ_SB_LAYOUT_EFFORT", "1000")
    slot, gather, p = M.moq_plan_gather_layout(src.n, src.ei, src.ej)
    rows, chosen = _check_valid(src.n, src.ei, src.ej, slot, gather)
    assert tuple(p[2:]) == _passes(src.n, slot, chosen)
    slot2, gather2, _ = M.moq_plan_gather_layout(src.n, src.ei, src.ej)
    assert np.array_equal(slot, slot2) and np.array_equal(gather, gather2)
    assert p[2] <= 0.8 * base[2] and p[3] <= base[3] + 4, (base, p)
    assert p[2] >= 3 * 64  # one pass per half-warp and round at best
    # irregular graphs and blocks of several replicas keep the default planner
    for g in (wl.random_graph(150, 0.02, 4, K=3), wl.heavy_hex_like(1001, K=4)):
        monkeypatch.setenv("MOQ_SB_LAYOUT_EFFORT", "0")
        a = M.moq_plan_gather_layout(g.n, g.ei, g.ej)
        monkeypatch.setenv("MOQ_SB_LAYOUT_EFFORT", "1000")
        b = M.moq_plan_gather_layout(g.n, g.ei, g.ej)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
