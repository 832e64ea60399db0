"""Pins of the oracle's exact parts: cuts, brute force, Pareto filter, hypervolume,
weight vectors and the counter-based RNG -- each against what the paper or the
mathematics fixes, never against the oracle itself."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from conftest import golden_lines, parse_points
from paper_2604_26477_b300 import workloads as wl


def _inst_from_edges(n, rows):
    ei = np.array([r[0] for r in rows], np.int32)
    ej = np.array([r[1] for r in rows], np.int32)
    w = np.array([r[2:] for r in rows], np.int32).T.copy()
    return wl.Instance(n, ei, ej, w)


# ----------------------------------------------------------------------------- RNG
def test_philox_known_answers(oracle):
    for line in golden_lines("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in line.split()]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_normal_moments_and_ks(oracle):
    # Eq. NI-SB asks for standard Gaussian noise: moments, KS, kurtosis
    z = np.array([oracle.normal(7, 3, r, i, m) for r in range(4) for i in range(50) for m in range(100)])
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 0.2
    # the bulk helper returns the same draws as single calls
    assert np.array_equal(oracle.normals(7, 3, 1, 2, 0, 100), z[(1 * 50 + 2) * 100:(1 * 50 + 3) * 100])
    # steps, spins, replicas, rounds and seeds are distinct draws
    base = oracle.normal(1, 0, 0, 0, 0)
    assert len({base, oracle.normal(1, 0, 0, 0, 1), oracle.normal(1, 0, 0, 1, 0), oracle.normal(1, 0, 1, 0, 0),
                oracle.normal(1, 1, 0, 0, 0), oracle.normal(2, 0, 0, 0, 0)}) == 6


def test_normal_tails_and_resolution(oracle):
    # a standard Gaussian's tail mass: P(|Z| > 3) = 2.700e-3, P(|Z| > 4.71) = 2.48e-6. A draw
    # from 16-bit uniforms is bounded by sqrt(32 ln 2) = 4.71 and fails the second check.
    z = np.concatenate([oracle.normals(11, 0, r, i, 0, 1_000_000) for r in range(4) for i in range(5)])
    N = z.size
    a = np.abs(z)
    p3 = 2 * stats.norm.sf(3.0)
    n3 = int((a > 3.0).sum())
    assert abs(n3 - N * p3) < 5 * np.sqrt(N * p3), n3
    bound = np.sqrt(32 * np.log(2))
    p4 = 2 * stats.norm.sf(bound)
    n4 = int((a > bound).sum())
    assert stats.poisson.cdf(n4, N * p4) > 1e-4 and stats.poisson.sf(n4 - 1, N * p4) > 1e-4, (n4, N * p4)
    assert n4 > 0
    # 53-bit uniforms: no two of a million draws coincide (16-bit pairs would collide ~100 times)
    assert np.unique(z[:1_000_000]).size == 1_000_000
    # the radius of Box-Muller: rho^2 / 2 = -ln u1 ~ Exp(1), checked on |eta| through the
    # half-normal law, and the sign is a fair coin
    assert stats.kstest(a[:200_000], stats.halfnorm.cdf).pvalue > 1e-3
    assert abs((z[:200_000] > 0).mean() - 0.5) < 0.005


def test_initial_state_uniform(oracle):
    xs = np.array([oracle.initial_state(11, 0, r, i, 0.1) for r in range(40) for i in range(100)])
    assert np.all(np.abs(xs) <= 0.1)
    u = (xs.ravel() + 0.1) / 0.2
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert np.all(xs.astype(np.float32).astype(np.float64) == xs)  # exactly a float


# ----------------------------------------------------------------------------- cuts
def test_triangle_golden(oracle):
    lines = golden_lines("triangle_cuts.txt")
    edges = [[int(t) for t in l.split()[1:]] for l in lines if l.startswith("edge")]
    inst = _inst_from_edges(3, edges)
    cfgs = [l for l in lines if l.startswith("config")]
    for c in cfgs:
        lhs, rhs = c.split("->")
        s = np.array([1 if t == "+" else -1 for t in lhs.split()[1:]])
        want = [int(t) for t in rhs.split()]
        got = oracle.cuts(inst, wl.signs_to_bits(s[None, :]))[0]
        assert list(got) == want
    bits, cuts = oracle.brute_force(inst)
    keep = oracle.pareto_filter(cuts)
    front = {tuple(cuts[k]) for k in keep}
    want_front = {tuple(p) for p in parse_points([l for l in lines if l.startswith("front")][0][5:])}
    assert front == want_front
    ref = oracle.reference_point(inst)
    assert list(ref) == [int(t) for t in [l for l in lines if l.startswith("ref")][0].split()[1:]]
    hv = oracle.hypervolume(cuts[keep], ref)
    assert hv == int([l for l in lines if l.startswith("hv")][0].split()[1])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cut_identities_bruteforce(oracle, seed):
    inst = wl.random_graph(12, 0.4, seed, K=3)
    bits, cuts = oracle.brute_force(inst)
    n, K = inst.n, inst.K
    # each edge is cut in exactly half of the 2^(n-1) configurations with s_0 = +1
    assert np.array_equal(cuts.sum(axis=0), (1 << (n - 2)) * inst.w.astype(np.int64).sum(axis=1))
    # all-equal spins cut nothing
    assert np.all(cuts[0] == 0)
    # flipping vertex i alone cuts its weighted degree
    for i in range(1, n):
        c = 1 << (i - 1)
        deg = np.zeros(K, np.int64)
        for e in range(inst.E):
            if inst.ei[e] == i or inst.ej[e] == i:
                deg += inst.w[:, e]
        assert np.array_equal(cuts[c], deg)
    # C(s) = C(-s): complement every spin
    W = bits.shape[1]
    mask = np.uint64((1 << n) - 1)
    assert np.array_equal(oracle.cuts(inst, bits ^ mask), cuts)
    # C_k = (sum_E J - H_k) / 2 from the Ising energies of the "Hamiltonian formulation"
    H = oracle.energies(inst, bits[:200])
    assert np.array_equal(2 * cuts[:200], inst.w.astype(np.int64).sum(axis=1) - H)


def test_bipartite_bipartition_cuts_everything(oracle):
    # 4x5 grid graph is bipartite: the checkerboard cuts every edge
    rows, cols = 4, 5
    edges = []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                edges.append((v, v + 1))
            if r + 1 < rows:
                edges.append((v, v + cols))
    rng = np.random.default_rng(0)
    inst = _inst_from_edges(rows * cols, [(a, b, int(rng.integers(1, 9)), int(rng.integers(-9, 9))) for a, b in edges])
    s = np.array([1 if (v // cols + v % cols) % 2 == 0 else -1 for v in range(rows * cols)])
    got = oracle.cuts(inst, wl.signs_to_bits(s[None, :]))[0]
    assert np.array_equal(got, inst.w.astype(np.int64).sum(axis=1))


def test_cuts_multiword(oracle):
    # n = 150 spans three words; compare against the +-1 formula evaluated with numpy
    inst = wl.random_regular(150, 5, K=3)
    bits = wl.random_sign_bits(20, 150, 9)
    s = wl.bits_to_signs(bits, 150).astype(np.int64)
    got = oracle.cuts(inst, bits)
    cut_mask = s[:, inst.ei] != s[:, inst.ej]  # edge cut <=> endpoints differ
    want = cut_mask.astype(np.int64) @ inst.w.T.astype(np.int64)
    assert np.array_equal(got, want)


# ----------------------------------------------------------------------------- Pareto
def _front_by_definition(cuts):
    """Non-dominated distinct vectors, each with its lowest index, by the definition."""
    M = cuts.shape[0]
    keep = []
    for a in range(M):
        u = cuts[a]
        dominated = np.any(np.all(cuts >= u, axis=1) & np.any(cuts > u, axis=1))
        first = np.flatnonzero(np.all(cuts == u, axis=1))[0] == a
        if not dominated and first:
            keep.append(a)
    return np.array(keep, np.int64)


@pytest.mark.parametrize("K,M,span", [(2, 300, 30), (3, 400, 12), (4, 300, 6), (3, 50, 2)])
def test_pareto_matches_definition(oracle, K, M, span):
    rng = np.random.default_rng(K * 1000 + M)
    cuts = rng.integers(-span, span, size=(M, K)).astype(np.int64)
    keep = oracle.pareto_filter(cuts)
    assert np.array_equal(keep, _front_by_definition(cuts))
    front = cuts[keep]
    # mutually non-dominated and distinct
    for i in range(len(front)):
        for j in range(len(front)):
            if i != j:
                assert not oracle.dominates(front[i], front[j])
                assert not np.array_equal(front[i], front[j])
    # every pool member is dominated by or equal to a front member
    for u in cuts:
        assert np.any(np.all(front >= u, axis=1))
    # idempotent, and the set of vectors does not depend on the pool order
    assert np.array_equal(oracle.pareto_filter(front), np.arange(len(front)))
    perm = rng.permutation(M)
    keep2 = oracle.pareto_filter(cuts[perm])
    assert {tuple(v) for v in cuts[perm][keep2]} == {tuple(v) for v in front}


# ----------------------------------------------------------------------------- HV
def _hv_inclusion_exclusion(points, ref):
    """Measure of the union of boxes by inclusion-exclusion (exact, small fronts)."""
    pts = [tuple(int(v) for v in p) for p in points]
    total = 0
    for size in range(1, len(pts) + 1):
        for sub in itertools.combinations(pts, size):
            vol = 1
            for k in range(len(ref)):
                side = min(p[k] for p in sub) - int(ref[k])
                if side <= 0:
                    vol = 0
                    break
                vol *= side
            total += vol if size % 2 else -vol
    return total


def test_hv_appendix_a(oracle):
    lines = golden_lines("app_a_hypervolume.txt")
    ref = [int(t) for t in lines[0].split()[1:]]
    for fl, hl in zip(lines[1::2], lines[2::2]):
        assert oracle.hypervolume(parse_points(fl[6:]), ref) == int(hl.split()[1])


@pytest.mark.parametrize("K", [2, 3, 4])
def test_hv_inclusion_exclusion(oracle, K):
    rng = np.random.default_rng(K)
    for trial in range(25):
        F = int(rng.integers(1, 10))
        pts = rng.integers(-5, 40, size=(F, K))
        ref = rng.integers(-10, 5, size=K)
        assert oracle.hypervolume(pts, ref) == _hv_inclusion_exclusion(pts, ref)


def test_hv_properties(oracle):
    rng = np.random.default_rng(5)
    K = 3
    pts = rng.integers(0, 1000, size=(60, K))
    ref = np.zeros(K, np.int64)
    # one point: the product of its sides
    assert oracle.hypervolume(pts[:1], ref) == int(np.prod(pts[0].astype(object)))
    hv_all = oracle.hypervolume(pts, ref)
    # only the non-dominated points matter; a dominated point adds nothing
    keep = oracle.pareto_filter(pts)
    assert oracle.hypervolume(pts[keep], ref) == hv_all
    # monotone as points are added (Pareto compliance, Appendix A)
    prev = 0
    for m in range(1, 61, 7):
        cur = oracle.hypervolume(pts[:m], ref)
        assert cur >= prev
        prev = cur
    # invariant to permuting the objectives
    for perm in itertools.permutations(range(K)):
        assert oracle.hypervolume(pts[:, perm], ref[list(perm)]) == hv_all
    # K = 2 staircase in closed form: sorted by y1 descending, strips of new y2
    p2 = rng.integers(0, 100, size=(30, 2))
    order = sorted(range(30), key=lambda i: -p2[i, 0])
    area, best = 0, 0
    for i in order:
        if p2[i, 1] > best:
            area += int(p2[i, 0]) * int(p2[i, 1] - best)
            best = int(p2[i, 1])
    assert oracle.hypervolume(p2, [0, 0]) == area


def test_hv_int128_range(oracle):
    # sides of 1.5e9 in four objectives (about 5e36) need 128-bit arithmetic
    side = 1_500_000_000
    pts = np.array([[side, side, side, side], [side + 7, 3, side, side]], np.int64)
    ref = np.zeros(4, np.int64)
    want = side ** 4 + 7 * 3 * side * side
    assert oracle.hypervolume(pts, ref) == want


# ----------------------------------------------------------------------------- lambda
def test_das_dennis_counts(oracle):
    # "190 evenly distributed Das-Dennis weight vectors for the three-objective problem
    # and 220 for the four-objective problem", interior points only
    assert oracle.das_dennis(3, 21, True).shape == (190, 3)
    assert oracle.das_dennis(4, 13, True).shape == (220, 4)
    for K, H in [(2, 5), (3, 7), (4, 6), (5, 8)]:
        full = oracle.das_dennis(K, H, False)
        inner = oracle.das_dennis(K, H, True)
        assert len(full) == math.comb(H + K - 1, K - 1)
        assert len(inner) == math.comb(H - 1, K - 1)
        m = np.rint(full * H).astype(int)
        assert np.all(m.sum(axis=1) == H) and np.allclose(m / H, full)
        assert np.all(np.rint(inner * H) >= 1)
        assert len({tuple(r) for r in m}) == len(m)
        assert [tuple(r) for r in m] == sorted(tuple(r) for r in m)


def test_dirichlet_moments(oracle):
    K = 3
    lam = oracle.dirichlet(20000, K, seed=3, round_=1)
    assert np.allclose(lam.sum(axis=1), 1.0, atol=1e-12) and np.all(lam > 0)
    # marginal of Dirichlet(1,..,1) is Beta(1, K-1): CDF 1 - (1 - x)^(K-1)
    assert stats.kstest(lam[:, 0], lambda x: 1 - (1 - x) ** (K - 1)).pvalue > 1e-3
    assert abs(lam[:, 1].var() - (K - 1) / (K * K * (K + 1))) < 3e-3
