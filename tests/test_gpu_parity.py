"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Exact parts (instance sums, cuts, Pareto archive, hypervolume, lattice counts) must
match bit for bit; SB forces match the double-precision oracle within the normwise
FP32 bound |f - f64| <= 1e-5 * c0 * sum_j |J(c)_ij phi(x_j)| per spin; trajectories
(chaotic) are compared by the distribution of final hypervolumes over 32 seeds.
"""
import numpy as np
import pytest
import torch
from scipy import stats

from conftest import golden_lines, parse_points
from paper_2604_26477_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-5


@pytest.fixture(scope="module")
def M():
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import moqaia
    assert torch.cuda.is_available()
    return moqaia


@pytest.fixture(scope="module")
def P(M):
    from paper_2604_26477_b300 import pipeline
    return pipeline


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _bits_dev(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).cuda()


def _bits_host(t):
    return t.cpu().numpy().view(np.uint64)


def _canonical(bits, n):
    """Flip configurations with s_0 = -1 (C(s) = C(-s))."""
    out = bits.copy()
    W = out.shape[1]
    flip = (out[:, 0] & np.uint64(1)) == 1
    for w in range(W):
        nb = min(64, n - 64 * w)
        mask = np.uint64((1 << nb) - 1) if nb < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        out[flip, w] ^= mask
    return out


INSTANCES = {
    "heavyhex_K3": lambda: wl.heavy_hex_like(1000, K=3),
    "heavyhex_K4": lambda: wl.heavy_hex_like(1001, K=4),
    "reg3_n150_K3": lambda: wl.random_regular(150, 7, K=3),
    "reg3_n1024_K3": lambda: wl.random_regular(1024, 8, K=3),
    "gnp_n40_K2": lambda: wl.random_graph(40, 0.2, 3, K=2),
    "gnp_n70_K8": lambda: wl.random_graph(70, 0.1, 4, K=8),
    "complete_n100_K3": lambda: wl.complete_graph(100, 5, K=3),
}


# ----------------------------------------------------------------------------- a1
@pytest.mark.parametrize("name", list(INSTANCES))
def test_instance_info(M, P, oracle, name):
    src = INSTANCES[name]()
    inst = P.Instance(src)
    info = inst.info
    w = src.w.astype(np.int64)
    deg = np.bincount(np.concatenate([src.ei, src.ej]), minlength=src.n)
    assert info["n"] == src.n and info["K"] == src.K and info["E"] == src.E and info["words"] == (src.n + 63) // 64
    assert info["max_degree"] == deg.max()
    assert info["weight_sum"] == list(w.sum(axis=1))
    assert info["abs_sum"] == list(np.abs(w).sum(axis=1))
    assert info["ref_point"] == list(oracle.reference_point(src))


def test_dense_constructor_matches_edge_list(M, P, oracle):
    # an upper-triangle weight matrix (zeros where no objective has an edge) gives the
    # instance of its non-zero pairs in row order
    src = wl.random_graph(37, 0.3, 21, K=3, wmax=9)
    n, K = src.n, src.K
    iu, ju = np.triu_indices(n, 1)
    pos = {(int(a), int(b)): q for q, (a, b) in enumerate(zip(iu, ju))}
    J = np.zeros((K, iu.size), np.int32)
    for e in range(src.E):
        J[:, pos[(int(src.ei[e]), int(src.ej[e]))]] = src.w[:, e]
    h = M.moq_create_instance_dense(n, K, J)
    try:
        info = M.moq_instance_get_info(h)
        assert info["E"] == src.E and info["weight_sum"] == list(src.w.astype(np.int64).sum(axis=1))
        assert info["ref_point"] == list(oracle.reference_point(src))
        bits = wl.random_sign_bits(300, n, 4)
        cuts = torch.zeros((300, K), dtype=torch.int64, device="cuda")
        M.moq_evaluate_cuts(h, _bits_dev(bits), 300, cuts)
        assert np.array_equal(cuts.cpu().numpy(), oracle.cuts(src, bits))
    finally:
        M.moq_destroy_instance(h)
    with pytest.raises(M.MoqError) as e:
        M.moq_create_instance_dense(1, K, np.zeros(0, np.int32))
    assert e.value.code == M.MOQ_ERR_ARG


def test_instance_rejects_bad_input(M):
    ei = np.array([0, 1], np.int32)
    with pytest.raises(M.MoqError) as e:
        M.moq_create_instance(4, 2, 2, ei, np.array([1, 1], np.int32), np.ones(4, np.int32))  # 1 >= 1
    assert e.value.code == M.MOQ_ERR_ARG
    with pytest.raises(M.MoqError) as e:
        M.moq_create_instance(4, 2, 2, ei, np.array([2, 4], np.int32), np.ones(4, np.int32))  # 4 >= n
    assert e.value.code == M.MOQ_ERR_ARG
    with pytest.raises(M.MoqError) as e:
        M.moq_create_instance(4, 2, 2, np.array([0, 0], np.int32), np.array([2, 2], np.int32), np.ones(4, np.int32))
    assert e.value.code == M.MOQ_ERR_ARG and "repeated" in str(e.value)
    with pytest.raises(M.MoqError) as e:
        M.moq_create_instance(4, 9, 0, [], [], [])
    assert e.value.code == M.MOQ_ERR_ARG


@pytest.mark.parametrize("n,edges", [(5, []), (2, [(0, 1)]), (7, [(0, 3), (2, 6)])])
def test_degenerate_graphs_through_the_whole_path(M, P, oracle, n, edges):
    # no edges, one edge between the only two spins, isolated spins beside two edges: the build,
    # both precisions and variants of the sampler, the cuts, the merge and the hypervolume all run
    # and give the oracle's integer results on the sampled configurations
    K, R = 3, 37
    rng = np.random.default_rng(n)
    ei = np.array([e[0] for e in edges], np.int32)
    ej = np.array([e[1] for e in edges], np.int32)
    w = rng.choice(np.r_[np.arange(-10, 0), np.arange(1, 11)], size=(K, len(edges))).astype(np.int32)
    src = wl.Instance(n, ei, ej, w, name=f"degenerate_n{n}_E{len(edges)}")
    inst = P.Instance(src)
    assert inst.info["E"] == len(edges) and inst.info["weight_sum"] == [int(x) for x in w.astype(np.int64).sum(axis=1)]
    assert list(inst.ref) == list(oracle.reference_point(src))
    lam = _dev(wl.dirichlet_lambdas(R, K, 3), torch.float32)
    for precision in ("fp32", "fp16"):
        for variant in ("dsb", "bsb"):
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            p = M.moq_default_params(variant=variant, steps=50, dt=0.5, alpha=0.1, precision=precision)
            M.moq_sample(inst.handle, lam, R, p, 9, 0, bits)
            cuts = torch.zeros((R, K), dtype=torch.int64, device="cuda")
            M.moq_evaluate_cuts(inst.handle, bits, R, cuts)
            hb = bits.cpu().numpy().view(np.uint64)
            want = oracle.cuts(src, hb)
            assert np.array_equal(cuts.cpu().numpy(), want)
            arch = P.Archive(n, K, capacity=64, max_batch=R)
            arch.merge(cuts, bits, R, 0)
            front = want[oracle.pareto_filter(want)]
            gc, _, _ = arch.copy_out()
            assert sorted(map(tuple, gc.tolist())) == sorted(map(tuple, front.tolist()))
            assert arch.hypervolume(inst.ref) == oracle.hypervolume(front, inst.ref)
            arch.close()
    inst.close()


# ----------------------------------------------------------------------------- a6
@pytest.mark.parametrize("name", list(INSTANCES))
def test_cuts_bit_exact(M, P, oracle, name):
    src = INSTANCES[name]()
    inst = P.Instance(src)
    Mn = 1000 + 37  # several blocks and a ragged tail
    bits = wl.random_sign_bits(Mn, src.n, 11)
    cuts = torch.zeros((Mn, src.K), dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, _bits_dev(bits), Mn, cuts)
    assert np.array_equal(cuts.cpu().numpy(), oracle.cuts(src, bits))
    M.moq_evaluate_cuts(inst.handle, _bits_dev(bits), 0, cuts)  # M = 0 is a no-op


@pytest.mark.parametrize("form", ["thread", "warp"])
@pytest.mark.parametrize("name,M_", [("gnp_n300_dense", 37), ("gnp_n300_dense", 1000), ("reg3_n1024_K3", 300),
                                     ("heavyhex_K4", 1), ("gnp_n70_K8", 517)])
def test_cuts_both_forms_bit_exact(M, P, oracle, monkeypatch, form, name, M_):
    # one thread per sample and one warp per sample (lanes split the edges, shuffle reduction)
    # give the oracle's exact cuts, K = 2..8, one or many words per sample, ragged blocks
    monkeypatch.setenv("MOQ_CUTS_FORM", form)
    src = wl.random_graph(300, 0.3, 5, K=3, wmax=1000) if name == "gnp_n300_dense" else INSTANCES[name]()
    inst = P.Instance(src)
    bits = wl.random_sign_bits(M_, src.n, 17)
    cuts = torch.zeros((M_, src.K), dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, _bits_dev(bits), M_, cuts)
    assert np.array_equal(cuts.cpu().numpy(), oracle.cuts(src, bits))


def test_cuts_every_configuration(M, P, oracle):
    src = wl.random_graph(14, 0.4, 9, K=3)
    inst = P.Instance(src)
    bits, want = oracle.brute_force(src)
    cuts = torch.zeros(want.shape, dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, _bits_dev(bits), bits.shape[0], cuts)
    assert np.array_equal(cuts.cpu().numpy(), want)


def test_cuts_golden_triangle(M, P):
    lines = golden_lines("triangle_cuts.txt")
    rows = [[int(t) for t in l.split()[1:]] for l in lines if l.startswith("edge")]
    src = wl.Instance(3, np.array([r[0] for r in rows], np.int32), np.array([r[1] for r in rows], np.int32),
                      np.array([r[2:] for r in rows], np.int32).T.copy())
    inst = P.Instance(src)
    cfgs = [l for l in lines if l.startswith("config")]
    s = np.array([[1 if t == "+" else -1 for t in c.split("->")[0].split()[1:]] for c in cfgs])
    want = np.array([[int(t) for t in c.split("->")[1].split()] for c in cfgs])
    cuts = torch.zeros(want.shape, dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, _bits_dev(wl.signs_to_bits(s)), len(cfgs), cuts)
    assert np.array_equal(cuts.cpu().numpy(), want)


# ----------------------------------------------------------------------------- a7
def _run_archive(M, P, oracle, cuts, bits, n, batches, capacity=1 << 14):
    K = cuts.shape[1]
    arch = P.Archive(n, K, capacity=capacity, max_batch=max(max(b) - min(b) for b in batches) + 1)
    for b in batches:
        lo, hi = b[0], b[-1] + 1
        size = arch.merge(_dev(cuts[lo:hi], torch.int64), _bits_dev(bits[lo:hi]), hi - lo, lo, want_size=True)
    gc, gb, gi = arch.copy_out()
    keep = oracle.pareto_filter(cuts)
    assert size == len(keep)
    assert np.array_equal(gi, keep)
    assert np.array_equal(gc, cuts[keep])
    assert np.array_equal(gb, _canonical(bits[keep], n))
    return arch


@pytest.mark.parametrize("K,span,Mtot", [(2, 40, 3000), (3, 12, 5000), (4, 6, 4000), (8, 3, 2000), (3, 1000, 20000),
                                         # batches of 2^13 and more take the dedup / survivor path
                                         (2, 40, 90000), (4, 6, 150000), (3, 1000, 120000), (6, 4, 70000)])
@pytest.mark.parametrize("form", ["warp", "thread"])
def test_pareto_archive_bit_exact(M, P, oracle, monkeypatch, K, span, Mtot, form):
    # both dominance forms (one warp per tested vector, or a thread per vector over tiles)
    monkeypatch.setenv("MOQ_FILTER_FORM", form)
    rng = np.random.default_rng(K * 7 + span)
    cuts = rng.integers(-span, span, size=(Mtot, K)).astype(np.int64)
    n = 70
    bits = wl.random_sign_bits(Mtot, n, K)
    cuts[::17] = cuts[5]  # many exact duplicates
    edges = sorted({0, Mtot} | set(rng.integers(1, Mtot, size=5).tolist()))
    batches = [list(range(a, b)) for a, b in zip(edges[:-1], edges[1:])]
    _run_archive(M, P, oracle, cuts, bits, n, batches)


@pytest.mark.parametrize("K,Mtot,span,noise", [(3, 100000, 100, 6), (4, 80000, 30, 3)])
@pytest.mark.parametrize("form", ["warp", "thread"])
def test_pareto_large_batches_with_large_fronts(M, P, oracle, monkeypatch, K, Mtot, span, noise, form):
    monkeypatch.setenv("MOQ_FILTER_FORM", form)
    # candidates near a simplex surface (fronts of thousands of points) with many exact
    # duplicates, merged in batches above and below 2^13: the dedup / survivor path and the
    # plain path must both keep the definition's front and the lowest index per vector
    rng = np.random.default_rng(K)
    cuts = rng.integers(0, span, size=(Mtot, K)).astype(np.int64)
    cuts[:, -1] = span * (K - 1) - cuts[:, :-1].sum(axis=1) + rng.integers(0, noise, Mtot)
    cuts[::11] = cuts[3]
    bits = wl.random_sign_bits(Mtot, 42, K + 1)
    cut_at = [0, 40000, 45000, Mtot]  # 40000 (dedup path), 5000 (plain path), the rest (dedup)
    batches = [list(range(a, b)) for a, b in zip(cut_at[:-1], cut_at[1:])]
    _run_archive(M, P, oracle, cuts, bits, 42, batches, capacity=1 << 15)


@pytest.mark.parametrize("K,offset,width", [
    (4, -(1 << 40), 32768),   # max - min = 2^15 - 1: the widest packed span, far from zero
    (4, 5, 32769),            # one value more: the plain int64 comparison
    (3, -(1 << 62), 1 << 63),  # near the int64 limits
    (6, 123, 30000),          # two packed words
])
@pytest.mark.parametrize("form", ["warp", "thread"])
def test_pareto_packed_and_plain_ranges(M, P, oracle, monkeypatch, K, offset, width, form):
    monkeypatch.setenv("MOQ_FILTER_FORM", form)
    # the filter packs vectors into 16-bit lanes only when every objective spans fewer than
    # 2^15 values; both sides of that switch must give the definition's front
    rng = np.random.default_rng(K + width % 97)
    Mtot, n = 3000, 42
    cuts = (offset + rng.integers(0, width, size=(Mtot, K), dtype=np.int64)).astype(np.int64)
    cuts[:, 0] = np.where(rng.random(Mtot) < 0.3, offset + width - 1 - (cuts[:, 1] - offset) // 2, cuts[:, 0])
    cuts[::13] = cuts[7]
    cuts[1, :] = offset  # the span's ends are attained
    cuts[2, 0] = offset + width - 1
    bits = wl.random_sign_bits(Mtot, n, K)
    _run_archive(M, P, oracle, cuts, bits, n, [list(range(0, 1800)), list(range(1800, Mtot))])


def test_copy_out_into_page_locked_buffers(M, P):
    # the archive's reused page-locked copy equals the plain copy: an empty front, a small one,
    # and a front of 3000 mutually non-dominated vectors, which outgrows the first 1024-row
    # buffers; a caller-owned array of the wrong row size is refused before any copy
    n, K = 70, 2
    arch = P.Archive(n, K, capacity=1 << 13, max_batch=4096)
    for m, base in ((0, 0), (5, 10), (3000, 1000)):
        arch.reset()
        if m:
            anti = np.array([[i, 5000 - i] for i in range(m)], np.int64)
            arch.merge(_dev(anti, torch.int64), _bits_dev(wl.random_sign_bits(m, n, m)), m, base)
        want = arch.copy_out()
        got = arch.copy_out(reuse=True)
        assert len(got[2]) == m and all(np.array_equal(a, b) for a, b in zip(want, got))
        assert got[1].dtype == np.uint64 and got[0].shape == (m, K) and got[1].shape == (m, 2)
    assert arch._pinned[2].shape[0] == 4096
    bad = (np.zeros((8, K), np.int64), np.zeros((8, 2), np.uint64), np.zeros(9, np.int64))
    with pytest.raises(ValueError):
        M.moq_archive_copy_out_into(arch.handle, *bad)


def test_pareto_edge_cases(M, P, oracle):
    n, K = 42, 3
    arch = P.Archive(n, K, capacity=8, max_batch=64)
    empty = torch.zeros((1, K), dtype=torch.int64, device="cuda")
    assert arch.merge(empty, torch.zeros((1, 1), dtype=torch.int64, device="cuda"), 0, 0, want_size=True) == 0
    # all candidates equal: one survivor, the lowest index
    c = np.tile(np.array([[3, 4, 5]], np.int64), (50, 1))
    b = wl.random_sign_bits(50, n, 1)
    assert arch.merge(_dev(c, torch.int64), _bits_dev(b), 50, 100, want_size=True) == 1
    gc, gb, gi = arch.copy_out()
    assert gi.tolist() == [100] and np.array_equal(gb, _canonical(b[:1], n))
    # an equal vector in a later batch does not replace the member
    assert arch.merge(_dev(c[:3], torch.int64), _bits_dev(b[:3]), 3, 200, want_size=True) == 1
    assert arch.copy_out()[2].tolist() == [100]
    # capacity: 9 mutually non-dominated vectors do not fit in 8 slots; archive unchanged
    anti = np.array([[i, 20 - i, 0] for i in range(9)], np.int64)
    with pytest.raises(M.MoqError) as e:
        arch.merge(_dev(anti, torch.int64), _bits_dev(wl.random_sign_bits(9, n, 2)), 9, 300, want_size=True)
    assert e.value.code == M.MOQ_ERR_CAPACITY
    assert arch.copy_out()[2].tolist() == [100]
    # the same into an empty archive: reported too, and the archive stays empty
    empty_arch = P.Archive(n, K, capacity=8, max_batch=64)
    with pytest.raises(M.MoqError) as e:
        empty_arch.merge(_dev(anti, torch.int64), _bits_dev(wl.random_sign_bits(9, n, 2)), 9, 300, want_size=True)
    assert e.value.code == M.MOQ_ERR_CAPACITY
    assert empty_arch.size() == 0
    empty_arch.close()
    with pytest.raises(M.MoqError):
        arch.merge(_dev(np.zeros((65, K), np.int64), torch.int64), _bits_dev(wl.random_sign_bits(65, n, 3)), 65, 0)


@pytest.mark.parametrize("K", [2, 3, 4])
def test_capacity_overflow_on_every_merge_path(M, P, K):
    # a merge whose front would exceed the archive's capacity is reported and leaves the
    # archive as it was: on the large-batch path (dedup, survivors; 9000 candidates), into an
    # empty and into a non-empty archive, and through moq_archive_merge
    n = 50
    rng = np.random.default_rng(K)
    anti = np.zeros((9000, K), np.int64)
    anti[:, 0] = np.arange(9000)
    anti[:, 1] = 20000 - np.arange(9000)
    anti = anti[rng.permutation(9000)]
    bits = _bits_dev(wl.random_sign_bits(9000, n, 3))
    arch = P.Archive(n, K, capacity=100, max_batch=9000)
    with pytest.raises(M.MoqError) as e:
        arch.merge(_dev(anti, torch.int64), bits, 9000, 0, want_size=True)
    assert e.value.code == M.MOQ_ERR_CAPACITY
    assert arch.size() == 0
    few = np.zeros((50, K), np.int64)
    few[:, 0] = 30000 + np.arange(50)
    few[:, 1] = 30000 - np.arange(50)
    assert arch.merge(_dev(few, torch.int64), bits[:50], 50, 10 ** 6, want_size=True) == 50
    before = arch.copy_out()
    with pytest.raises(M.MoqError) as e:  # 9000 more, none dominated by the 50: overflow
        big = anti.copy()
        big[:, 0] += 40000
        arch.merge(_dev(big, torch.int64), bits, 9000, 0, want_size=True)
    assert e.value.code == M.MOQ_ERR_CAPACITY
    after = arch.copy_out()
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    # archive into archive: 9 mutually non-dominated members into an empty archive of 8 slots
    src = P.Archive(n, K, capacity=64, max_batch=64)
    assert src.merge(_dev(anti[:9], torch.int64), bits[:9], 9, 0, want_size=True) == 9
    dst = P.Archive(n, K, capacity=8, max_batch=64)
    dst.merge_from(src)
    with pytest.raises(M.MoqError) as e:
        dst.size()
    assert e.value.code == M.MOQ_ERR_CAPACITY
    assert dst.size() == 0  # the latch is cleared once reported
    for a in (arch, src, dst):
        a.close()


# ----------------------------------------------------------------------------- a8
def _hv_points(M, pts, ref):
    F, K = pts.shape
    ws = torch.zeros(M.moq_hypervolume_workspace_size(F, K), dtype=torch.uint8, device="cuda")
    return M.moq_hypervolume_points(_dev(pts, torch.int64), F, K, ref, ws)


def test_hv_appendix_a(M):
    lines = golden_lines("app_a_hypervolume.txt")
    ref = [int(t) for t in lines[0].split()[1:]]
    for fl, hl in zip(lines[1::2], lines[2::2]):
        assert _hv_points(M, parse_points(fl[6:]), ref) == int(hl.split()[1])


@pytest.mark.parametrize("K,F,span", [(2, 700, 10000), (3, 1500, 300), (3, 2100, 20), (4, 300, 100), (4, 260, 8),
                                      (4, 2500, 150), (4, 1100, 10 ** 6), (3, 3000, 10 ** 7)])
def test_hv_bit_exact(M, oracle, K, F, span):
    rng = np.random.default_rng(K * 100 + F)
    pts = rng.integers(-span // 10, span, size=(F, K)).astype(np.int64)
    ref = np.zeros(K, np.int64)
    # keep it mostly a front: project onto a noisy simplex surface, plus dominated points
    if K >= 3:
        pts[: F // 2, -1] = span * 2 - pts[: F // 2, :-1].sum(axis=1)
    assert _hv_points(M, pts, ref) == oracle.hypervolume(pts, ref)


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("offset", [(1 << 32) - 1, 1 << 32, 1 << 45])
def test_hv4_walk_widths(M, oracle, k, offset):
    # K = 4 fronts within the shared-memory form take the 32-bit walk while every kept point
    # lies less than 2^32 above the reference point in y_0, y_1 and y_2, the 128-bit walk
    # otherwise: one point of a 900-point front is lifted to `offset` above the reference in
    # objective k (2^32 - 1: still 32-bit; 2^32 and 2^45: 128-bit), with a negative reference
    rng = np.random.default_rng(11 + k)
    F = 900
    pts = rng.integers(0, 60, size=(F, 4)).astype(np.int64)
    pts[:, -1] = 180 - pts[:, :-1].sum(axis=1) + rng.integers(0, 3, F)
    ref = np.array([-5, -3, -2, -1], np.int64)
    pts[17, k] = ref[k] + offset
    want = oracle.hypervolume(pts[oracle.pareto_filter(pts)], ref)
    assert _hv_points(M, pts, ref) == want


@pytest.mark.parametrize("K,F", [(3, 7000), (4, 7000)])
def test_hv_large_mostly_dominated(M, oracle, K, F):
    # beyond the shared-memory fast path: many points, few of them on the front; the
    # hypervolume of the whole set equals the oracle's on the oracle-filtered front
    rng = np.random.default_rng(F + K)
    pts = rng.integers(0, 1000, size=(F, K)).astype(np.int64)
    front = rng.integers(900, 1100, size=(40, K)).astype(np.int64)
    pts[rng.choice(F, size=40, replace=False)] = front
    ref = np.zeros(K, np.int64)
    keep = oracle.pareto_filter(pts)
    assert _hv_points(M, pts, ref) == oracle.hypervolume(pts[keep], ref)


@pytest.mark.parametrize("span,F,noise", [(25, 30000, 3), (40, 30000, 2)])
def test_hv4_large_fronts_streamed(M, oracle, span, F, noise):
    # K = 4 fronts of about 8000 and 19000 points (beyond the shared-memory form: the slabs
    # are streamed in chunks, sub-slabs walked in batches), with ties in every objective
    rng = np.random.default_rng(span)
    pts = rng.integers(0, span, size=(F, 4)).astype(np.int64)
    pts[:, -1] = span * 3 - pts[:, :-1].sum(axis=1) + rng.integers(0, noise, F)
    ref = np.zeros(4, np.int64)
    front = pts[oracle.pareto_filter(pts)]
    assert len(front) > 6144
    want = oracle.hypervolume(front, ref)
    assert _hv_points(M, front, ref) == want
    assert _hv_points(M, pts, ref) == want  # dominated points add nothing


@pytest.mark.parametrize("K,count", [(2, 131), (3, 9), (4, 6)])
def test_hv_many_equals_one_call_per_archive(M, P, oracle, K, count):
    # moq_hypervolume_many over archives of one K (more than one 128-archive chunk for K = 2,
    # empty archives and fronts of different sizes included) gives each archive's exact
    # hypervolume: the oracle's on the oracle's filter of its candidates, and moq_hypervolume's
    rng = np.random.default_rng(K * 1000 + count)
    n = 70
    archs, refs, want = [], [], []
    for i in range(count):
        arch = P.Archive(n, K, capacity=1 << 14, max_batch=4096)
        m = 0 if i % 5 == 3 else int(rng.integers(1, 3000 if K < 4 else 800))
        span = int(rng.integers(20, 10 ** 6))
        c = rng.integers(0, span, size=(max(m, 1), K)).astype(np.int64)
        if K >= 3 and m:
            c[: m // 2, -1] = 2 * span - c[: m // 2, :-1].sum(axis=1)
        ref = rng.integers(-span // 4, span // 8, size=K).astype(np.int64)
        if m:
            arch.merge(_dev(c[:m], torch.int64), _bits_dev(wl.random_sign_bits(m, n, i)), m, 0)
            front = c[:m][oracle.pareto_filter(c[:m])]
            want.append(oracle.hypervolume(front, ref))
        else:
            want.append(0)
        archs.append(arch)
        refs.append(ref)
    got = P.Archive.hypervolume_many(archs, refs)
    assert got == want
    assert got == [a.hypervolume(r) for a, r in zip(archs, refs)]
    assert P.Archive.hypervolume_many(archs, refs) == want  # a second call on the same archives
    other = P.Archive(n, 5, capacity=64, max_batch=64)
    with pytest.raises(M.MoqError) as e:
        P.Archive.hypervolume_many([archs[0], other], [np.zeros(5, np.int64), np.zeros(5, np.int64)])
    assert e.value.code == M.MOQ_ERR_ARG
    other.close()
    # an archive whose merge overflowed: the call reports it (as moq_archive_size does) and
    # clears the latch, so the next call gives every hypervolume again
    small = P.Archive(n, K, capacity=8, max_batch=64)
    anti = np.zeros((9, K), np.int64)
    anti[:, 0] = np.arange(9)
    anti[:, 1] = 20 - np.arange(9)
    with pytest.raises(M.MoqError):  # the merge itself reports the overflow
        small.merge(_dev(anti, torch.int64), _bits_dev(wl.random_sign_bits(9, n, 5)), 9, 0, want_size=True)
    small.merge(_dev(anti, torch.int64), _bits_dev(wl.random_sign_bits(9, n, 5)), 9, 0)  # latched, not read
    with pytest.raises(M.MoqError) as e:
        P.Archive.hypervolume_many([archs[1], small], [refs[1], np.zeros(K, np.int64)])
    assert e.value.code == M.MOQ_ERR_CAPACITY
    assert P.Archive.hypervolume_many([archs[1], small], [refs[1], np.zeros(K, np.int64)]) == [want[1], 0]
    small.close()
    for a in archs:
        a.close()


@pytest.mark.parametrize("F", [6143, 6144, 6145])
@pytest.mark.parametrize("wide", [False, True])
def test_hv4_at_the_shared_memory_limit(M, oracle, F, wide):
    # K = 4 point sets at the largest size the shared-memory slab kernels take (6144) and one
    # point either side, mostly on a front with ties; with one coordinate lifted 2^40 above the
    # reference the 128-bit walk runs instead of the 32-bit one
    rng = np.random.default_rng(F + 7 * wide)
    pts = rng.integers(0, 40, size=(F, 4)).astype(np.int64)
    pts[:, -1] = 120 - pts[:, :-1].sum(axis=1) + rng.integers(0, 2, F)
    if wide:
        pts[5, 0] = 1 << 40
    ref = np.array([-1, -2, 0, -3], np.int64)
    want = oracle.hypervolume(pts[oracle.pareto_filter(pts)], ref)
    assert _hv_points(M, pts, ref) == want


def test_hv_edge_cases(M, oracle):
    ref = np.zeros(3, np.int64)
    assert _hv_points(M, np.zeros((0, 3), np.int64), ref) == 0
    assert _hv_points(M, np.array([[5, 6, 7]], np.int64), ref) == 210
    assert _hv_points(M, np.array([[5, 6, 7], [5, 6, 7], [1, 1, 1]], np.int64), ref) == 210
    assert _hv_points(M, np.array([[5, -1, 7], [2, 2, 2]], np.int64), ref) == 8  # first spans nothing
    side = 1_500_000_000
    big = np.array([[side, side, side, side], [side + 7, 3, side, side]], np.int64)
    assert _hv_points(M, big, np.zeros(4, np.int64)) == side ** 4 + 7 * 3 * side * side
    with pytest.raises(M.MoqError) as e:
        _hv_points(M, np.ones((2, 5), np.int64), np.zeros(5, np.int64))
    assert e.value.code == M.MOQ_ERR_UNSUPPORTED


# ----------------------------------------------------------------------------- a2..a5
def _abs_force_scale(src, lam, phi, c0):
    """c0 * sum_j |J(c)_ij phi_j| per replica and spin (the normwise force bound)."""
    Jc = lam.astype(np.float64) @ src.w.astype(np.float64)  # (R, E)
    out = np.zeros(phi.shape)
    np.add.at(out.T, src.ei, (np.abs(Jc * phi[:, src.ej])).T)
    np.add.at(out.T, src.ej, (np.abs(Jc * phi[:, src.ei])).T)
    return out * c0[:, None]


@pytest.mark.parametrize("name", ["heavyhex_K3", "heavyhex_K4", "reg3_n1024_K3", "gnp_n40_K2", "gnp_n70_K8"])
@pytest.mark.parametrize("variant", ["dsb", "bsb"])
def test_force_matches_fp64(M, P, oracle, name, variant):
    # one step with a_0 = a0 (no linear term), y0 = 0, alpha = 0 and dt = 2^-10: the
    # momentum after the step is dt * force exactly, so y_out / dt exposes the force
    src = INSTANCES[name]()
    inst = P.Instance(src)
    R = 67
    lam = wl.dirichlet_lambdas(R, src.K, 3)
    rng = np.random.default_rng(1)
    x0 = rng.uniform(-0.5, 0.5, (R, src.n)).astype(np.float32)
    dt = 2.0 ** -10
    y_out = torch.zeros((R, src.n), dtype=torch.float32, device="cuda")
    x_out = torch.zeros_like(y_out)
    p = M.moq_default_params(variant=variant, steps=1, dt=dt, a0=1.0, alpha=0.0,
                             schedule=torch.ones(1, device="cuda"), x_init=_dev(x0, torch.float32),
                             y_init=torch.zeros((R, src.n), device="cuda"), x_out=x_out, y_out=y_out)
    bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
    M.moq_sample(inst.handle, _dev(lam, torch.float32), R, p, 0, 0, bits)
    ref = oracle.sb(src, lam.astype(np.float64), variant=variant, steps=1, dt=dt, a0=1.0, alpha=0.0,
                    schedule=[1.0], x_init=x0.astype(np.float64), y_init=np.zeros((R, src.n)))
    f_gpu = y_out.cpu().numpy().astype(np.float64) / dt
    f_ref = ref["y"] / dt
    phi = np.where(x0 >= 0, 1.0, -1.0) if variant == "dsb" else x0.astype(np.float64)
    scale = _abs_force_scale(src, lam, phi, ref["c0"])
    err = np.abs(f_gpu - f_ref)
    assert np.all(err <= FORCE_RTOL * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())
    assert np.allclose(x_out.cpu().numpy(), ref["x"], rtol=0, atol=1e-6)


def test_one_step_golden(M, P):
    lines = golden_lines("sb_one_step.txt")
    rows = [[int(t) for t in l.split()[1:]] for l in lines if l.startswith("edge")]
    src = wl.Instance(3, np.array([r[0] for r in rows], np.int32), np.array([r[1] for r in rows], np.int32),
                      np.array([r[2:] for r in rows], np.int32).T.copy())
    inst = P.Instance(src)
    lam = np.array([[float(v) for v in [l for l in lines if l.startswith("lambda")][0].split()[1:]]], np.float32)
    for c in [l for l in lines if l.startswith("case")]:
        parts = c[4:].split("|")
        x0, y0, y1, x1 = (np.array([float(v) for v in q.split()], np.float32) for q in parts[1:])
        xo = torch.zeros((1, 3), device="cuda")
        yo = torch.zeros((1, 3), device="cuda")
        p = M.moq_default_params(variant=parts[0].strip(), steps=1, dt=0.5, a0=1.0, alpha=0.0,
                                 schedule=torch.full((1,), 0.5, device="cuda"), x_init=_dev(x0[None], torch.float32),
                                 y_init=_dev(y0[None], torch.float32), x_out=xo, y_out=yo)
        M.moq_sample(inst.handle, _dev(lam, torch.float32), 1, p, 0, 0, torch.zeros((1, 1), dtype=torch.int64, device="cuda"))
        assert np.allclose(yo.cpu().numpy()[0], y1, atol=1e-6)
        assert np.allclose(xo.cpu().numpy()[0], x1, atol=1e-6)


def test_initial_state_bit_exact(M, P, oracle):
    src = INSTANCES["heavyhex_K3"]()
    inst = P.Instance(src)
    R = 40
    xo = torch.zeros((R, src.n), device="cuda")
    yo = torch.zeros((R, src.n), device="cuda")
    p = M.moq_default_params(steps=0, init_amp=0.1, x_out=xo, y_out=yo)
    bits = torch.zeros((R, 1), dtype=torch.int64, device="cuda")
    M.moq_sample(inst.handle, _dev(wl.dirichlet_lambdas(R, 3, 0), torch.float32), R, p, 12345, 6, bits)
    want = np.array([[oracle.initial_state(12345, 6, r, i, 0.1) for i in range(src.n)] for r in range(R)])
    assert np.array_equal(xo.cpu().numpy().astype(np.float64), want[..., 0])
    assert np.array_equal(yo.cpu().numpy().astype(np.float64), want[..., 1])
    s = wl.bits_to_signs(_bits_host(bits), src.n)
    assert np.array_equal(s, np.where(want[..., 0] >= 0, 1, -1))


def test_kernel_noise_against_the_oracle_gaussian(M, P, oracle):
    # The samplers draw eta by Box-Muller on the two 16-bit halves of a Philox word, a
    # cheaper generator than the oracle's 53-bit uniforms (the paper's standard Gaussian).
    # Measured against the oracle: with J = 0, x = y = 0 and a = a0, one step leaves
    # y = dt * alpha * eta. The kernel's law agrees with the oracle's by a two-sample KS test
    # on millions of draws, and its one departure is the bound |eta| <= sqrt(32 ln 2) = 4.71
    # (a Gaussian exceeds it with probability 2.5e-6; the oracle's tail is pinned on the CPU).
    n, R = 1000, 4096
    ring = np.arange(n, dtype=np.int32)
    nxt = np.roll(ring, -1)
    src = wl.Instance(n, np.minimum(ring, nxt), np.maximum(ring, nxt), np.zeros((2, n), np.int32))
    inst = P.Instance(src)
    yo = torch.zeros((R, n), device="cuda")
    z = torch.zeros((R, n), device="cuda")
    p = M.moq_default_params(steps=1, dt=0.5, alpha=0.2, schedule=torch.ones(1, device="cuda"), x_init=z, y_init=z,
                             y_out=yo)
    M.moq_sample(inst.handle, _dev(np.full((R, 2), 0.5), torch.float32), R, p, 21, 0,
                 torch.zeros((R, inst.W), dtype=torch.int64, device="cuda"))
    eta = yo.cpu().numpy().ravel().astype(np.float64) / (0.5 * 0.2)
    want = np.concatenate([oracle.normals(21, 0, r, 0, 0, 250_000) for r in range(4)])
    assert abs(eta.mean()) < 2e-3 and abs(eta.var() - 1.0) < 3e-3
    assert stats.ks_2samp(eta, want).pvalue > 1e-3
    assert np.abs(eta).max() <= np.sqrt(32 * np.log(2)) * (1 + 1e-6)
    assert np.abs(eta).max() > 4.0  # the bound is reached, not a narrower law


@pytest.mark.parametrize("T,variant,schedule", [(1, "bsb", False), (2, "bsb", False), (3, "bsb", True),
                                                 (6, "bsb", False), (7, "bsb", True), (25, "bsb", False),
                                                 (9, "dsb", False), (11, "dsb", True)])
def test_short_trajectory(M, P, oracle, T, variant, schedule):
    # without noise a few FP32 steps stay close to the FP64 trajectory (step counts that
    # are not multiples of four exercise the unrolled loop's tail); dSB is compared only
    # on replicas whose start has no spin within 1e-3 of the sign switch
    src = INSTANCES["heavyhex_K4"]()
    inst = P.Instance(src)
    R = 64
    lam = wl.dirichlet_lambdas(R, 4, 5)
    xo = torch.zeros((R, src.n), device="cuda")
    yo = torch.zeros((R, src.n), device="cuda")
    sched = np.linspace(0.0, 1.0, T) ** 2 if schedule else None
    p = M.moq_default_params(variant=variant, steps=T, dt=0.5, x_out=xo, y_out=yo,
                             schedule=None if sched is None else _dev(sched, torch.float32))
    bits = torch.zeros((R, 1), dtype=torch.int64, device="cuda")
    M.moq_sample(inst.handle, _dev(lam, torch.float32), R, p, 3, 0, bits)
    ref = oracle.sb(src, lam.astype(np.float64), variant=variant, steps=T, dt=0.5, seed=3,
                    schedule=None if sched is None else sched.astype(np.float32).astype(np.float64))
    ok = np.ones(R, bool)
    if variant == "dsb":
        x0 = np.array([[oracle.initial_state(3, 0, r, i)[0] for i in range(src.n)] for r in range(R)])
        ok = np.all(np.abs(x0) > 1e-3, axis=1)
        assert ok.sum() >= R // 4
    assert np.abs(xo.cpu().numpy()[ok] - ref["x"][ok]).max() < 1e-4
    assert np.abs(yo.cpu().numpy()[ok] - ref["y"][ok]).max() < 1e-4


@pytest.mark.parametrize("variant", ["dsb", "bsb"])
def test_sampler_invariants_and_determinism(M, P, variant):
    src = INSTANCES["reg3_n150_K3"]()
    inst = P.Instance(src)
    R = 300
    lam = _dev(wl.dirichlet_lambdas(R, 3, 9), torch.float32)
    xo = torch.zeros((R, src.n), device="cuda")
    yo = torch.zeros((R, src.n), device="cuda")
    p = M.moq_default_params(variant=variant, steps=500, dt=0.5, alpha=0.15, x_out=xo, y_out=yo)
    b1 = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
    b2 = torch.zeros_like(b1)
    b3 = torch.zeros_like(b1)
    M.moq_sample(inst.handle, lam, R, p, 77, 1, b1)
    x, y = xo.cpu().numpy(), yo.cpu().numpy()
    assert np.all(np.abs(x) <= 1.0) and np.all(y[np.abs(x) == 1.0] == 0.0)
    assert np.array_equal(wl.bits_to_signs(_bits_host(b1), src.n), np.where(x >= 0, 1, -1))
    M.moq_sample(inst.handle, lam, R, p, 77, 1, b2)
    assert torch.equal(b1, b2)  # same seed and round: identical
    M.moq_sample(inst.handle, lam, R, p, 77, 2, b3)
    assert not torch.equal(b1, b3)


def test_handles_reuse_pooled_memory(M, P):
    # instances and archives take their arrays from the library's memory pool: handles of the
    # same size come back after destruction, the cached memory can be returned to the driver,
    # and handles made before and after give the same results
    src = INSTANCES["heavyhex_K3"]()
    R = 512
    lam = _dev(wl.dirichlet_lambdas(R, 3, 2), torch.float32)
    params = M.moq_default_params(variant="dsb", steps=64, dt=0.5, alpha=0.1)
    hvs = []
    for it in range(3):
        inst = P.Instance(src)
        arch = P.Archive(src.n, src.K, capacity=1 << 12, max_batch=R)
        buf = P.RoundBuffers(R, src.n, src.K)
        P.sample_round(inst, arch, buf, params, 5, 0, lam=lam)
        hvs.append(arch.hypervolume(inst.ref))
        arch.close()
        inst.close()
        if it == 1:
            M.moq_release_cached_memory()
    assert hvs[0] == hvs[1] == hvs[2] > 0


@pytest.mark.parametrize("world", [2, 3])
def test_replica_shards_reproduce_one_call(M, P, world):
    # the multi-GPU path: each rank samples a contiguous replica shard with the shard's first
    # replica as offset; together the shards are bit-identical to one call over all replicas
    from paper_2604_26477_b300.shard import replica_shard
    src = INSTANCES["heavyhex_K4"]()
    inst = P.Instance(src)
    R = 1001
    lam = _dev(wl.dirichlet_lambdas(R, 4, 12), torch.float32)
    whole = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
    M.moq_sample(inst.handle, lam, R, M.moq_default_params(variant="dsb", steps=400, dt=0.5, alpha=0.1), 5, 3, whole)
    for q in range(world):
        first, count = replica_shard(R, q, world)
        part = torch.zeros((count, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(variant="dsb", steps=400, dt=0.5, alpha=0.1, replica_offset=first)
        M.moq_sample(inst.handle, lam[first:first + count].contiguous(), count, p, 5, 3, part)
        assert torch.equal(part, whole[first:first + count])


@pytest.mark.parametrize("name,R,T,variant,alpha,sched,state", [
    ("heavyhex_K4", 1001, 203, "dsb", 0.1, False, False), ("heavyhex_K3", 77, 96, "bsb", 0.1, True, True),
    ("heavyhex_K4", 2, 13, "dsb", 0.0, False, True), ("reg3_n1024_K3", 9, 64, "dsb", 0.15, False, False),
    ("reg4_n300_K3", 31, 101, "bsb", 0.0, False, False), ("reg3_n150_K3", 5, 42, "dsb", 0.1, False, True),
    ("triangle_K2", 301, 50, "dsb", 0.2, False, False)])
def test_replica_pairs_match_single_replica_threads(M, P, monkeypatch, name, R, T, variant, alpha, sched, state):
    # the sampler form with two replicas per thread (float2 gathers, shared pump and barrier)
    # and the one-replica form give the same samples and final x, y bit for bit: odd and tiny
    # R (a half-empty last pair), step counts with tails, both variants, with and without
    # noise, an explicit pump, caller start states, degree bounds 3 and 4
    if name == "reg4_n300_K3":
        src = wl.random_regular(300, 9, K=3, d=4)
    elif name == "triangle_K2":  # n = 3: blocks of 3 Rp threads hold 4 Rp reduction slots
        src = wl.Instance(3, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32),
                          np.array([[3, -2, 5], [1, 4, -2]], np.int32))
    else:
        src = INSTANCES[name]()
    inst = P.Instance(src)
    n = src.n
    lam = _dev(wl.dirichlet_lambdas(R, src.K, 6), torch.float32)
    schedule = torch.linspace(0.0, 1.0, T, device="cuda") ** 0.5 if sched else None
    rng = np.random.default_rng(8)
    x0 = _dev(rng.uniform(-0.2, 0.2, (R, n)), torch.float32) if state else None
    y0 = _dev(rng.uniform(-0.1, 0.1, (R, n)), torch.float32) if state else None
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MOQ_SB_PAIR", mode)
        xo = torch.zeros((R, n), device="cuda")
        yo = torch.zeros((R, n), device="cuda")
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(variant=variant, steps=T, dt=0.5, alpha=alpha, schedule=schedule, x_init=x0, y_init=y0,
                                 x_out=xo, y_out=yo, replica_offset=3)
        M.moq_sample(inst.handle, lam, R, p, 21, 4, bits)
        torch.cuda.synchronize()
        out[mode] = (bits.cpu(), xo.cpu(), yo.cpu())
    for a, b in zip(out["1"], out["0"]):
        assert torch.equal(a, b)
    assert R < 3 or len(torch.unique(out["1"][0], dim=0)) > 1


@pytest.mark.parametrize("variant", ["dsb", "bsb"])
def test_bipartite_reaches_max_cut(M, P, variant):
    rows, cols = 6, 7
    e = []
    rng = np.random.default_rng(3)
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                e.append((v, v + 1))
            if r + 1 < rows:
                e.append((v, v + cols))
    ei = np.array([a for a, _ in e], np.int32)
    ej = np.array([b for _, b in e], np.int32)
    w = np.stack([rng.integers(1, 6, len(e)), rng.integers(-5, 6, len(e))]).astype(np.int32)
    src = wl.Instance(rows * cols, ei, ej, w)
    inst = P.Instance(src)
    R = 64
    lam = torch.tensor([[1.0, 0.0]] * R, device="cuda")
    bits = torch.zeros((R, 1), dtype=torch.int64, device="cuda")
    M.moq_sample(inst.handle, lam, R, M.moq_default_params(variant=variant, steps=600, dt=0.5), 5, 0, bits)
    cuts = torch.zeros((R, 2), dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, bits, R, cuts)
    c1 = cuts[:, 0].cpu().numpy()
    assert c1.max() == w[0].sum() and np.mean(c1 == w[0].sum()) >= 0.5


def test_sampler_recovers_bruteforce_front(M, P, oracle):
    src = wl.random_graph(12, 0.5, 21, K=3, wmax=10)
    bf_bits, bf_cuts = oracle.brute_force(src)
    front = bf_cuts[oracle.pareto_filter(bf_cuts)]
    inst = P.Instance(src)
    R = 4096
    arch = P.Archive(src.n, 3, capacity=4096, max_batch=R)
    buf = P.RoundBuffers(R, src.n, 3)
    params = M.moq_default_params(steps=200, dt=0.5, alpha=0.3)
    for rnd in range(2):
        P.sample_round(inst, arch, buf, params, seed=2, round_=rnd)
    gc, gb, gi = arch.copy_out()
    fset = {tuple(v) for v in front}
    assert {tuple(v) for v in gc} <= fset  # every archived vector is a true front vector
    assert len(gc) >= 0.8 * len(fset)
    assert arch.hypervolume(inst.ref) >= 0.98 * oracle.hypervolume(front, inst.ref)
    # the archived representatives have exactly the archived cut vectors
    assert np.array_equal(oracle.cuts(src, gb), gc)


def test_final_hv_distribution_matches_oracle(M, P, oracle):
    # chaotic trajectories: compare the distribution of the final front's hypervolume
    # over 32 seeds (two-sample Mann-Whitney U) between the GPU and the FP64 oracle
    src = INSTANCES["heavyhex_K3"]()
    inst = P.Instance(src)
    R, T = 128, 300
    lam = wl.dirichlet_lambdas(R, 3, 77)
    lam_d = _dev(lam, torch.float32)
    params = M.moq_default_params(steps=T, dt=0.5, alpha=0.15)
    bits = torch.zeros((R, 1), dtype=torch.int64, device="cuda")
    hv_gpu, hv_cpu = [], []
    for seed in range(32):
        M.moq_sample(inst.handle, lam_d, R, params, seed, 0, bits)
        c = oracle.cuts(src, _bits_host(bits))
        hv_gpu.append(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref))
        o = oracle.sb(src, lam.astype(np.float64), steps=T, dt=0.5, alpha=0.15, seed=1000 + seed)
        c = oracle.cuts(src, o["bits"])
        hv_cpu.append(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref))
    p = stats.mannwhitneyu(hv_gpu, hv_cpu).pvalue
    assert p > 0.01, (p, np.median(hv_gpu), np.median(hv_cpu))
    assert abs(np.median(hv_gpu) / np.median(hv_cpu) - 1) < 0.02


def test_sampler_rejects_what_it_does_not_run(M, P):
    lam = torch.full((8, 3), 1.0 / 3, device="cuda")
    bits = torch.zeros((8, 17), dtype=torch.int64, device="cuda")
    big = P.Instance(wl.random_regular(1026, 3, K=3))  # n > 1024: beyond the on-chip sampler
    with pytest.raises(M.MoqError) as e:
        M.moq_sample(big.handle, lam, 8, M.moq_default_params(steps=4), 1, 0, bits)
    assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    star = wl.Instance(20, np.zeros(19, np.int32), np.arange(1, 20, dtype=np.int32), np.ones((3, 19), np.int32))
    hub = P.Instance(star)  # a vertex of degree 19 > 16
    with pytest.raises(M.MoqError) as e:
        M.moq_sample(hub.handle, lam, 8, M.moq_default_params(steps=4), 1, 0, bits)
    assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    small = P.Instance(INSTANCES["heavyhex_K3"]())
    with pytest.raises(M.MoqError) as e:
        M.moq_sample(small.handle, lam, 8, M.moq_default_params(steps=4, variant=7), 1, 0, bits)
    assert e.value.code == M.MOQ_ERR_ARG
    with pytest.raises(M.MoqError) as e:
        M.moq_sample(small.handle, lam, -1, M.moq_default_params(steps=4), 1, 0, bits)
    assert e.value.code == M.MOQ_ERR_ARG
    M.moq_sample(small.handle, lam, 0, M.moq_default_params(steps=4), 1, 0, bits)  # R = 0: nothing to do


# ----------------------------------------------------------------------------- lambda
def test_das_dennis_lattice(M, oracle):
    for K, H in [(3, 21), (4, 13), (2, 9), (5, 7)]:
        want = oracle.das_dennis(K, H, True)
        buf = torch.zeros((len(want) + 5, K), device="cuda")
        cnt = M.moq_lambda_das_dennis(K, H, True, buf, len(want) + 5)
        assert cnt == len(want)
        assert np.abs(buf[:cnt].cpu().numpy() - want).max() < 1e-6
        assert np.array_equal(np.rint(buf[:cnt].cpu().numpy() * H).astype(int), np.rint(want * H).astype(int))
    with pytest.raises(M.MoqError) as e:
        M.moq_lambda_das_dennis(3, 21, True, torch.zeros((10, 3), device="cuda"), 10)
    assert e.value.code == M.MOQ_ERR_CAPACITY


def test_dirichlet_matches_oracle(M, oracle):
    R, K = 5000, 4
    buf = torch.zeros((R, K), device="cuda")
    M.moq_lambda_dirichlet(K, R, 99, 3, buf)
    want = oracle.dirichlet(R, K, 99, 3)
    assert np.abs(buf.cpu().numpy() - want).max() < 2e-6


# ----------------------------------------------------------------------------- full path
def test_full_round_matches_oracle(M, P, oracle):
    # the benchmark's launch configuration: n=42, K=4, 16384 replicas, dSB; cuts, front
    # and hypervolume of the GPU samples must equal the oracle's on the same samples
    src = wl.heavy_hex_like(1001, K=4)
    inst = P.Instance(src)
    R = 16384
    arch = P.Archive(src.n, 4, capacity=1 << 16, max_batch=R)
    buf = P.RoundBuffers(R, src.n, 4)
    params = M.moq_default_params(steps=2000, dt=0.5, alpha=0.1)  # the benchmark's T
    P.sample_round(inst, arch, buf, params, seed=1, round_=0)
    bits = _bits_host(buf.bits)
    cuts = oracle.cuts(src, bits)
    assert np.array_equal(buf.cuts.cpu().numpy(), cuts)
    keep = oracle.pareto_filter(cuts)
    gc, gb, gi = arch.copy_out()
    assert np.array_equal(gi, keep) and np.array_equal(gc, cuts[keep])
    assert np.array_equal(gb, _canonical(bits[keep], src.n))
    assert len(keep) > 1000  # a front of the benchmark's size (about 2300 points)
    assert arch.hypervolume(inst.ref) == oracle.hypervolume(cuts[keep], inst.ref)


@pytest.mark.parametrize("K,max_batch", [(3, 4096), (4, 700)])
def test_archive_merge_is_the_front_of_the_union(M, P, oracle, K, max_batch):
    # two archives fed disjoint rounds, merged, hold exactly the front one archive fed every
    # round holds -- the oracle's filter of the whole pool, each vector with its lowest global
    # index -- also when the source front enters in several batches (max_batch < its size)
    src = wl.heavy_hex_like(1003, K=K)
    inst = P.Instance(src)
    R = 2048
    params = M.moq_default_params(steps=300, dt=0.5, alpha=0.1)
    a = P.Archive(src.n, K, capacity=1 << 16, max_batch=max_batch)
    b = P.Archive(src.n, K, capacity=1 << 16, max_batch=R)
    whole = P.Archive(src.n, K, capacity=1 << 16, max_batch=R)
    buf = P.RoundBuffers(R, src.n, K)
    pool_cuts, pool_bits = [], []
    for rnd in range(4):
        M.moq_lambda_dirichlet(K, R, 5, rnd, buf.lam)
        M.moq_sample(inst.handle, buf.lam, R, params, 5, rnd, buf.bits)
        M.moq_evaluate_cuts(inst.handle, buf.bits, R, buf.cuts)
        if rnd < 2:
            for o in range(0, R, max_batch):
                m = min(max_batch, R - o)
                a.merge(buf.cuts[o:o + m], buf.bits[o:o + m], m, rnd * R + o)
        else:
            b.merge(buf.cuts, buf.bits, R, rnd * R)
        whole.merge(buf.cuts, buf.bits, R, rnd * R)
        pool_cuts.append(buf.cuts.cpu().numpy())
        pool_bits.append(_bits_host(buf.bits).copy())
    a.merge_from(b)
    ca, ba, ia = a.copy_out()
    cw, bw, iw = whole.copy_out()
    oa, ow = np.argsort(ia), np.argsort(iw)
    assert np.array_equal(ia[oa], iw[ow]) and np.array_equal(ca[oa], cw[ow]) and np.array_equal(ba[oa], bw[ow])
    cuts = np.concatenate(pool_cuts)
    keep = oracle.pareto_filter(cuts)
    assert np.array_equal(np.sort(ia), keep) and np.array_equal(ca[oa], cuts[keep])
    assert np.array_equal(ba[oa], _canonical(np.concatenate(pool_bits)[keep], src.n))
    assert len(keep) > max_batch or K == 3
    with pytest.raises(M.MoqError) as e:
        a.merge_from(a)
    assert e.value.code == M.MOQ_ERR_ARG
    for x in (a, b, whole):
        x.close()


def test_exhaustive_front_matches_brute_force(M, P, oracle):
    # the enumeration behind the Appendix E reference fronts (pipeline.exhaustive_front, GPU
    # cuts and merges in chunks of 2^20) against the oracle's brute force and filter: the same
    # front, the same hypervolume, the same per-objective minima (n = 22: two chunks)
    src = wl.app_e_correlated(22, 1.0, 9)
    inst = P.Instance(src)
    arch, lo = P.exhaustive_front(inst)
    gc, gb, gi = arch.copy_out()
    bits, cuts = oracle.brute_force(src)
    keep = oracle.pareto_filter(cuts)
    assert {tuple(v) for v in gc.tolist()} == {tuple(v) for v in cuts[keep].tolist()}
    assert np.array_equal(lo.cpu().numpy(), cuts.min(axis=0))
    ref = cuts.min(axis=0) - 1
    assert arch.hypervolume(ref) == oracle.hypervolume(cuts[keep], ref)
    assert np.array_equal(oracle.cuts(src, gb), gc)  # each representative has its cut vector
    arch.close()


@pytest.mark.parametrize("variant,alpha", [("dsb", 0.1), ("bsb", 0.0), ("bsb", 0.2)])
@pytest.mark.parametrize("n,d,R", [(1024, 3, 601), (700, 3, 1021), (650, 4, 999), (100, 3, 37)])
def test_two_spins_per_thread_give_the_pair_form_bits(M, P, monkeypatch, variant, alpha, n, d, R):
    # two spins per thread (taken by default for n > 640; MOQ_SB_TWOSPIN forces either form):
    # each replica's arithmetic and noise counters are the pair form's, ragged R and T included
    src = wl.random_regular(n, 45, K=3, d=d)
    inst = P.Instance(src)
    lam = torch.from_numpy(wl.dirichlet_lambdas(R, 3, 7)).cuda()
    out = {}
    for two in ("0", "1"):
        monkeypatch.setenv("MOQ_SB_TWOSPIN", two)
        monkeypatch.setenv("MOQ_SB_PAIR", "1")
        xo = torch.zeros((R, n), device="cuda")
        yo = torch.zeros((R, n), device="cuda")
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(variant=variant, steps=203, dt=0.5, alpha=alpha, x_out=xo, y_out=yo)
        M.moq_sample(inst.handle, lam, R, p, 9, 3, bits)
        out[two] = (bits.cpu(), xo.cpu(), yo.cpu())
    for a, b in zip(out["0"], out["1"]):
        assert torch.equal(a, b)


def test_two_spins_per_thread_from_a_given_state_and_schedule(M, P, monkeypatch):
    n, R, T = 900, 300, 120
    src = wl.random_regular(n, 46, K=3)
    inst = P.Instance(src)
    lam = torch.from_numpy(wl.dirichlet_lambdas(R, 3, 8)).cuda()
    g = torch.Generator().manual_seed(4)
    x0 = (torch.rand((R, n), generator=g) - 0.5).cuda()
    y0 = (0.2 * torch.randn((R, n), generator=g)).cuda()
    sched = torch.linspace(0.0, 1.3, T).float().cuda()
    out = {}
    for two in ("0", "1"):
        monkeypatch.setenv("MOQ_SB_TWOSPIN", two)
        monkeypatch.setenv("MOQ_SB_PAIR", "1")
        xo = torch.zeros((R, n), device="cuda")
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(steps=T, dt=0.5, alpha=0.1, x_init=x0, y_init=y0, x_out=xo, schedule=sched)
        M.moq_sample(inst.handle, lam, R, p, 8, 0, bits)
        out[two] = (bits.cpu(), xo.cpu())
    assert torch.equal(out["0"][0], out["1"][0]) and torch.equal(out["0"][1], out["1"][1])


@pytest.mark.parametrize("layout", ["0", "1", "long"])
@pytest.mark.parametrize("form", ["single", "pair", "two_spin"])
@pytest.mark.parametrize("name,variant", [("reg3_n1024_K3", "dsb"), ("reg3_n1024_K3", "bsb"), ("heavyhex_K4", "bsb")])
def test_force_matches_fp64_in_every_form_and_layout(M, P, oracle, monkeypatch, layout, form, name, variant):
    # the one-step force of every FP32 sparse form, on the bank-conflict layout (gather order
    # changes the FP32 summation order only), with the longer search for regular graphs, and
    # on the plain one, within the normwise bound
    monkeypatch.setenv("MOQ_SB_LAYOUT", "0" if layout == "0" else "1")
    monkeypatch.setenv("MOQ_SB_LAYOUT_EFFORT", "300" if layout == "long" else "0")  # the longer search
    monkeypatch.setenv("MOQ_SB_PAIR", "0" if form == "single" else "1")
    monkeypatch.setenv("MOQ_SB_TWOSPIN", "1" if form == "two_spin" else "0")
    src = INSTANCES[name]()
    inst = P.Instance(src)
    R = 41
    lam = wl.dirichlet_lambdas(R, src.K, 5)
    rng = np.random.default_rng(2)
    x0 = rng.uniform(-0.5, 0.5, (R, src.n)).astype(np.float32)
    dt = 2.0 ** -10
    y_out = torch.zeros((R, src.n), dtype=torch.float32, device="cuda")
    x_out = torch.zeros_like(y_out)
    p = M.moq_default_params(variant=variant, steps=1, dt=dt, a0=1.0, alpha=0.0,
                             schedule=torch.ones(1, device="cuda"), x_init=_dev(x0, torch.float32),
                             y_init=torch.zeros((R, src.n), device="cuda"), x_out=x_out, y_out=y_out)
    bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
    M.moq_sample(inst.handle, _dev(lam, torch.float32), R, p, 0, 0, bits)
    ref = oracle.sb(src, lam.astype(np.float64), variant=variant, steps=1, dt=dt, a0=1.0, alpha=0.0,
                    schedule=[1.0], x_init=x0.astype(np.float64), y_init=np.zeros((R, src.n)))
    f_gpu = y_out.cpu().numpy().astype(np.float64) / dt
    phi = np.where(x0 >= 0, 1.0, -1.0) if variant == "dsb" else x0.astype(np.float64)
    scale = _abs_force_scale(src, lam, phi, ref["c0"])
    err = np.abs(f_gpu - ref["y"] / dt)
    assert np.all(err <= FORCE_RTOL * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())
    assert np.allclose(x_out.cpu().numpy(), ref["x"], rtol=0, atol=1e-6)
    got = wl.bits_to_signs(bits.cpu().numpy().view(np.uint64), src.n) < 0
    assert np.array_equal(got, x_out.cpu().numpy() < 0)


@pytest.mark.parametrize("n,R", [(641, 1), (641, 2), (999, 3), (1023, 5), (700, 64), (896, 3), (898, 2)])
def test_two_spins_and_quads_at_shape_edges(M, P, monkeypatch, n, R):
    # odd n, the first size past the block limit of the pair forms, replica counts below one
    # block, the last size of the two-spin build bounded for 448 threads (896) and the first
    # past it (898): the two-spin (FP32) and four-replica (FP16) forms against their pair
    # forms, bit for bit
    if n % 2:  # a 3-regular graph on n - 1 spins and one more spin joined to two of them
        base = wl.random_regular(n - 1, 47, K=3)
        ei = np.concatenate([base.ei, np.array([0, 1], np.int32)])
        ej = np.concatenate([base.ej, np.array([n - 1, n - 1], np.int32)])
        w = np.concatenate([base.w, np.array([[5, -7], [3, 9], [-2, 4]], np.int32)], axis=1)
        src = wl.Instance(n, ei, ej, w)
    else:
        src = wl.random_regular(n, 47, K=3)
    inst = P.Instance(src)
    lam = torch.from_numpy(wl.dirichlet_lambdas(R, 3, 9)).cuda()
    for prec, knob in (("fp32", "MOQ_SB_TWOSPIN"), ("fp16", "MOQ_SB_QUAD")):
        out = {}
        for v in ("0", "1"):
            monkeypatch.setenv(knob, v)
            monkeypatch.setenv("MOQ_SB_PAIR", "1")
            xo = torch.zeros((R, src.n), device="cuda")
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            p = M.moq_default_params(steps=77, dt=0.5, alpha=0.1, precision=prec, x_out=xo)
            M.moq_sample(inst.handle, lam, R, p, 10, 1, bits)
            out[v] = (bits.cpu(), xo.cpu())
        assert torch.equal(out["0"][0], out["1"][0]) and torch.equal(out["0"][1], out["1"][1]), prec


@pytest.mark.parametrize("Mtot", [3000, 20000])
def test_pareto_candidates_at_an_8_byte_offset(M, P, oracle, Mtot):
    # candidate cut vectors that start 8 bytes past a 16-byte boundary (a view into a larger
    # tensor): the same front as from an aligned copy, and the definition's
    K, n = 4, 42
    rng = np.random.default_rng(Mtot)
    cuts = rng.integers(-30, 30, size=(Mtot, K)).astype(np.int64)
    cuts[::9] = cuts[4]
    bits = wl.random_sign_bits(Mtot, n, 3)
    raw = torch.zeros(Mtot * K + 1, dtype=torch.int64, device="cuda")
    view = raw[1:].view(Mtot, K)
    view.copy_(torch.from_numpy(cuts))
    assert view.data_ptr() % 16 == 8
    fronts = []
    for c in (view, _dev(cuts, torch.int64)):
        arch = P.Archive(n, K, capacity=1 << 14, max_batch=Mtot)
        arch.merge(c, _bits_dev(bits), Mtot, 0)
        fronts.append(arch.copy_out())
        arch.close()
    for a, b in zip(*fronts):
        assert np.array_equal(a, b)
    keep = oracle.pareto_filter(cuts)  # pool indices (ascending) of the distinct non-dominated vectors
    assert np.array_equal(fronts[0][0], cuts[keep]) and np.array_equal(fronts[0][2], keep)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_layout_argument_reproduces_the_environment_choice(M, P, monkeypatch, precision):
    # moq_create_instance_layout with MOQ_LAYOUT_PLAIN, MOQ_LAYOUT_DEFAULT and an effort m > 0
    # builds the instances that moq_create_instance builds under MOQ_SB_LAYOUT=0, the default
    # environment and MOQ_SB_LAYOUT_EFFORT=m: the same samples and end states, bit for bit; and
    # the argument wins over the environment
    src = wl.random_regular(300, 11, K=3)
    R, T = 203, 90
    lam = _dev(wl.dirichlet_lambdas(R, src.K, 4), torch.float32)

    def sample(inst):
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        xo = torch.zeros((R, src.n), device="cuda")
        p = M.moq_default_params(steps=T, dt=0.5, alpha=0.1, x_out=xo, precision=precision)
        M.moq_sample(inst.handle, lam, R, p, 5, 1, bits)
        torch.cuda.synchronize()
        out = (bits.cpu(), xo.cpu())
        inst.close()
        return out

    cases = [("0", "0", M.MOQ_LAYOUT_PLAIN), ("1", "0", M.MOQ_LAYOUT_DEFAULT), ("1", "300", 300)]
    for env_layout, env_effort, arg in cases:
        monkeypatch.setenv("MOQ_SB_LAYOUT", env_layout)
        monkeypatch.setenv("MOQ_SB_LAYOUT_EFFORT", env_effort)
        by_env = sample(P.Instance(src))
        monkeypatch.setenv("MOQ_SB_LAYOUT", "1" if env_layout == "0" else "0")  # the argument wins
        by_arg = sample(P.Instance(src, layout=arg))
        assert torch.equal(by_env[0], by_arg[0]) and torch.equal(by_env[1], by_arg[1])
    with pytest.raises(M.MoqError):
        P.Instance(src, layout=-2)
