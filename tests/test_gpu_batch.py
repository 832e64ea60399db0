"""Batched sampling of uneven instances in one persistent launch: bit-exact against
single-instance calls with the same replica offsets (for every tile shape the autotuner
may pick), exact cuts against the oracle, the autotuner's choice, and a CUDA graph of
the batched round."""
import numpy as np
import pytest
import torch

from paper_2604_26477_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import moqaia
    return moqaia


@pytest.fixture(scope="module")
def P(M):
    from paper_2604_26477_b300 import pipeline
    return pipeline


def _srcs():
    return [wl.heavy_hex_like(1000, K=3), wl.random_regular(150, 7, K=3), wl.random_regular(1024, 8, K=3),
            wl.random_regular(500, 9, K=3), wl.heavy_hex_like(1002, K=3), wl.random_regular(64, 10, K=3)]


@pytest.fixture(scope="module")
def batch(P):
    srcs = _srcs()
    insts = [P.Instance(s) for s in srcs]
    reps = [300, 77, 5, 40, 1, 33]
    b = P.Batch(insts, reps)
    b.lam.copy_(torch.from_numpy(wl.dirichlet_lambdas(b.total_R, 3, 17)))
    return srcs, insts, b


@pytest.mark.parametrize("variant,alpha", [("dsb", 0.15), ("bsb", 0.0)])
@pytest.mark.parametrize("tile", [(1024, 1), (512, 2), (512, 4), (256, 4), (0, 0)])
def test_batch_matches_single_instance(M, P, batch, variant, alpha, tile):
    srcs, insts, b = batch
    b.set_tiles(*tile)
    params = M.moq_default_params(variant=variant, steps=301, dt=0.5, alpha=alpha)
    b.sample(params, seed=5, round_=2)
    for k, inst in enumerate(insts):
        R = int(b.replicas[k])
        lam = b.lam[int(b.rep_off[k]):int(b.rep_off[k + 1])].contiguous()
        single = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p1 = M.moq_default_params(variant=variant, steps=301, dt=0.5, alpha=alpha, replica_offset=int(b.rep_off[k]))
        M.moq_sample(inst.handle, lam, R, p1, 5, 2, single)
        assert torch.equal(b.bits_of(k), single), (k, tile)


def test_batch_cuts_exact(M, P, batch, oracle):
    srcs, insts, b = batch
    b.set_tiles(1024, 1)
    b.sample(M.moq_default_params(steps=100, dt=0.5, alpha=0.1), seed=1, round_=0)
    b.evaluate_cuts()
    for k, src in enumerate(srcs):
        bits = b.bits_of(k).cpu().numpy().view(np.uint64)
        assert np.array_equal(b.cuts_of(k).cpu().numpy(), oracle.cuts(src, bits))


def test_batch_tiles_and_tuner(M, P, batch, tmp_path, monkeypatch):
    srcs, insts, b = batch
    with pytest.raises(M.MoqError):
        b.set_tiles(256, 1)  # 256 slots cannot hold n = 1024
    with pytest.raises(M.MoqError):
        b.set_tiles(1024, 2)
    with pytest.raises(M.MoqError):
        b.set_tiles(1024, 4)
    monkeypatch.setenv("MOQ_TUNE_CACHE", str(tmp_path / "tiles.json"))
    from paper_2604_26477_b300 import autotune
    monkeypatch.setattr(autotune, "_CACHE_PATH", str(tmp_path / "tiles.json"))
    tile, timings = b.tune(M.moq_default_params(steps=200, dt=0.5, alpha=0.1), probe_steps=32)
    legal = autotune.legal(max(s.n for s in srcs))
    assert tile in legal and set(timings) == {f"{bd}x{spt}" for bd, spt in legal}
    assert {"1024x1", "512x2", "512x4", "256x4", "0x0"} <= set(timings)
    assert timings[f"{tile[0]}x{tile[1]}"] == min(timings.values())
    tile2, _ = b.tune(M.moq_default_params(steps=200, dt=0.5, alpha=0.1))  # from the cache
    assert tile2 == tile


@pytest.mark.parametrize("tile", [(512, 2), (0, 0)])
def test_batch_round_in_cuda_graph(M, P, batch, tile):
    srcs, insts, b = batch
    b.set_tiles(*tile)
    params = M.moq_default_params(steps=64, dt=0.5, alpha=0.1)
    b.sample(params, seed=3, round_=0)
    b.evaluate_cuts()
    torch.cuda.synchronize()
    want_bits, want_cuts = b.bits.clone(), b.cuts.clone()
    b.bits.zero_()
    b.cuts.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            b.sample(params, seed=3, round_=0, stream=s.cuda_stream)
            b.evaluate_cuts(stream=s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.bits, want_bits) and torch.equal(b.cuts, want_cuts)


@pytest.mark.parametrize("tile", [(1024, 1), (0, 0)])
def test_batch_active_replicas(M, P, tile):
    # moq_batch_set_replicas: instance b samples (and gets cuts for) its first replicas[b]
    # replicas only, 0 skipping it, with the layout and noise counters unchanged
    srcs = _srcs()
    insts = [P.Instance(s) for s in srcs]
    reps = [300, 77, 5, 40, 1, 33]
    b = P.Batch(insts, reps)
    b.lam.copy_(torch.from_numpy(wl.dirichlet_lambdas(b.total_R, 3, 18)))
    b.set_tiles(*tile)
    params = M.moq_default_params(steps=120, dt=0.5, alpha=0.1)
    b.sample(params, seed=4, round_=1)
    b.evaluate_cuts()
    full_bits, full_cuts = b.bits.clone(), b.cuts.clone()
    active = [0, 77, 5, 0, 1, 20]
    M.moq_batch_set_replicas(b.handle, np.array(active, np.int32))
    b.bits.fill_(-1)
    b.cuts.fill_(-1)
    b.sample(params, seed=4, round_=1)
    b.evaluate_cuts()
    torch.cuda.synchronize()
    for k, inst in enumerate(insts):
        bits_k, cuts_k = b.bits_of(k), b.cuts_of(k)
        a = active[k]
        want_b = full_bits[int(b.word_off[k]):int(b.word_off[k + 1])].view(reps[k], inst.W)
        assert torch.equal(bits_k[:a], want_b[:a])
        assert torch.equal(cuts_k[:a], full_cuts[int(b.rep_off[k]):int(b.rep_off[k]) + a])
        assert bool((bits_k[a:] == -1).all()) and bool((cuts_k[a:] == -1).all())  # untouched
    with pytest.raises(M.MoqError) as e:
        M.moq_batch_set_replicas(b.handle, np.array([301, 0, 0, 0, 0, 0], np.int32))
    assert e.value.code == M.MOQ_ERR_ARG


@pytest.mark.parametrize("batched,learned,prec", [(False, False, "fp32"), (True, False, "fp16"), (True, True, "fp16")])
def test_batch_time_to_target_reaches_every_instance(M, P, oracle, batched, learned, prec):
    # the batch driver stops each instance at its own target; the targets here are the
    # 99% of the hypervolume of the oracle's filter of one plain round, so every arm gets there
    srcs = [wl.random_regular(n, 60 + n, K=3) for n in (42, 130, 300)]
    R = 256
    targets = []
    for src in srcs:
        inst = P.Instance(src)
        buf = P.RoundBuffers(R, src.n, 3)
        arch = P.Archive(src.n, 3, capacity=1 << 14, max_batch=R)
        P.sample_round(inst, arch, buf, M.moq_default_params(steps=300, dt=0.5), seed=0, round_=0)
        c = oracle.cuts(src, buf.bits.cpu().numpy().view(np.uint64))
        targets.append(int(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref)) * 99 // 100)
        arch.close()
        inst.close()
    params = M.moq_default_params(steps=400, dt=0.5, alpha=0.1, precision=prec)
    res = P.time_to_target_batch(srcs, targets, params, R, seed=1, max_rounds=64, batched=batched, learned=learned)
    assert res["reached"] and all(1 <= r <= res["rounds"] for r in res["rounds_per_instance"])
    assert res["samples"] <= R * len(srcs) * res["rounds"]


def test_parallel_instance_builds_match_sequential_ones(M, P):
    # pipeline.create_instances builds on host threads (the layout planning runs in parallel):
    # every instance is the sequential build's, so the samples are the same bits
    srcs = _srcs()
    seq = [P.Instance(s) for s in srcs]
    par = P.create_instances(srcs)
    p = M.moq_default_params(steps=90, dt=0.5, alpha=0.1)
    for a, b, src in zip(seq, par, srcs):
        assert a.info == b.info
        lam = torch.from_numpy(wl.dirichlet_lambdas(70, 3, 12)).cuda()
        out = []
        for inst in (a, b):
            bits = torch.zeros((70, inst.W), dtype=torch.int64, device="cuda")
            M.moq_sample(inst.handle, lam, 70, p, 3, 1, bits)
            out.append(bits.cpu())
        assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("tile", [(1024, 1), (256, 4), (0, 0)])
def test_batch_with_degenerate_instances(M, P, oracle, tile):
    # a batch holding a graph without edges, the two-spin graph and isolated spins beside a
    # regular graph: every instance's samples equal its single-instance call, cuts the oracle's
    e0 = np.zeros(0, np.int32)
    srcs = [wl.Instance(5, e0, e0, np.zeros((3, 0), np.int32), name="edgeless5"),
            wl.Instance(2, np.array([0], np.int32), np.array([1], np.int32), np.array([[3], [-2], [7]], np.int32),
                        name="pair2"),
            wl.Instance(7, np.array([0, 2], np.int32), np.array([3, 6], np.int32),
                        np.array([[1, -4], [2, 2], [-9, 5]], np.int32), name="isolated7"),
            wl.random_regular(200, 12, K=3)]
    insts = [P.Instance(s) for s in srcs]
    reps = [19, 64, 7, 45]
    b = P.Batch(insts, reps)
    b.lam.copy_(torch.from_numpy(wl.dirichlet_lambdas(b.total_R, 3, 23)))
    b.set_tiles(*tile)
    params = M.moq_default_params(variant="dsb", steps=97, dt=0.5, alpha=0.15)
    b.sample(params, seed=4, round_=1)
    b.evaluate_cuts()
    for k, (src, inst) in enumerate(zip(srcs, insts)):
        R = int(b.replicas[k])
        lam = b.lam[int(b.rep_off[k]):int(b.rep_off[k + 1])].contiguous()
        single = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p1 = M.moq_default_params(variant="dsb", steps=97, dt=0.5, alpha=0.15, replica_offset=int(b.rep_off[k]))
        M.moq_sample(inst.handle, lam, R, p1, 4, 1, single)
        assert torch.equal(b.bits_of(k), single), (src.name, tile)
        bits = b.bits_of(k).cpu().numpy().view(np.uint64)
        assert np.array_equal(b.cuts_of(k).cpu().numpy(), oracle.cuts(src, bits)), src.name
    b.close()
    for h in insts:
        h.close()


@pytest.mark.parametrize("tile", [(512, 2), (0, 0)])
def test_zero_sized_calls(M, P, tile):
    # nothing to do is not an error: no replicas, no samples, no weight vectors, a batch whose
    # instances all have zero active replicas; the outputs around them stay untouched
    src = wl.random_regular(100, 3, K=3)
    inst = P.Instance(src)
    lam = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    bits = torch.full((1, inst.W), 7, dtype=torch.int64, device="cuda")
    for precision in ("fp32", "fp16"):
        M.moq_sample(inst.handle, lam, 0, M.moq_default_params(steps=10, precision=precision), 1, 0, bits)
    cuts = torch.full((1, 3), -5, dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, bits, 0, cuts)
    M.moq_lambda_dirichlet(3, 0, 1, 0, lam)
    arch = P.Archive(src.n, 3, capacity=16, max_batch=16)
    assert arch.merge(cuts, bits, 0, 0, want_size=True) == 0
    torch.cuda.synchronize()
    assert int(bits.min()) == 7 and int(bits.max()) == 7 and int(cuts.min()) == -5 and int(cuts.max()) == -5
    insts = [inst, P.Instance(wl.heavy_hex_like(1003, K=3))]
    b = P.Batch(insts, [8, 8])
    b.set_tiles(*tile)
    M.moq_batch_set_replicas(b.handle, np.zeros(2, np.int32))
    b.bits.fill_(3)
    b.cuts.fill_(-1)
    b.sample(M.moq_default_params(steps=10), seed=1, round_=0)
    b.evaluate_cuts()
    torch.cuda.synchronize()
    assert int(b.bits.min()) == 3 and int(b.bits.max()) == 3 and int(b.cuts.min()) == -1 and int(b.cuts.max()) == -1
    b.close()
    # the dense samplers and the dense cut evaluation with no replicas
    d = M.moq_dense_create(inst.handle, 64)
    d32 = M.moq_dense_fp32_create(inst.handle, 64)
    try:
        p = M.moq_default_params(steps=10)
        M.moq_sample_dense(d, lam, 0, p, 1, 0, bits)
        M.moq_sample_dense_fp8(d, lam, 0, p, 1, 0, bits)
        M.moq_sample_dense_split(d, lam, 0, p, 1, 0, bits)
        M.moq_sample_dense_fp32(d32, lam, 0, p, 1, 0, bits)
        M.moq_dense_evaluate_cuts(d, bits, 0, cuts)
        torch.cuda.synchronize()
        assert int(bits.min()) == 7 and int(bits.max()) == 7 and int(cuts.min()) == -5 and int(cuts.max()) == -5
    finally:
        M.moq_dense_destroy(d)
        M.moq_dense_fp32_destroy(d32)
    arch.close()
    for h in insts:
        h.close()
