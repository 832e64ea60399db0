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
@pytest.mark.parametrize("tile", [(1024, 1), (512, 2), (0, 0)])
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
    monkeypatch.setenv("MOQ_TUNE_CACHE", str(tmp_path / "tiles.json"))
    from paper_2604_26477_b300 import autotune
    monkeypatch.setattr(autotune, "_CACHE_PATH", str(tmp_path / "tiles.json"))
    tile, timings = b.tune(M.moq_default_params(steps=200, dt=0.5, alpha=0.1), probe_steps=32)
    assert tile in [(1024, 1), (512, 2), (0, 0)] and set(timings) == {"1024x1", "512x2", "0x0"}
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
