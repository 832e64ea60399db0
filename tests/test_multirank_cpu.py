"""The multi-GPU host logic on the CPU: replica shards, the max-over-ranks timing and the
one exchange of fronts, with two gloo ranks (no GPU)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_replica_shards_partition_the_range():
    from paper_2604_26477_b300.shard import replica_shard
    for R in (0, 1, 7, 1000, 1001, 16384):
        for world in (1, 2, 3, 8):
            shards = [replica_shard(R, q, world) for q in range(world)]
            assert sum(c for _, c in shards) == R
            assert shards[0][0] == 0
            for (f0, c0), (f1, _) in zip(shards, shards[1:]):
                assert f1 == f0 + c0  # contiguous, in rank order
            assert max(c for _, c in shards) - min(c for _, c in shards) <= 1
    with pytest.raises(ValueError):
        replica_shard(10, 2, 2)


def _all_cuts(R_total, K):
    """Stand-in for the cut vectors of one large call: a fixed function of the global
    replica index, so shards see exactly their slice (as replica offsets make the sampler do)."""
    rng = np.random.default_rng(31)
    cuts = rng.integers(0, 40, size=(R_total, K)).astype(np.int64)
    cuts[::9] = cuts[4]  # duplicates across the shard boundary
    bits = rng.integers(0, 2 ** 63, size=(R_total, 2), dtype=np.int64).view(np.uint64)
    return cuts, bits


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle as O
    from paper_2604_26477_b300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        R_total, K = 1001, 3
        first, count = shard.replica_shard(R_total, rank, world)
        cuts, bits = _all_cuts(R_total, K)
        c, b = cuts[first:first + count], bits[first:first + count]
        keep = O.pareto_filter(c)  # this rank's front (lowest local index per vector)
        g_cuts, g_bits, g_index, owner = shard.gather_fronts(c[keep], b[keep], first + keep)
        # front of the union = front of the union of the parts' fronts; rows arrive in rank
        # order, so the lowest global index of equal vectors comes first
        re = O.pareto_filter(g_cuts)
        want = O.pareto_filter(cuts)
        assert np.array_equal(g_index[re], want)
        assert np.array_equal(g_cuts[re], cuts[want])
        assert np.array_equal(g_bits[re], bits[want])
        assert np.array_equal(np.unique(owner), np.arange(world))
        assert shard.max_over_ranks([rank + 0.5, 10.0 - rank]) == [world - 0.5, 10.0]
        assert shard.sum_over_ranks([float(count)]) == [float(R_total)]
        with open(os.path.join(out_dir, f"ok{rank}"), "w") as fh:
            fh.write(str(len(re)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_fronts_and_time(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    sizes = {(tmp_path / f"ok{q}").read_text() for q in range(2)}
    assert len(sizes) == 1 and int(sizes.pop()) > 0


def test_single_process_is_the_identity():
    from paper_2604_26477_b300 import shard
    cuts, bits = _all_cuts(50, 2)
    out = shard.gather_fronts(cuts, bits, np.arange(50))
    assert np.array_equal(out[0], cuts) and np.array_equal(out[1], bits) and np.array_equal(out[2], np.arange(50))
    assert shard.max_over_ranks([1.0, 2.0]) == [1.0, 2.0]


def test_bench_launches_its_own_ranks():
    # bench.py --gpus 2 without a launcher around it starts two ranks itself (torch.distributed.run,
    # rendezvous on 127.0.0.1); the reference arm runs on rank 0 alone and prints one line
    import json
    import subprocess
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3", "--cpu-seconds", "1"],
                       capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["impl"] == "reference" and line["value"] > 0
