"""Host logic of the multi-GPU path: one process per GPU, replica shards, one optional
exchange of fronts.

The units of the method -- (instance, weight vector, replica) -- are independent (the paper
runs every weight vector and replica in one parallel run), so N ranks split the replica
range and sample with no communication. With ``replica_offset`` = the shard's first replica,
the noise counters of every replica are those of a single call over the whole range, so the
union of the shards' samples equals that call's samples bit for bit.

The only exchange is optional and happens once, after sampling: every rank's archive front
is gathered to all ranks, where the union is filtered again (the front of a union is the
front of the union of the parts' fronts). Timings are combined as the maximum over ranks.
All collectives go through ``torch.distributed`` (NCCL on GPUs, gloo on the CPU); nothing
here does arithmetic of the method.
"""
from __future__ import annotations

import socket
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as dist


def free_port() -> int:
    """A TCP port on 127.0.0.1 that is free right now (for the rendezvous of a local launch)."""
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch_ranks(n: int, script_argv: list[str], master_port: int | None = None) -> int:
    """Runs ``python <script_argv>`` as n processes on this node (one per GPU) through
    torch.distributed.run, with the rendezvous on 127.0.0.1; each process reads RANK,
    LOCAL_RANK and WORLD_SIZE from its environment. Returns the launcher's exit code."""
    if n < 1:
        raise ValueError("need n >= 1")
    port = master_port or free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={port}"] + list(script_argv)
    return subprocess.call(cmd)


def replica_shard(R_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first replica, count) of rank's contiguous share of R_total replicas; the first
    R_total % world ranks take one more."""
    if world < 1 or not 0 <= rank < world or R_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, R_total >= 0")
    base, extra = divmod(R_total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def _device():
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(values) -> list[float]:
    """Element-wise maximum of a list of floats over all ranks (identity without a process group)."""
    t = torch.tensor(list(values), dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = t.to(_device())
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def sum_over_ranks(values) -> list[float]:
    """Element-wise sum of a list of floats over all ranks (identity without a process group)."""
    t = torch.tensor(list(values), dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = t.to(_device())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().tolist()


def gather_fronts(cuts: np.ndarray, bits: np.ndarray, index: np.ndarray):
    """All-gather every rank's front: returns (cuts, bits, index, rank_of_row) concatenated
    in rank order, the same on every rank. cuts is F x K int64, bits F x W uint64, index F
    int64 (the global sample index of each row)."""
    cuts = np.ascontiguousarray(cuts, np.int64)
    bits = np.ascontiguousarray(bits, np.uint64)
    index = np.ascontiguousarray(index, np.int64)
    F, K = cuts.shape
    W = bits.shape[1] if bits.ndim == 2 else 0
    if bits.shape[0] != F or index.shape != (F,):
        raise ValueError("cuts, bits and index must have the same number of rows")
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return cuts, bits, index, np.zeros(F, np.int64)
    world, dev = dist.get_world_size(), _device()
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([F], dtype=torch.int64, device=dev))
    sizes = [int(x.item()) for x in sizes]
    cap = max(max(sizes), 1)
    row = np.zeros((cap, K + W + 1), np.int64)  # one padded row layout: cuts | bits | index
    row[:F, :K] = cuts
    row[:F, K:K + W] = bits.view(np.int64)
    row[:F, K + W] = index
    send = torch.from_numpy(row).to(dev)
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send)
    parts = [r.cpu().numpy()[:s] for r, s in zip(recv, sizes)]
    allrows = np.concatenate(parts, axis=0)
    owner = np.concatenate([np.full(s, q, np.int64) for q, s in enumerate(sizes)])
    return (np.ascontiguousarray(allrows[:, :K]), np.ascontiguousarray(allrows[:, K:K + W]).view(np.uint64),
            np.ascontiguousarray(allrows[:, K + W]), owner)
