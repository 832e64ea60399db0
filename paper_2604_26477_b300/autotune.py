"""Autotuner for the batched sampler's tile shape.

For a batch of instances the persistent sampler can run with blocks of 256, 512 or 1024
threads and one or two spin slots per thread; the replicas per work item follow from the
tile (Rb = min(32, threads * slots / n)). The alternative is one launch of the
single-instance sampler per instance, whose block shape follows each instance's n. Results do not depend on the tile, only speed
does, so the tuner times every legal shape on the batch itself with a short probe
trajectory (CUDA events on the launching stream, after one warm-up launch) and keeps
the fastest. Winners are cached in a JSON file keyed by the batch's shape signature
(K, variant, noise, histogram of n in 64-wide buckets, largest n, replicas), so a
workload is tuned once per machine.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np
import torch

from . import moqaia as M

# (0, 0): one launch of the single-instance sampler per instance (blocks sized per instance)
CANDIDATES = [(1024, 1), (512, 2), (512, 1), (256, 2), (256, 1), (512, 4), (256, 4), (0, 0)]
_CACHE_PATH = os.environ.get("MOQ_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "moqaia_tiles.json"))
_lock = threading.Lock()


def _key(ns, reps, K, variant, noise):
    hist = np.bincount(np.asarray(ns) // 64, minlength=17)[:17].tolist()
    return f"K{K}-v{variant}-noise{int(noise)}-max{max(ns)}-R{int(np.sum(reps))}-h{','.join(map(str, hist))}"


def _load():
    try:
        with open(_CACHE_PATH) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
    tmp = _CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE_PATH)


def legal(max_n):
    return [(bd, spt) for bd, spt in CANDIDATES
            if (bd, spt) == (0, 0) or (bd * spt >= max_n and not (spt >= 2 and bd > 512))]


def tune_batch(batch_handle, ns, reps, K, lam_all, bits_all, params, probe_steps=64, use_cache=True):
    """Pick and set the fastest tile for the batch. Returns (tile, timings in ms)."""
    key = _key(ns, reps, K, params.variant, params.alpha != 0.0)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        bd, spt = cache[key]["tile"]
        M.moq_batch_set_tiles(batch_handle, bd, spt)
        return (bd, spt), cache[key]["ms"]
    probe = M.moq_default_params(variant=params.variant, steps=probe_steps, dt=params.dt, a0=params.a0,
                                 alpha=params.alpha, init_amp=params.init_amp)
    stream = torch.cuda.current_stream()
    timings = {}
    for bd, spt in legal(max(ns)):
        M.moq_batch_set_tiles(batch_handle, bd, spt)
        M.moq_sample_batch(batch_handle, lam_all, probe, 1, 0, bits_all)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for rep in range(3):
            M.moq_sample_batch(batch_handle, lam_all, probe, 1, rep, bits_all)
        e1.record(stream)
        e1.synchronize()
        timings[f"{bd}x{spt}"] = e0.elapsed_time(e1) / 3
    best = min(timings, key=timings.get)
    bd, spt = (int(v) for v in best.split("x"))
    M.moq_batch_set_tiles(batch_handle, bd, spt)
    if use_cache:
        with _lock:
            cache = _load()
            cache[key] = {"tile": [bd, spt], "ms": timings}
            _store(cache)
    return (bd, spt), timings
