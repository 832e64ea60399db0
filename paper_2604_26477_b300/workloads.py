"""Seeded synthetic MO-MaxCut instances and weight-vector batches.

This module is the only code shared by the CPU oracle and the CUDA path. It draws
inputs; it computes nothing the method computes (no cuts, no dynamics, no
dominance, no hypervolume). Every generator is a pure function of its seed.

Graph families (the paper's public instances are not available, so these stand in
for them with the same shapes):

* ``heavy_hex_like`` -- 42 nodes, 50 edges, maximum degree 3: degree-3 sites joined
  through degree-2 bridges, the shape of the 42-qubit heavy-hex MO-MaxCut
  instances used in the paper's "Results and discussion" section.
* ``random_regular`` -- random d-regular graphs (pairing model with rejection),
  the uneven-size batch workload.
* ``complete_graph`` -- K_n with Gaussian integer weights, the dense workload.
* ``app_e_correlated`` -- the correlated three-objective family of Appendix E.

Weights are integers (int32), one row per objective: ``w[k, e]`` is J^(k) of edge
``e = (ei[e], ej[e])`` with ``ei[e] < ej[e]``; edges are sorted by ``(i, j)``.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Instance:
    """An MO-MaxCut instance: graph G=(V,E) with K integer edge-weight sets."""

    n: int
    ei: np.ndarray  # (E,) int32, ei < ej
    ej: np.ndarray  # (E,) int32
    w: np.ndarray  # (K, E) int32, row k = objective k
    name: str = ""
    # per objective, the factor by which the stored integer weights exceed the source's
    # (None: all 1); a weighted sum over the source's weights takes lambda_k / scale_k
    objective_scale: np.ndarray | None = None

    @property
    def K(self) -> int:
        return int(self.w.shape[0])

    @property
    def E(self) -> int:
        return int(self.ei.shape[0])


def _sorted_edges(edges, n):
    arr = np.array(sorted((min(a, b), max(a, b)) for a, b in edges), dtype=np.int64)
    if arr.size == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    assert np.all(arr[:, 0] < arr[:, 1]) and np.all(arr[:, 1] < n)
    assert len({(int(a), int(b)) for a, b in arr}) == len(arr), "duplicate edge"
    return arr[:, 0].astype(np.int32), arr[:, 1].astype(np.int32)


def pairing_regular_edges(n: int, d: int, rng: np.random.Generator, max_tries: int = 10000):
    """Edges of a uniformly random simple d-regular graph on n nodes (pairing model).

    n*d must be even. Stubs are matched by a random permutation; matchings with a
    loop or a repeated edge are rejected and redrawn.
    """
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    stubs = np.repeat(np.arange(n), d)
    for _ in range(max_tries):
        p = rng.permutation(stubs).reshape(-1, 2)
        a, b = np.minimum(p[:, 0], p[:, 1]), np.maximum(p[:, 0], p[:, 1])
        if np.any(a == b):
            continue
        key = a.astype(np.int64) * n + b
        if np.unique(key).size != key.size:
            continue
        return list(zip(a.tolist(), b.tolist()))
    raise RuntimeError("pairing model failed to produce a simple graph")


def nonzero_uniform_weights(K: int, E: int, lo: int, hi: int, rng: np.random.Generator):
    """i.i.d. integer weights uniform on {lo..hi} minus {0}, shape (K, E)."""
    vals = np.array([v for v in range(lo, hi + 1) if v != 0], dtype=np.int32)
    return vals[rng.integers(0, vals.size, size=(K, E))].astype(np.int32)


def heavy_hex_like(seed: int, K: int = 3, wmax: int = 10) -> Instance:
    """42 nodes / 50 edges / max degree 3, heavy-hex-like, weights in {-wmax..wmax}\\{0}.

    Recipe: a random 3-regular graph on 16 hub nodes (24 edges); every edge is
    subdivided once by a degree-2 bridge node (40 nodes, 48 edges); two random edges
    are subdivided once more (42 nodes, 50 edges). Labels are then shuffled.
    """
    rng = np.random.default_rng(seed)
    hubs = 16
    base = pairing_regular_edges(hubs, 3, rng)
    edges = []
    nxt = hubs
    for a, b in base:
        edges += [(a, nxt), (nxt, b)]
        nxt += 1
    for _ in range(2):
        idx = int(rng.integers(0, len(edges)))
        a, b = edges.pop(idx)
        edges += [(a, nxt), (nxt, b)]
        nxt += 1
    n = nxt
    perm = rng.permutation(n)
    edges = [(int(perm[a]), int(perm[b])) for a, b in edges]
    ei, ej = _sorted_edges(edges, n)
    w = nonzero_uniform_weights(K, ei.size, -wmax, wmax, rng)
    return Instance(n, ei, ej, w, name=f"heavyhex42_K{K}_s{seed}")


def random_regular(n: int, seed: int, K: int = 3, d: int = 3, wmax: int = 100) -> Instance:
    """Random d-regular graph on n nodes, weights in {-wmax..wmax}\\{0}."""
    rng = np.random.default_rng(seed)
    ei, ej = _sorted_edges(pairing_regular_edges(n, d, rng), n)
    w = nonzero_uniform_weights(K, ei.size, -wmax, wmax, rng)
    return Instance(n, ei, ej, w, name=f"reg{d}_n{n}_K{K}_s{seed}")


def uneven_regular_batch(count: int, seed: int, nmin: int = 42, nmax: int = 1024, K: int = 3, wmax: int = 100):
    """``count`` random 3-regular instances with n ~ U[nmin, nmax] rounded up to even."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ns = ns + (ns % 2)
    return [random_regular(int(nn), seed * 100003 + i, K=K, wmax=wmax) for i, nn in enumerate(ns)]


def complete_graph(n: int, seed: int, K: int = 3, scale: float = 1000.0) -> Instance:
    """K_n with weights round(scale * N(0,1)) i.i.d. per edge and objective."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    w = np.rint(scale * rng.standard_normal((K, iu.size))).astype(np.int32)
    return Instance(n, iu.astype(np.int32), ju.astype(np.int32), w, name=f"K{n}_K{K}_s{seed}")


def random_graph(n: int, p: float, seed: int, K: int = 3, wmax: int = 10) -> Instance:
    """Erdos-Renyi G(n, p) with weights in {-wmax..wmax}\\{0} (small test instances)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    ei, ej = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    w = nonzero_uniform_weights(K, ei.size, -wmax, wmax, rng)
    return Instance(n, ei, ej, w, name=f"gnp{n}_{p}_K{K}_s{seed}")


def app_e_correlated(n: int, density: float, seed: int) -> Instance:
    """Appendix E family: A, B ~ U{-25..25}; J1 = A + B, J2 = 0.2 A - 5 B, J3 ~ U{-25..25}.

    J2 is multiplied by 5 (J2 = A - 25 B) so that every weight is an integer;
    scaling one objective leaves the Pareto set unchanged. A random mask keeps each
    edge with probability ``density``.
    """
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    A = rng.integers(-25, 26, size=iu.size)
    B = rng.integers(-25, 26, size=iu.size)
    C = rng.integers(-25, 26, size=iu.size)
    keep = rng.random(iu.size) < density
    w = np.stack([A + B, A - 25 * B, C])[:, keep].astype(np.int32)
    return Instance(n, iu[keep].astype(np.int32), ju[keep].astype(np.int32), w, name=f"appE_n{n}_d{density}_s{seed}",
                    objective_scale=np.array([1, 5, 1], np.int64))


def dirichlet_lambdas(R: int, K: int, seed: int) -> np.ndarray:
    """R weight vectors drawn uniformly on the simplex (Dirichlet(1,...,1)), float32 (R, K)."""
    rng = np.random.default_rng(seed)
    return rng.dirichlet(np.ones(K), size=R).astype(np.float32)


def random_sign_bits(M: int, n: int, seed: int) -> np.ndarray:
    """M uniformly random spin configurations packed as (M, ceil(n/64)) uint64.

    Bit (i mod 64) of word i // 64 is 1 when s_i = -1. Bits at positions >= n are 0.
    """
    rng = np.random.default_rng(seed)
    W = (n + 63) // 64
    out = rng.integers(0, 2**63, size=(M, W), dtype=np.int64).astype(np.uint64)
    out ^= rng.integers(0, 2, size=(M, W), dtype=np.int64).astype(np.uint64) << np.uint64(63)
    tail = n - 64 * (W - 1)
    if tail < 64:
        out[:, W - 1] &= np.uint64((1 << tail) - 1)
    return out


def signs_to_bits(s: np.ndarray) -> np.ndarray:
    """(M, n) array of +-1 spins -> (M, ceil(n/64)) uint64 with bit=1 for s=-1."""
    s = np.atleast_2d(s)
    M, n = s.shape
    W = (n + 63) // 64
    out = np.zeros((M, W), dtype=np.uint64)
    neg = (s < 0)
    for i in range(n):
        out[:, i // 64] |= neg[:, i].astype(np.uint64) << np.uint64(i % 64)
    return out


def bits_to_signs(bits: np.ndarray, n: int) -> np.ndarray:
    """Inverse of ``signs_to_bits``: (M, W) uint64 -> (M, n) int8 of +-1."""
    bits = np.atleast_2d(bits)
    out = np.empty((bits.shape[0], n), dtype=np.int8)
    for i in range(n):
        b = (bits[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)
        out[:, i] = np.where(b == 1, -1, 1)
    return out
