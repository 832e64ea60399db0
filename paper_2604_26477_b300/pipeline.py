"""Round driver over the C ABI: owned handles, device buffers and the repeat-until-target
loop of the paper ("Results and discussion": SB is called repeatedly over the weight
vectors until the front is covered; end-to-end time counts model construction,
sampling and filtering).

Everything here is marshalling and orchestration; each computation is one C-ABI call.
"""
from __future__ import annotations

import os
import threading
import time

import numpy as np
import torch

from . import moqaia as M


def source_scalarisation(lam, objective_scale):
    """Weight vectors for an instance whose stored integer weights are objective_scale[k] times
    the source's (an objective scaled to make its weights integers leaves the Pareto set
    unchanged, but the weighted sum J(c) = sum_k c_k J^(k) would over-weight it): column k of
    ``lam`` (torch, R x K) is divided by objective_scale[k] in place, so that the sampler's
    J(c) on the stored weights equals the source's scalarisation. Returns ``lam``."""
    if objective_scale is None:
        return lam
    for k, s in enumerate(np.asarray(objective_scale).tolist()):
        if s != 1:
            lam[:, k] /= float(s)
    return lam


def exhaustive_front(inst: "Instance", chunk_log2: int = 20, stream=None):
    """The exact front of a small instance (n <= 32) by enumeration: every configuration
    with s_0 = +1 (C(s) = C(-s)) in chunks of 2^chunk_log2, evaluated by
    ``moq_evaluate_cuts`` and merged into one archive (``moq_pareto_front``; sample index =
    configuration number). Returns (archive, per-objective minimum cut as a torch tensor)."""
    n, K = inst.n, inst.K
    if n > 32:
        raise ValueError("exhaustive_front enumerates 2^(n-1) configurations: n <= 32")
    total = 1 << (n - 1)
    chunk = min(total, 1 << chunk_log2)
    arch = Archive(n, K, capacity=1 << 19, max_batch=chunk)
    bits = torch.zeros((chunk, inst.W), dtype=torch.int64, device="cuda")
    cuts = torch.zeros((chunk, K), dtype=torch.int64, device="cuda")
    lo = torch.full((K,), 2 ** 62, dtype=torch.int64, device="cuda")
    for c in range(total // chunk):
        # configuration number q sets spins 1..n-1 from its bits (spin 0 stays +1)
        bits[:, 0] = (torch.arange(chunk, device="cuda", dtype=torch.int64) + c * chunk) << 1
        M.moq_evaluate_cuts(inst.handle, bits, chunk, cuts, stream)
        torch.minimum(lo, cuts.min(dim=0).values, out=lo)
        arch.merge(cuts, bits, chunk, c * chunk, stream=stream)
    return arch, lo


class Instance:
    """Device copy of an MO-MaxCut instance (``moq_create_instance``)."""

    def __init__(self, inst, stream=None, layout=None):
        self.src = inst
        self.handle = M.moq_create_instance(inst.n, inst.K, inst.E, inst.ei, inst.ej, inst.w, stream, layout)
        self.info = M.moq_instance_get_info(self.handle)
        self.n, self.K, self.W = inst.n, inst.K, self.info["words"]
        self.ref = np.array(self.info["ref_point"], np.int64)

    def close(self):
        if getattr(self, "handle", None):
            M.moq_destroy_instance(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_build_streams = threading.local()


def create_instances(srcs, stream=None, threads=None, layout_effort=None, layout=None):
    """``Instance`` of every source, built on host threads where some build plans its layout:
    the build's host part (the samplers' shared-memory layout) runs in parallel, and the
    device part of each build is ordered on a stream of its own thread -- on one shared
    stream the builds' pageable copies, kernels and synchronisations queue behind one another.
    Builds with the plain layout alone run one after another on the calling thread. Every
    build has finished on the device when this returns, so the instances are ready for any
    stream, ``stream`` included. ``layout``: as ``moq_create_instance_layout`` (None: from the environment),
    one for all or a list with one per source; ``layout_effort`` = m > 0 is the same as
    ``layout=m`` (the longer layout search, m slot exchanges per spin, for regular graphs)."""
    import concurrent.futures

    srcs = list(srcs)
    if layout_effort is not None:
        layout = int(layout_effort)
    layouts = list(layout) if isinstance(layout, (list, tuple)) else [layout] * len(srcs)
    if len(layouts) != len(srcs):
        raise ValueError("one layout per source")
    if len(srcs) < 2 or all(lay == M.MOQ_LAYOUT_PLAIN for lay in layouts):
        # no host planning to overlap: one thread, where the builds' CUDA calls do not
        # contend for the driver (16 plain builds: 12 ms on 16 threads against 4 ms here)
        return [Instance(s, stream, lay) for s, lay in zip(srcs, layouts)]
    dev = torch.cuda.current_device()

    def build(job):
        s, lay = job
        torch.cuda.set_device(dev)
        if not hasattr(_build_streams, "s"):
            _build_streams.s = torch.cuda.Stream(device=dev)
        return Instance(s, _build_streams.s, lay)

    # the builds start after the work queued so far (on the caller's stream, or anywhere)
    stream.synchronize() if isinstance(stream, torch.cuda.Stream) else torch.cuda.synchronize(dev)
    workers = threads or min(len(srcs), os.cpu_count() or 1, 16)
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(build, zip(srcs, layouts)))


class Archive:
    """Device archive of the non-dominated front (``moq_archive_create``)."""

    def __init__(self, n, K, capacity=1 << 18, max_batch=1 << 16):
        self.n, self.K, self.W = n, K, (n + 63) // 64
        self.capacity, self.max_batch = capacity, max_batch
        self.handle = M.moq_archive_create(n, K, capacity, max_batch)

    def merge(self, cuts, bits, m, index_base, want_size=False, stream=None):
        return M.moq_pareto_front(self.handle, cuts, bits, m, index_base, want_size, stream)

    def size(self, stream=None):
        return M.moq_archive_size(self.handle, stream)

    @staticmethod
    def hypervolume_many(archives, refs, stream=None):
        """Exact hypervolume of every archive's front (one K), two synchronisations in all."""
        if not archives:
            return []
        return M.moq_hypervolume_many([a.handle for a in archives], np.stack([np.asarray(r, np.int64) for r in refs]),
                                      stream)

    def hypervolume(self, ref, stream=None):
        return M.moq_hypervolume(self.handle, ref, stream)

    def copy_out(self, stream=None, reuse=False):
        """The front on the host: (cuts (F,K) int64, bits (F,W) uint64, index (F,) int64). With
        ``reuse`` the copies land in page-locked buffers kept by the archive (one DMA each, no
        staging through pageable memory, grown to the next power of two when the front
        outgrows them); the arrays returned are views of those buffers, overwritten by the
        next ``copy_out(reuse=True)``."""
        if not reuse:
            return M.moq_archive_copy_out(self.handle, self.K, self.W, stream)
        need = 1024
        while True:
            pin = getattr(self, "_pinned", None)
            if pin is None or pin[2].shape[0] < need:
                rows = 1 << max(10, (need - 1).bit_length())
                keep = [torch.empty((rows, self.K), dtype=torch.int64, pin_memory=True),
                        torch.empty((rows, self.W), dtype=torch.int64, pin_memory=True),
                        torch.empty((rows,), dtype=torch.int64, pin_memory=True)]
                self._pinned_keep = keep  # the page-locked tensors behind the numpy views
                pin = self._pinned = (keep[0].numpy(), keep[1].numpy().view(np.uint64), keep[2].numpy())
            F = M.moq_archive_copy_out_into(self.handle, *pin, stream=stream)
            if F <= pin[2].shape[0]:
                return pin[0][:F], pin[1][:F], pin[2][:F]
            need = F

    def reset(self, stream=None):
        M.moq_archive_reset(self.handle, stream)

    def merge_from(self, other: "Archive", stream=None):
        """Merges another archive's front into this one (``moq_archive_merge``)."""
        M.moq_archive_merge(self.handle, other.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            M.moq_archive_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many instances sampled by one persistent launch (``moq_batch_create``)."""

    def __init__(self, instances, replicas, device="cuda"):
        self.instances = instances  # Instance objects, kept alive for the batch's lifetime
        self.replicas = np.asarray(replicas, np.int32)
        self.K = instances[0].K
        self.handle = M.moq_batch_create([h.handle for h in instances], self.replicas)
        self.rep_off, self.word_off = M.moq_batch_layout(self.handle, len(instances))
        self.total_R = int(self.rep_off[-1])
        self.lam = torch.zeros((self.total_R, self.K), dtype=torch.float32, device=device)
        self.bits = torch.zeros(int(self.word_off[-1]), dtype=torch.int64, device=device)
        self.cuts = torch.zeros((self.total_R, self.K), dtype=torch.int64, device=device)
        self.tile = None

    def tune(self, params, probe_steps=64):
        from . import autotune
        self.tile, timings = autotune.tune_batch(self.handle, [h.n for h in self.instances], self.replicas, self.K,
                                                 self.lam, self.bits, params, probe_steps=probe_steps)
        return self.tile, timings

    def set_tiles(self, block_threads, slots_per_thread):
        self.tile = (block_threads, slots_per_thread)
        return M.moq_batch_set_tiles(self.handle, block_threads, slots_per_thread)

    def sample(self, params, seed, round_, stream=None):
        M.moq_sample_batch(self.handle, self.lam, params, seed, round_, self.bits, stream)

    def evaluate_cuts(self, stream=None):
        M.moq_evaluate_cuts_batch(self.handle, self.bits, self.cuts, stream)

    def bits_of(self, b):
        """Instance b's packed samples as a (replicas, W) view."""
        W = self.instances[b].W
        return self.bits[int(self.word_off[b]):int(self.word_off[b + 1])].view(int(self.replicas[b]), W)

    def cuts_of(self, b):
        return self.cuts[int(self.rep_off[b]):int(self.rep_off[b + 1])]

    def close(self):
        if getattr(self, "handle", None):
            M.moq_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RoundBuffers:
    """Device buffers of one sampling round of R replicas."""

    def __init__(self, R, n, K, device="cuda"):
        W = (n + 63) // 64
        self.R = R
        self.bits = torch.zeros((R, W), dtype=torch.int64, device=device)
        self.cuts = torch.zeros((R, K), dtype=torch.int64, device=device)
        self.lam = torch.zeros((R, K), dtype=torch.float32, device=device)


DENSE_FORMS = {"bf16": "moq_sample_dense", "fp8": "moq_sample_dense_fp8", "split": "moq_sample_dense_split"}


def sample_round(inst: Instance, archive: Archive, buf: RoundBuffers, params, seed: int, round_: int,
                 lam=None, index_base=None, stream=None, dense=None, dense_form: str = "bf16"):
    """One pass of the hot path: (lambda) -> sample -> cuts -> Pareto merge. Asynchronous.

    With ``lam=None`` the round draws its own uniform-simplex weight vectors on the GPU.
    With ``dense`` (a ``moq_dense_create`` handle for ``inst``) the round runs the
    tensor-core sampler with the operands ``dense_form`` names ("bf16", "fp8" for dSB with
    E4M3 operands, "split" for the FP32 force from split BF16 operands) and the tensor-core
    cut evaluation.
    """
    R = buf.R
    if lam is None:
        M.moq_lambda_dirichlet(inst.K, R, seed, round_, buf.lam, stream)
        lam = buf.lam
    if dense is not None:
        getattr(M, DENSE_FORMS[dense_form])(dense, lam, R, params, seed, round_, buf.bits, stream)
        M.moq_dense_evaluate_cuts(dense, buf.bits, R, buf.cuts, stream)
    else:
        M.moq_sample(inst.handle, lam, R, params, seed, round_, buf.bits, stream)
        M.moq_evaluate_cuts(inst.handle, buf.bits, R, buf.cuts, stream)
    archive.merge(buf.cuts, buf.bits, R, R * round_ if index_base is None else index_base, stream=stream)


class LearnedProposer:
    """Surrogate-guided weight vectors (the learned proposal; not in the paper).

    Every round's (lambda, cut vector) pairs become training rows of the surrogate MLP
    (inputs: lambda and the instance's 8 graph statistics; targets: cuts normalised by the
    reference point and sum |J^(k)|), which takes ``train_steps`` Adam steps on the newest
    rows. The next round's batch is a fraction ``rho`` of proposed weight vectors -- the
    candidates whose predicted cuts reach furthest beyond the current front -- and the rest
    uniform on the simplex (exploration, and the fallback before any data exists).
    The network trains and predicts on the tensor cores (``engine``; BF16 operands, FP32
    accumulation). Defaults (2048 candidates, 5 Adam steps per round, a quarter of each round
    proposed) were picked on held-out n = 300 instances: 8192 candidates and 20 steps gave about as many
    samples to the target but twice the time per round, and proposing half or three quarters
    of each round needed more samples than a quarter.

    With ``overlap`` the surrogate works on a second stream, off the rounds' critical path:
    once a round is merged (``observe`` with the archive), the next round's weight vectors are
    proposed there while the main stream computes the round's hypervolume, and the Adam steps
    on the round's rows follow while the next round samples. The proposal for round t + 1 thus
    sees the archive after round t and the model trained through round t - 1 (the first model
    is trained before its first proposal). Proposal and training are ordered on that stream, so
    they never run at the same time, and a round starts sampling only once its proposal is done.
    """

    def __init__(self, inst: Instance, R: int, rho=0.25, n_candidates=2048, max_rows=1 << 20, train_steps=5,
                 batch=4096, lr=3e-3, seed=0, device="cuda", overlap=True, engine="tensor_cores"):
        self.inst, self.R, self.K = inst, R, inst.K
        self.rho, self.n_candidates, self.train_steps, self.batch, self.lr, self.seed = \
            rho, n_candidates, train_steps, batch, lr, seed
        self.features = np.asarray(inst.info["features"], np.float32)
        self.din = self.K + self.features.size
        self.offset = np.asarray(inst.info["ref_point"], np.int64)
        self.scale = np.maximum(np.asarray(inst.info["abs_sum"], np.int64), 1)
        self.mlp = M.moq_mlp_create(self.din, self.K, batch, n_candidates, seed + 1)
        M.moq_mlp_set_engine(self.mlp, engine)
        self.max_rows = max_rows
        self.X = torch.zeros((max_rows, self.din), dtype=torch.float32, device=device)
        self.T = torch.zeros((max_rows, self.K), dtype=torch.float32, device=device)
        self.rows = 0
        self.lam = torch.zeros((R, self.K), dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.side = torch.cuda.Stream(device=device) if overlap else None
        self.trained_steps = 0
        self.ready = None  # event: the next round's vectors are proposed (second stream)

    def lambdas(self, round_, arch: Archive):
        if self.ready is not None:  # proposed on the second stream after the last round's merge
            torch.cuda.current_stream().wait_event(self.ready)
            self.ready = None
            return self.lam
        self._propose(round_, arch, stream=None)
        return self.lam

    def _propose(self, round_, arch, stream):
        n_prop = int(self.rho * self.R) if self.rows > 0 else 0
        if n_prop > 0:
            M.moq_lambda_propose(self.mlp, arch.handle, self.features, self.offset, self.scale, self.n_candidates,
                                 self.seed + 7, round_, self.lam, n_prop, stream)
        if n_prop < self.R:
            M.moq_lambda_dirichlet(self.K, self.R - n_prop, self.seed, round_, self.lam[n_prop:], stream)

    def observe(self, lam, cuts, m, arch: Archive = None, round_: int = None):
        """Adds the round's (lambda, cut) rows; with ``overlap`` and the merged ``arch`` of round
        ``round_``, also queues the next round's proposal and the Adam steps on the second stream."""
        at = self.rows % self.max_rows
        m = min(m, self.max_rows - at)
        M.moq_mlp_make_rows(self.K, self.features, lam, cuts, m, self.offset, self.scale, self.X[at:], self.T[at:])
        self.rows += m
        filled = min(self.rows, self.max_rows)
        newest = (self.rows - 1) % self.max_rows
        if self.side is None or arch is None:
            self._train(newest, filled, stream=None)
            return
        self.side.wait_stream(torch.cuda.current_stream())  # rows, merge and lambda reads are done
        if self.trained_steps == 0:
            self._train(newest, filled, stream=self.side)  # the first model before its first proposal
            self._propose(round_ + 1, arch, stream=self.side)
            self.ready = self.side.record_event()
            return
        self._propose(round_ + 1, arch, stream=self.side)
        self.ready = self.side.record_event()
        self._train(newest, filled, stream=self.side)  # runs while the next round samples

    def _train(self, newest, filled, stream):
        for s in range(self.train_steps):  # batches walk back from the newest rows
            end = newest + 1 - s * self.batch
            while end <= 0:
                end += filled
            start = max(0, end - self.batch)
            M.moq_mlp_train_step(self.mlp, self.X[start:end], self.T[start:end], end - start, self.lr, self.loss, stream)
        self.trained_steps += self.train_steps

    def close(self):
        if getattr(self, "mlp", None):
            if getattr(self, "side", None) is not None:
                self.side.synchronize()
            M.moq_mlp_destroy(self.mlp)
            self.mlp = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def round_layout(params, n=None):
    """The samplers' memory layout the round drivers build with by default, by the sampler's
    precision and the graph size.

    The bank-conflict planner is host work inside every time-to-target clock (0.2 ms at
    n = 42, 3-12 ms at n = 1024 depending on the host; 16 builds of n = 68..932 took 24-33 ms
    on 16 threads against 2.4-3.9 ms for plain builds on one thread). The float16 samplers
    gather 4-byte half2 words and gain little from it, the FP32 pair forms gather 8-byte
    words and gain 4-16 % per launch. Measured on 16 random 3-regular instances (1024
    replicas per round, 8 seeds): float16 NI-dSB (T = 3000) batched reached 99 % of the plain
    sampler's hypervolume in 60 ms with the plain layout against 82 ms with the planner
    (99.9 %: 277 against 300 ms); plain FP32 dSB one instance at a time took 71 against 83 ms
    at 99 % (6 rounds) but 876 against 716 ms at 99.9 % (60 rounds), so for FP32 the planner
    pays back only over long jobs, and callers that know theirs is short pass
    ``layout=M.MOQ_LAYOUT_PLAIN``. On small graphs the planner gains about 1 % (n = 42: 44
    against 39 8-byte passes per gather step) for 0.2 ms or more of a sub-millisecond clock.
    So float16 rounds and graphs of up to 128 spins build with the plain layout, larger FP32
    ones with the planner.
    """
    fp16 = getattr(params, "precision", M.MOQ_PREC_FP32) == M.MOQ_PREC_FP16
    return M.MOQ_LAYOUT_PLAIN if fp16 or (n is not None and n <= 128) else M.MOQ_LAYOUT_DEFAULT


def time_to_target(src, target_hv: int, params, R: int, seed: int = 0, max_rounds: int = 1000,
                   capacity=1 << 18, learned: bool = False, proposer_kwargs=None, dense: bool = False,
                   dense_form: str = "bf16", layout=None):
    """Repeat sampling rounds until the archive's hypervolume reaches ``target_hv``.

    The clock covers instance construction (with the samplers' memory ``layout``; None:
    ``round_layout(params, n)``), every round (weight vectors, sampling, cuts, Pareto merge, the
    surrogate's training and proposal when ``learned``) and the hypervolume checks (one
    synchronisation per round).
    Returns dict(seconds, rounds, samples, hv, front, reached, trace) with trace a list of
    (samples, hv) after each round.
    """
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    inst = Instance(src, layout=round_layout(params, src.n) if layout is None else layout)
    arch = Archive(src.n, src.K, capacity=capacity, max_batch=R)
    buf = RoundBuffers(R, src.n, src.K)
    dh = M.moq_dense_create(inst.handle, R) if dense else None
    prop = LearnedProposer(inst, R, seed=seed, **(proposer_kwargs or {})) if learned else None
    hv, rounds, trace = 0, 0, []
    while rounds < max_rounds:
        lam = prop.lambdas(rounds, arch) if prop else None
        sample_round(inst, arch, buf, params, seed, rounds, lam=lam, dense=dh, dense_form=dense_form)
        if prop:
            prop.observe(lam, buf.cuts, R, arch, rounds)
        rounds += 1
        hv = arch.hypervolume(inst.ref)
        trace.append((rounds * R, hv))
        if hv >= target_hv:
            break
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    front = arch.size()
    if prop:
        prop.close()
    if dh is not None:
        M.moq_dense_status(dh)
        M.moq_dense_destroy(dh)
    arch.close()
    inst.close()
    return {"seconds": secs, "rounds": rounds, "samples": rounds * R, "hv": hv, "front": front,
            "reached": hv >= target_hv, "trace": trace}


class BatchLearnedProposer:
    """One surrogate for every instance of a batch (the learned proposal; not in the paper).

    The MLP's inputs carry each instance's eight graph statistics, so one network serves the
    whole batch: every round's (lambda, cut vector) rows of each active instance are added
    (cuts normalised by that instance's reference point and sum |J^(k)|), the network takes
    ``train_steps`` Adam steps on the newest rows, and for each active instance a fraction
    ``rho`` of its next weight vectors are the candidates predicted to reach furthest beyond
    that instance's front; the rest stay uniform on the simplex. As in LearnedProposer, the
    proposal for round t + 1 (after round t's merges) and the training run on a second stream
    while the main stream checks hypervolumes and samples.
    """

    def __init__(self, instances, R, rho=0.25, n_candidates=2048, max_rows=1 << 20, train_steps=5, batch=4096,
                 lr=3e-3, seed=0, device="cuda", engine="tensor_cores"):
        self.K, self.R = instances[0].K, R
        self.rho, self.n_candidates, self.train_steps, self.batch, self.lr, self.seed = \
            rho, n_candidates, train_steps, batch, lr, seed
        self.n_prop = int(rho * R)
        self.feats = [np.asarray(h.info["features"], np.float32) for h in instances]
        self.offs = [np.asarray(h.info["ref_point"], np.int64) for h in instances]
        self.scales = [np.maximum(np.asarray(h.info["abs_sum"], np.int64), 1) for h in instances]
        self.din = self.K + self.feats[0].size
        self.mlp = M.moq_mlp_create(self.din, self.K, batch, n_candidates, seed + 1)
        M.moq_mlp_set_engine(self.mlp, engine)
        self.max_rows = max_rows
        self.X = torch.zeros((max_rows, self.din), dtype=torch.float32, device=device)
        self.T = torch.zeros((max_rows, self.K), dtype=torch.float32, device=device)
        self.prop = torch.zeros((len(instances), max(self.n_prop, 1), self.K), dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.rows = 0
        self.side = torch.cuda.Stream(device=device)
        self.ready = None
        self.proposed = []
        self.trained = False

    def apply(self, lam_all, rep_off):
        """Overwrites the first rho * R weight vectors of every instance proposed for this round
        (main stream, after the round's uniform vectors were drawn)."""
        if self.ready is None:
            return
        torch.cuda.current_stream().wait_event(self.ready)
        for b in self.proposed:
            r0 = int(rep_off[b])
            lam_all[r0:r0 + self.n_prop].copy_(self.prop[b, :self.n_prop])
        self.ready = None

    def observe(self, lam_all, cuts_all, rep_off, active, archives, round_):
        """Adds the round's rows of the active instances, then queues on the second stream the
        next round's proposals for them and the Adam steps."""
        for b in active:
            r0 = int(rep_off[b])
            at = self.rows % self.max_rows
            m = min(self.R, self.max_rows - at)
            M.moq_mlp_make_rows(self.K, self.feats[b], lam_all[r0:r0 + m], cuts_all[r0:r0 + m], m, self.offs[b],
                                self.scales[b], self.X[at:], self.T[at:])
            self.rows += m
        filled = min(self.rows, self.max_rows)
        newest = (self.rows - 1) % self.max_rows
        self.side.wait_stream(torch.cuda.current_stream())
        first = not self.trained
        if first:
            self._train(newest, filled)  # the first model before its first proposal
            self.trained = True
        if self.n_prop > 0:
            for b in active:
                M.moq_lambda_propose(self.mlp, archives[b].handle, self.feats[b], self.offs[b], self.scales[b],
                                     self.n_candidates, self.seed + 7 + b, round_ + 1, self.prop[b], self.n_prop, self.side)
        self.proposed = list(active)
        self.ready = self.side.record_event()
        if not first:
            self._train(newest, filled)  # runs while the next round samples

    def _train(self, newest, filled):
        for s in range(self.train_steps):
            end = newest + 1 - s * self.batch
            while end <= 0:
                end += filled
            start = max(0, end - self.batch)
            M.moq_mlp_train_step(self.mlp, self.X[start:end], self.T[start:end], end - start, self.lr, self.loss, self.side)

    def close(self):
        if getattr(self, "mlp", None):
            self.side.synchronize()
            M.moq_mlp_destroy(self.mlp)
            self.mlp = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def time_to_target_batch(srcs, targets, params, R: int, seed: int = 0, max_rounds: int = 256, batched: bool = True,
                         learned: bool = False, tiles=(0, 0), capacity=1 << 18, proposer_kwargs=None,
                         layout=None):
    """Rounds over a set of instances until every instance's archive reaches its target
    hypervolume (the job is done when the whole set is).

    ``batched``: each round is one ``moq_sample_batch`` call and one batched cut evaluation
    over the instances still short of their target (``moq_batch_set_replicas`` drops the
    others), tile shape ``tiles`` ((0, 0): per-instance launches over internal streams);
    else one ``sample_round`` per such instance in turn. Every instance has its own archive,
    and after each round every active instance's hypervolume is checked. ``learned`` adds the
    batch surrogate (``BatchLearnedProposer``). The clock covers instance construction (on
    host threads, with the samplers' memory ``layout``; None: ``round_layout(params, n)``),
    every round and the checks (the active instances' hypervolumes with one
    ``moq_hypervolume_many`` call per round, two synchronisations).
    Returns dict(seconds, rounds, samples, reached, rounds_per_instance).
    """
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = len(srcs)
    insts = create_instances(srcs, layout=[round_layout(params, s.n) for s in srcs] if layout is None else layout)
    archs = [Archive(s.n, s.K, capacity=capacity, max_batch=R) for s in srcs]
    K = insts[0].K
    active = list(range(B))
    done_at = [0] * B
    rounds, samples = 0, 0
    batch = prop = None
    if batched:
        batch = Batch(insts, [R] * B)
        batch.set_tiles(*tiles)
        prop = BatchLearnedProposer(insts, R, seed=seed, **(proposer_kwargs or {})) if learned else None
    else:
        bufs = {}
    while active and rounds < max_rounds:
        if batched:
            M.moq_lambda_dirichlet(K, batch.total_R, seed, rounds, batch.lam)
            if prop:
                prop.apply(batch.lam, batch.rep_off)
            batch.sample(params, seed, rounds)
            batch.evaluate_cuts()
            for b in active:
                archs[b].merge(batch.cuts_of(b), batch.bits_of(b), R, R * rounds)
            if prop:
                prop.observe(batch.lam, batch.cuts, batch.rep_off, active, archs, rounds)
        else:
            for b in active:
                if srcs[b].n not in bufs:
                    bufs[srcs[b].n] = RoundBuffers(R, srcs[b].n, K)
                sample_round(insts[b], archs[b], bufs[srcs[b].n], params, seed, rounds)
        samples += R * len(active)
        rounds += 1
        still = []
        hvs = Archive.hypervolume_many([archs[b] for b in active], [insts[b].ref for b in active])
        for b, hv in zip(active, hvs):
            if hv >= targets[b]:
                done_at[b] = rounds
            else:
                still.append(b)
        if batched and len(still) < len(active) and still:
            reps = np.zeros(B, np.int32)
            reps[still] = R
            M.moq_batch_set_replicas(batch.handle, reps)
        active = still
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    if prop:
        prop.close()
    if batch is not None:
        batch.close()
    for a in archs:
        a.close()
    for h in insts:
        h.close()
    return {"seconds": secs, "rounds": rounds, "samples": samples, "reached": not active,
            "rounds_per_instance": done_at}
