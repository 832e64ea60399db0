"""The paper's float16 form of the sparse sampler (p->precision = MOQ_PREC_FP16) through the C
ABI: the one-step force against the FP64 oracle within the FP16 bound, invariants, shards and
batches bit for bit, and the distribution of final hypervolumes against the FP32 form and the
oracle over 32 seeds (trajectories are chaotic)."""
import numpy as np
import pytest
import torch
from scipy import stats

from paper_2604_26477_b300 import workloads as wl

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11  # unit roundoff of FP16 (round to nearest)


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


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _circulant(n, hops, seed, K, wmax=10):
    """Spin i joined to i +- h (mod n) for h in hops: every degree is 2 len(hops)."""
    rng = np.random.default_rng(seed)
    pairs = sorted({(min(i, (i + h) % n), max(i, (i + h) % n)) for i in range(n) for h in hops})
    ei = np.array([a for a, _ in pairs], np.int32)
    ej = np.array([b for _, b in pairs], np.int32)
    w = rng.integers(1, wmax + 1, size=(K, len(pairs))) * rng.choice([-1, 1], size=(K, len(pairs)))
    return wl.Instance(n, ei, ej, w.astype(np.int32))


INSTANCES = {
    "heavyhex_K3": lambda: wl.heavy_hex_like(1000, K=3),
    "heavyhex_K4": lambda: wl.heavy_hex_like(1001, K=4),
    "reg3_n1024_K3": lambda: wl.random_regular(1024, 8, K=3),
    "reg4_n300_K3": lambda: wl.random_regular(300, 9, K=3, d=4),
    "circ8_n64_K2": lambda: _circulant(64, (1, 2, 3, 4), 4, K=2),
}


def _abs_terms_and_degree(src, lam, phi, c0):
    """c0 sum_j |J(c)_ij phi_j| per (replica, spin) and the degree of each spin."""
    Jc = lam @ src.w.astype(np.float64)  # R x E
    out = np.zeros(phi.shape)
    np.add.at(out.T, src.ei, (np.abs(Jc * phi[:, src.ej])).T)
    np.add.at(out.T, src.ej, (np.abs(Jc * phi[:, src.ei])).T)
    deg = np.bincount(np.concatenate([src.ei, src.ej]), minlength=src.n)
    return out * c0[:, None], deg


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("variant", ["dsb", "bsb"])
def test_fp16_force_within_its_bound(M, P, oracle, name, variant):
    # one step from x0 exact in FP16, y0 = 0, a_m = a0 (no linear term), alpha = 0, dt = 1/2:
    # y after the step is dt * force exactly (a power-of-two scaling), so y_out / dt is the
    # FP16 force. Bound: each coupling rounded once to FP16 and one rounding per multiply-add
    # of the force sum, |f - f64| <= (deg + 2) 2^-11 c0 sum_j |J(c)_ij phi_j| per spin.
    src = INSTANCES[name]()
    inst = P.Instance(src)
    R, dt = 67, 0.5
    lam = wl.dirichlet_lambdas(R, src.K, 3)
    x0 = np.random.default_rng(1).uniform(-0.5, 0.5, (R, src.n)).astype(np.float16).astype(np.float32)
    y_out = torch.zeros((R, src.n), device="cuda")
    x_out = torch.zeros_like(y_out)
    p = M.moq_default_params(variant=variant, steps=1, dt=dt, a0=1.0, alpha=0.0, precision="fp16",
                             schedule=torch.ones(1, device="cuda"), x_init=_dev(x0),
                             y_init=torch.zeros((R, src.n), device="cuda"), x_out=x_out, y_out=y_out)
    M.moq_sample(inst.handle, _dev(lam), R, p, 0, 0, torch.zeros((R, inst.W), dtype=torch.int64, device="cuda"))
    ref = oracle.sb(src, lam.astype(np.float64), variant=variant, steps=1, dt=dt, a0=1.0, alpha=0.0,
                    schedule=[1.0], x_init=x0.astype(np.float64), y_init=np.zeros((R, src.n)))
    f16 = y_out.cpu().numpy().astype(np.float64) / dt
    f64 = ref["y"] / dt
    phi = np.where(x0 >= 0, 1.0, -1.0) if variant == "dsb" else x0.astype(np.float64)
    scale, deg = _abs_terms_and_degree(src, lam, phi, ref["c0"])
    bound = (deg[None, :] + 2) * U16 * scale
    err = np.abs(f16 - f64)
    # spins the wall reached (|x| near 1 after the step: y is reset) carry no force to compare
    free = (np.abs(ref["x"]) < 0.999) & (np.abs(x_out.cpu().numpy()) < 0.999)
    assert free.mean() > 0.95
    assert np.all(err[free] <= bound[free] + 1e-30), float((err[free] / np.maximum(scale[free], 1e-30)).max())
    assert (err[free] > 0).any()  # the FP16 arithmetic really rounds (not the FP32 path)


@pytest.mark.parametrize("variant", ["dsb", "bsb"])
def test_fp16_invariants_determinism_and_shards(M, P, variant):
    from paper_2604_26477_b300.shard import replica_shard
    src = wl.random_regular(150, 7, K=3)
    inst = P.Instance(src)
    R = 301
    lam = _dev(wl.dirichlet_lambdas(R, 3, 9))
    xo = torch.zeros((R, src.n), device="cuda")
    yo = torch.zeros((R, src.n), device="cuda")
    p = M.moq_default_params(variant=variant, steps=503, dt=0.5, alpha=0.15, precision="fp16", x_out=xo, y_out=yo)
    b1 = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
    b2 = torch.zeros_like(b1)
    M.moq_sample(inst.handle, lam, R, p, 77, 1, b1)
    x, y = xo.cpu().numpy(), yo.cpu().numpy()
    # |x| <= 1 always; unlike FP32, x also lands on exactly +-1 by rounding (FP16 spacing 2^-11
    # below 1) without crossing the strict wall |x| > 1, so y = 0 only where the wall acted
    assert np.all(np.abs(x) <= 1.0)
    assert np.all(x.astype(np.float16).astype(np.float32) == x)  # the state is FP16
    assert np.all(y.astype(np.float16).astype(np.float32) == y)
    assert np.array_equal(wl.bits_to_signs(b1.cpu().numpy().view(np.uint64), src.n), np.where(x >= 0, 1, -1))
    M.moq_sample(inst.handle, lam, R, p, 77, 1, b2)
    assert torch.equal(b1, b2)
    # shards with replica offsets reproduce the single call bit for bit
    for q in range(3):
        first, count = replica_shard(R, q, 3)
        part = torch.zeros((count, inst.W), dtype=torch.int64, device="cuda")
        pq = M.moq_default_params(variant=variant, steps=503, dt=0.5, alpha=0.15, precision="fp16", replica_offset=first)
        M.moq_sample(inst.handle, lam[first:first + count].contiguous(), count, pq, 77, 1, part)
        assert torch.equal(part, b1[first:first + count])


def test_fp16_final_hv_distribution(M, P, oracle):
    # the FP16 form's final fronts are distributed like the FP32 form's and the FP64 oracle's
    src = wl.heavy_hex_like(1000, K=3)
    inst = P.Instance(src)
    R, T = 128, 300
    lam = wl.dirichlet_lambdas(R, 3, 77)
    lam_d = _dev(lam)
    bits = torch.zeros((R, 1), dtype=torch.int64, device="cuda")
    hv = {"fp16": [], "fp32": [], "oracle": []}
    for seed in range(32):
        for prec in ("fp16", "fp32"):
            M.moq_sample(inst.handle, lam_d, R, M.moq_default_params(steps=T, dt=0.5, alpha=0.15, precision=prec), seed, 0, bits)
            c = oracle.cuts(src, bits.cpu().numpy().view(np.uint64))
            hv[prec].append(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref))
        o = oracle.sb(src, lam.astype(np.float64), steps=T, dt=0.5, alpha=0.15, seed=1000 + seed)
        c = oracle.cuts(src, o["bits"])
        hv["oracle"].append(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref))
    for other in ("fp32", "oracle"):
        p = stats.mannwhitneyu(hv["fp16"], hv[other]).pvalue
        assert p > 0.01, (other, p, np.median(hv["fp16"]), np.median(hv[other]))
        assert abs(np.median(hv["fp16"]) / np.median(hv[other]) - 1) < 0.02


def test_fp16_batch_equals_single_calls(M, P):
    insts = [P.Instance(wl.random_regular(n, 40 + q, K=3)) for q, n in enumerate((42, 300, 130, 1024))]
    reps = [96, 33, 64, 17]
    batch = P.Batch(insts, reps)
    M.moq_batch_set_tiles(batch.handle, 0, 0)  # per-instance launches
    lam = _dev(wl.dirichlet_lambdas(sum(reps), 3, 5))
    p = M.moq_default_params(steps=211, dt=0.5, alpha=0.1, precision="fp16")
    bits = batch.bits
    M.moq_sample_batch(batch.handle, lam, p, 3, 2, bits)
    for q, inst in enumerate(insts):
        r0, w0 = int(batch.rep_off[q]), int(batch.word_off[q])
        one = torch.zeros((reps[q], inst.W), dtype=torch.int64, device="cuda")
        pq = M.moq_default_params(steps=211, dt=0.5, alpha=0.1, precision="fp16", replica_offset=r0)
        M.moq_sample(inst.handle, lam[r0:r0 + reps[q]].contiguous(), reps[q], pq, 3, 2, one)
        assert torch.equal(one.reshape(-1), bits[w0:w0 + reps[q] * inst.W])
    M.moq_batch_set_tiles(batch.handle, 1024, 1)
    with pytest.raises(M.MoqError) as e:
        M.moq_sample_batch(batch.handle, lam, p, 3, 2, bits)
    assert e.value.code == M.MOQ_ERR_UNSUPPORTED


def test_fp16_rejects_what_it_does_not_run(M, P):
    inst = P.Instance(_circulant(64, (1, 2, 3, 4, 5, 6), 5, K=2))  # degree 12: the FP32 form runs it, FP16 does not
    lam = _dev(wl.dirichlet_lambdas(8, 2, 1))
    bits = torch.zeros((8, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(M.MoqError) as e:
        M.moq_sample(inst.handle, lam, 8, M.moq_default_params(precision="fp16"), 0, 0, bits)
    assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    with pytest.raises(M.MoqError) as e:
        M.moq_sample(inst.handle, lam, 8, M.moq_default_params(precision=7), 0, 0, bits)
    assert e.value.code == M.MOQ_ERR_ARG


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
@pytest.mark.parametrize("n,R", [(600, 4096), (520, 301), (300, 2000)])
def test_register_capped_build_gives_the_same_bits(M, P, monkeypatch, prec, n, R):
    # blocks of up to 640 threads may run a register-capped build of the pair / FP16 kernels (two
    # resident blocks per SM): the same arithmetic, so the same samples and final state
    src = wl.random_regular(n, 41, K=3)
    inst = P.Instance(src)
    lam = _dev(wl.dirichlet_lambdas(R, 3, 4))
    out = {}
    for cap in ("0", "1"):
        monkeypatch.setenv("MOQ_SB_CAP", cap)
        monkeypatch.setenv("MOQ_SB_PAIR", "1")
        xo = torch.zeros((R, n), device="cuda")
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(steps=203, dt=0.5, alpha=0.1, precision=prec, x_out=xo)
        M.moq_sample(inst.handle, lam, R, p, 6, 1, bits)
        out[cap] = (bits.cpu(), xo.cpu())
    assert torch.equal(out["0"][0], out["1"][0]) and torch.equal(out["0"][1], out["1"][1])


@pytest.mark.parametrize("variant,alpha", [("dsb", 0.1), ("bsb", 0.0), ("bsb", 0.2)])
@pytest.mark.parametrize("n,d,R", [(700, 3, 1021), (1024, 3, 600), (300, 4, 999), (42, 3, 517)])
def test_fp16_quads_give_the_same_bits_as_pairs(M, P, monkeypatch, variant, alpha, n, d, R):
    # four replicas per thread (two FP16 pairs, taken by default for large graphs; MOQ_SB_QUAD
    # forces either form) run each replica's arithmetic and noise counters of the pair form:
    # same samples and final state, ragged replica counts and step counts included
    src = wl.heavy_hex_like(1000, K=3) if n == 42 else wl.random_regular(n, 43, K=3, d=d)
    inst = P.Instance(src)
    lam = _dev(wl.dirichlet_lambdas(R, 3, 5))
    out = {}
    for quad in ("0", "1"):
        monkeypatch.setenv("MOQ_SB_QUAD", quad)
        xo = torch.zeros((R, n), device="cuda")
        yo = torch.zeros((R, n), device="cuda")
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(variant=variant, steps=203, dt=0.5, alpha=alpha, precision="fp16", x_out=xo, y_out=yo)
        M.moq_sample(inst.handle, lam, R, p, 7, 2, bits)
        out[quad] = (bits.cpu(), xo.cpu(), yo.cpu())
    for a, b in zip(out["0"], out["1"]):
        assert torch.equal(a, b)


def test_fp16_quads_from_a_given_state(M, P, monkeypatch):
    # a given initial (x, y) reaches the same place in both forms
    n, R = 800, 403
    src = wl.random_regular(n, 44, K=3)
    inst = P.Instance(src)
    lam = _dev(wl.dirichlet_lambdas(R, 3, 6))
    g = torch.Generator().manual_seed(3)
    x0 = (torch.rand((R, n), generator=g) - 0.5).cuda()
    y0 = (0.2 * torch.randn((R, n), generator=g)).cuda()
    out = {}
    for quad in ("0", "1"):
        monkeypatch.setenv("MOQ_SB_QUAD", quad)
        xo = torch.zeros((R, n), device="cuda")
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        p = M.moq_default_params(steps=150, dt=0.5, alpha=0.1, precision="fp16", x_init=x0, y_init=y0, x_out=xo)
        M.moq_sample(inst.handle, lam, R, p, 8, 0, bits)
        out[quad] = (bits.cpu(), xo.cpu())
    assert torch.equal(out["0"][0], out["1"][0]) and torch.equal(out["0"][1], out["1"][1])
