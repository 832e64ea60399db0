"""The tensor-core (tcgen05) dense sampler against the CPU oracle.

dSB with integer couplings |J| <= 256 is exact in BF16 and phi = +-1 is exact, so the
per-objective products are exact and the force must match the FP64 oracle within the
FP32 normwise bound (1e-5). bSB rounds x to BF16 for the products: the stated bound is
|f - f64| <= 4e-3 * c0 * sum_j |J(c)_ij x_j| (BF16 has a 2^-9 relative rounding).
"""
import numpy as np
import pytest
import torch
from scipy import stats

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


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _abs_force_scale(src, lam, phi, c0):
    Jc = lam.astype(np.float64) @ src.w.astype(np.float64)
    out = np.zeros(phi.shape)
    np.add.at(out.T, src.ei, (np.abs(Jc * phi[:, src.ej])).T)
    np.add.at(out.T, src.ej, (np.abs(Jc * phi[:, src.ei])).T)
    return out * c0[:, None]


def _force(M, P, src, variant, R, seed=1):
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, R)
    try:
        lam = wl.dirichlet_lambdas(R, src.K, seed)
        rng = np.random.default_rng(seed)
        x0 = rng.uniform(-0.5, 0.5, (R, src.n)).astype(np.float32)
        dt = 2.0 ** -10
        yo = torch.zeros((R, src.n), device="cuda")
        xo = torch.zeros((R, src.n), device="cuda")
        p = M.moq_default_params(variant=variant, steps=1, dt=dt, alpha=0.0, schedule=torch.ones(1, device="cuda"),
                                 x_init=_dev(x0), y_init=torch.zeros((R, src.n), device="cuda"), x_out=xo, y_out=yo)
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense(d, _dev(lam), R, p, 0, 0, bits)
        M.moq_dense_status(d)
        torch.cuda.synchronize()
    finally:
        M.moq_dense_destroy(d)
    return lam, x0, yo.cpu().numpy().astype(np.float64) / dt, xo.cpu().numpy()


@pytest.mark.parametrize("n,R,K", [(200, 300, 3), (128, 128, 4), (70, 130, 2), (300, 64, 3)])
def test_dense_dsb_force_exact(M, P, oracle, n, R, K):
    src = wl.random_graph(n, 1.0, n + R, K=K, wmax=100)  # complete graph, |J| <= 100
    lam, x0, f_gpu, _ = _force(M, P, src, "dsb", R)
    ref = oracle.sb(src, lam.astype(np.float64), variant="dsb", steps=1, dt=2.0 ** -10, alpha=0.0, schedule=[1.0],
                    x_init=x0.astype(np.float64), y_init=np.zeros((R, n)))
    f_ref = ref["y"] / 2.0 ** -10
    scale = _abs_force_scale(src, lam, np.where(x0 >= 0, 1.0, -1.0), ref["c0"])
    err = np.abs(f_gpu - f_ref)
    assert np.all(err <= 1e-5 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())


def test_dense_bsb_force_bf16_bound(M, P, oracle):
    src = wl.random_graph(260, 0.7, 5, K=3, wmax=100)
    R = 200
    lam, x0, f_gpu, _ = _force(M, P, src, "bsb", R)
    ref = oracle.sb(src, lam.astype(np.float64), variant="bsb", steps=1, dt=2.0 ** -10, alpha=0.0, schedule=[1.0],
                    x_init=x0.astype(np.float64), y_init=np.zeros((R, src.n)))
    scale = _abs_force_scale(src, lam, x0.astype(np.float64), ref["c0"])
    err = np.abs(f_gpu - ref["y"] / 2.0 ** -10)
    assert np.all(err <= 4e-3 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())


def test_dense_short_trajectory(M, P, oracle):
    # dSB, no noise: products are exact, so a few steps follow the FP64 trajectory closely
    # (replicas with a spin within 1e-3 of the sign switch at the start are left out)
    src = wl.random_graph(150, 1.0, 8, K=3, wmax=50)
    inst = P.Instance(src)
    R, T = 256, 6
    d = M.moq_dense_create(inst.handle, R)
    lam = wl.dirichlet_lambdas(R, 3, 2)
    xo = torch.zeros((R, src.n), device="cuda")
    yo = torch.zeros((R, src.n), device="cuda")
    p = M.moq_default_params(variant="dsb", steps=T, dt=0.5, x_out=xo, y_out=yo)
    bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
    M.moq_sample_dense(d, _dev(lam), R, p, 4, 0, bits)
    M.moq_dense_status(d)
    ref = oracle.sb(src, lam.astype(np.float64), variant="dsb", steps=T, dt=0.5, seed=4)
    x0 = np.array([[oracle.initial_state(4, 0, r, i)[0] for i in range(src.n)] for r in range(R)])
    ok = np.all(np.abs(x0) > 1e-3, axis=1)
    assert ok.sum() >= 8
    assert np.abs(xo.cpu().numpy()[ok] - ref["x"][ok]).max() < 1e-4
    s = np.where(xo.cpu().numpy() >= 0, 1, -1)
    assert np.array_equal(wl.bits_to_signs(bits.cpu().numpy().view(np.uint64), src.n), s)
    M.moq_dense_destroy(d)


def test_dense_noise_is_gaussian(M, P):
    # J = 0 (all weights zero), x = y = 0, a = a0: after one step y = dt * alpha * eta
    n, R = 130, 260
    iu, ju = np.triu_indices(n, 1)
    src = wl.Instance(n, iu.astype(np.int32), ju.astype(np.int32), np.zeros((2, iu.size), np.int32))
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, R)
    yo = torch.zeros((R, n), device="cuda")
    z = torch.zeros((R, n), device="cuda")
    p = M.moq_default_params(steps=1, dt=0.5, alpha=0.2, schedule=torch.ones(1, device="cuda"), x_init=z, y_init=z, y_out=yo)
    M.moq_sample_dense(d, _dev(np.full((R, 2), 0.5)), R, p, 9, 0, torch.zeros((R, 3), dtype=torch.int64, device="cuda"))
    eta = yo.cpu().numpy().ravel() / (0.5 * 0.2)
    assert abs(eta.mean()) < 0.02 and abs(eta.var() - 1) < 0.03
    assert stats.kstest(eta[:20000], "norm").pvalue > 1e-3
    assert len(np.unique(eta)) > 0.99 * eta.size
    M.moq_dense_destroy(d)


def test_dense_final_hv_distribution(M, P, oracle):
    # chaotic trajectories: the final front's hypervolume over 16 seeds is distributed
    # like the FP64 oracle's
    src = wl.app_e_correlated(25, 1.0, 3)
    inst = P.Instance(src)
    R, T = 256, 120
    d = M.moq_dense_create(inst.handle, R)
    lam = wl.dirichlet_lambdas(R, 3, 5)
    params = M.moq_default_params(steps=T, dt=0.5, alpha=0.1)
    bits = torch.zeros((R, 1), dtype=torch.int64, device="cuda")
    hv_g, hv_c = [], []
    for seed in range(16):
        M.moq_sample_dense(d, _dev(lam), R, params, seed, 0, bits)
        c = oracle.cuts(src, bits.cpu().numpy().view(np.uint64))
        hv_g.append(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref))
        o = oracle.sb(src, lam.astype(np.float64), steps=T, dt=0.5, alpha=0.1, seed=500 + seed)
        c = oracle.cuts(src, o["bits"])
        hv_c.append(oracle.hypervolume(c[oracle.pareto_filter(c)], inst.ref))
    M.moq_dense_status(d)
    M.moq_dense_destroy(d)
    assert stats.mannwhitneyu(hv_g, hv_c).pvalue > 0.01
    assert abs(np.median(hv_g) / np.median(hv_c) - 1) < 0.03


@pytest.mark.parametrize("n,R,K,variant,alpha,sched", [(25, 300, 3, "dsb", 0.1, False), (128, 129, 2, "bsb", 0.1, False),
                                                      (100, 1, 3, "bsb", 0.0, True), (70, 640, 2, "dsb", 0.0, False),
                                                      (128, 256, 3, "dsb", 0.2, True)])
def test_dense_resident_matches_step_kernel(M, P, monkeypatch, n, R, K, variant, alpha, sched):
    # graphs of at most 128 spins run all steps in one launch from shared memory and TMEM;
    # the per-step kernel (MOQ_DENSE_RESIDENT=0) does the same arithmetic, so bits, x and y
    # agree bit for bit (ragged and single replica tiles, both variants, with and without
    # noise and an explicit pump schedule)
    src = wl.random_graph(n, 1.0, 40 + n + R, K=K, wmax=200)
    inst = P.Instance(src)
    T = 60
    lam = _dev(wl.dirichlet_lambdas(R, K, 3))
    schedule = torch.linspace(0.0, 1.0, T, device="cuda") ** 2 if sched else None
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MOQ_DENSE_RESIDENT", mode)
        d = M.moq_dense_create(inst.handle, R)
        try:
            xo = torch.zeros((R, n), device="cuda")
            yo = torch.zeros((R, n), device="cuda")
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            p = M.moq_default_params(variant=variant, steps=T, dt=0.5, alpha=alpha, schedule=schedule, x_out=xo, y_out=yo)
            M.moq_sample_dense(d, lam, R, p, 11, 2, bits)
            M.moq_dense_status(d)
            out[mode] = (bits.cpu(), xo.cpu(), yo.cpu())
        finally:
            M.moq_dense_destroy(d)
    for a, b in zip(out["1"], out["0"]):
        assert torch.equal(a, b)
    assert len(torch.unique(out["1"][0], dim=0)) > 1 or R == 1


@pytest.mark.parametrize("n,Mn,K,wmax", [(150, 300, 3, 50), (257, 129, 2, 60000), (128, 700, 4, 5000), (90, 1, 3, 128),
                                         (100, 40, 3, 127)])
def test_dense_cuts_bit_exact(M, P, oracle, n, Mn, K, wmax):
    # exact cuts on the tensor cores (J = 256 J_hi + J_lo, +-1 operands, integer epilogue)
    # against the oracle's literal sum and the CUDA-core edge walk; ragged n and M, weights
    # up to the split bound, and weights small enough for the single-part path
    src = wl.random_graph(n, 0.9, n + Mn, K=K, wmax=wmax)
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, max(Mn, 64))
    try:
        bits = wl.random_sign_bits(Mn, n, 5)
        bits[0] = 0  # all s = +1: every cut is 0
        bd = torch.from_numpy(bits.view(np.int64)).cuda()
        cuts = torch.zeros((Mn, K), dtype=torch.int64, device="cuda")
        M.moq_dense_evaluate_cuts(d, bd, Mn, cuts)
        M.moq_dense_status(d)
        got = cuts.cpu().numpy()
        assert np.array_equal(got, oracle.cuts(src, bits))
        ref = torch.zeros_like(cuts)
        M.moq_evaluate_cuts(inst.handle, bd, Mn, ref)
        assert torch.equal(cuts, ref)
        assert np.all(got[0] == 0)
    finally:
        M.moq_dense_destroy(d)


def test_dense_cuts_reject_large_weights(M, P):
    src = wl.random_graph(40, 1.0, 3, K=2, wmax=10)
    src.w[0, 0] = 70000
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, 16)
    try:
        cuts = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
        with pytest.raises(M.MoqError) as e:
            M.moq_dense_evaluate_cuts(d, torch.zeros((4, 1), dtype=torch.int64, device="cuda"), 4, cuts)
        assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    finally:
        M.moq_dense_destroy(d)


def test_round_driver_on_the_dense_sampler(M, P):
    # the round driver runs the tensor-core sampler and cut evaluation when asked; the
    # archive it fills reaches the hypervolume of a reference run on the same sampler
    src = wl.complete_graph(150, 12, K=3)
    inst = P.Instance(src)
    dh = M.moq_dense_create(inst.handle, 512)
    arch = P.Archive(src.n, 3, capacity=1 << 16, max_batch=512)
    buf = P.RoundBuffers(512, src.n, 3)
    params = M.moq_default_params(variant="dsb", steps=300, dt=0.5, alpha=0.1)
    for rnd in range(4):
        P.sample_round(inst, arch, buf, params, 7, rnd, dense=dh)
    M.moq_dense_status(dh)
    target = arch.hypervolume(inst.ref)
    c, _, _ = arch.copy_out()
    ref_cuts = torch.zeros((512, 3), dtype=torch.int64, device="cuda")
    M.moq_evaluate_cuts(inst.handle, buf.bits, 512, ref_cuts)  # the last round's cuts, CUDA-core path
    assert torch.equal(ref_cuts, buf.cuts)
    M.moq_dense_destroy(dh)
    arch.close()
    out = P.time_to_target(src, target, params, 512, seed=7, max_rounds=4, dense=True)
    assert out["reached"] and out["rounds"] <= 4 and out["hv"] >= target


# ---- the plain FP32 form on the CUDA cores -------------------------------------------

def _force_fp32(M, P, src, variant, R, seed=1):
    inst = P.Instance(src)
    d = M.moq_dense_fp32_create(inst.handle, R)
    try:
        lam = wl.dirichlet_lambdas(R, src.K, seed)
        rng = np.random.default_rng(seed)
        x0 = rng.uniform(-0.5, 0.5, (R, src.n)).astype(np.float32)
        dt = 2.0 ** -10
        yo = torch.zeros((R, src.n), device="cuda")
        p = M.moq_default_params(variant=variant, steps=1, dt=dt, alpha=0.0, schedule=torch.ones(1, device="cuda"),
                                 x_init=_dev(x0), y_init=torch.zeros((R, src.n), device="cuda"), y_out=yo)
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense_fp32(d, _dev(lam), R, p, 0, 0, bits)
        torch.cuda.synchronize()
    finally:
        M.moq_dense_fp32_destroy(d)
    return lam, x0, yo.cpu().numpy().astype(np.float64) / dt


@pytest.mark.parametrize("n,R,K,variant", [(300, 200, 3, "dsb"), (300, 200, 3, "bsb"), (130, 129, 4, "bsb"),
                                           (64, 1, 2, "dsb"), (257, 70, 2, "bsb")])
def test_dense_fp32_force_within_1e5(M, P, oracle, n, R, K, variant):
    # the dense workload's weights (round(1000 N(0,1)), |J| up to about 5000, far from exact
    # in BF16): with FP32 couplings and phi the force meets the 1e-5 normwise FP32 bound
    # against the FP64 oracle for both variants (ragged spin and replica tiles)
    src = wl.complete_graph(n, 70 + n, K=K)
    lam, x0, f_gpu = _force_fp32(M, P, src, variant, R)
    ref = oracle.sb(src, lam.astype(np.float64), variant=variant, steps=1, dt=2.0 ** -10, alpha=0.0, schedule=[1.0],
                    x_init=x0.astype(np.float64), y_init=np.zeros((R, n)))
    phi = np.where(x0 >= 0, 1.0, -1.0) if variant == "dsb" else x0.astype(np.float64)
    scale = _abs_force_scale(src, lam, phi, ref["c0"])
    err = np.abs(f_gpu - ref["y"] / 2.0 ** -10)
    assert np.all(err <= 1e-5 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())


def test_dense_fp32_bsb_short_trajectory(M, P, oracle):
    # noise-free bSB is continuous in the state: a few FP32 steps stay on the FP64 trajectory
    src = wl.complete_graph(200, 91, K=3)
    inst = P.Instance(src)
    R, T = 192, 8
    d = M.moq_dense_fp32_create(inst.handle, R)
    try:
        lam = wl.dirichlet_lambdas(R, 3, 6)
        xo = torch.zeros((R, src.n), device="cuda")
        yo = torch.zeros((R, src.n), device="cuda")
        p = M.moq_default_params(variant="bsb", steps=T, dt=0.5, x_out=xo, y_out=yo)
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense_fp32(d, _dev(lam), R, p, 4, 0, bits)
        ref = oracle.sb(src, lam.astype(np.float64), variant="bsb", steps=T, dt=0.5, seed=4)
        assert np.abs(xo.cpu().numpy() - ref["x"]).max() < 1e-4
        assert np.abs(yo.cpu().numpy() - ref["y"]).max() < 1e-4
    finally:
        M.moq_dense_fp32_destroy(d)


@pytest.mark.parametrize("n,R,K,alpha,sched", [(300, 300, 3, 0.1, False), (100, 130, 3, 0.15, False), (257, 64, 4, 0.1, True),
                                                (129, 1, 2, 0.0, False)])
def test_dense_fp32_matches_tensor_core_form_bitwise(M, P, n, R, K, alpha, sched):
    # dSB with |J| <= 256: every per-objective product is an exact integer in both forms,
    # and the start state, noise counters, force combination and update are the same, so
    # the FP32 CUDA-core form and the BF16 tensor-core form (per-step or resident kernel)
    # give the same bits, x and y over a noisy trajectory
    src = wl.random_graph(n, 1.0, 7 + n + R, K=K, wmax=256)
    inst = P.Instance(src)
    T = 40
    lam = _dev(wl.dirichlet_lambdas(R, K, 12))
    schedule = torch.linspace(0.0, 1.0, T, device="cuda") ** 2 if sched else None
    out = {}
    for form in ("bf16", "fp32"):
        d = (M.moq_dense_create if form == "bf16" else M.moq_dense_fp32_create)(inst.handle, R)
        try:
            xo = torch.zeros((R, n), device="cuda")
            yo = torch.zeros((R, n), device="cuda")
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            p = M.moq_default_params(variant="dsb", steps=T, dt=0.5, alpha=alpha, schedule=schedule, x_out=xo, y_out=yo)
            if form == "bf16":
                M.moq_sample_dense(d, lam, R, p, 21, 3, bits)
                M.moq_dense_status(d)
            else:
                M.moq_sample_dense_fp32(d, lam, R, p, 21, 3, bits)
            out[form] = (bits.cpu(), xo.cpu(), yo.cpu())
        finally:
            (M.moq_dense_destroy if form == "bf16" else M.moq_dense_fp32_destroy)(d)
    for a, b in zip(out["bf16"], out["fp32"]):
        assert torch.equal(a, b)
    assert R == 1 or len(torch.unique(out["fp32"][0], dim=0)) > 1


def test_dense_fp32_rejects_bad_arguments(M, P):
    src = wl.random_graph(40, 1.0, 3, K=2, wmax=10)
    inst = P.Instance(src)
    d = M.moq_dense_fp32_create(inst.handle, 16)
    try:
        p = M.moq_default_params(steps=3)
        bits = torch.zeros((32, 1), dtype=torch.int64, device="cuda")
        with pytest.raises(M.MoqError) as e:
            M.moq_sample_dense_fp32(d, _dev(np.full((32, 2), 0.5)), 32, p, 0, 0, bits)
        assert e.value.code == M.MOQ_ERR_ARG
    finally:
        M.moq_dense_fp32_destroy(d)


# ---- the FP8 (E4M3) form of the dSB step ------------------------------------------------

@pytest.mark.parametrize("n,R,K,alpha,sched", [(300, 300, 3, 0.1, False), (100, 130, 3, 0.15, False), (257, 64, 4, 0.1, True),
                                                (129, 1, 2, 0.0, False)])
def test_dense_fp8_matches_bf16_form_for_small_weights(M, P, n, R, K, alpha, sched):
    # |J| <= 16 is exact in E4M3 (row scale 1) and phi = +-1 is exact, so every per-objective
    # product is the same exact integer as with BF16 operands: the FP8 form gives the bits,
    # x and y of moq_sample_dense (per-step or resident kernel) over a noisy trajectory
    src = wl.random_graph(n, 1.0, 3 + n + R, K=K, wmax=16)
    inst = P.Instance(src)
    T = 40
    lam = _dev(wl.dirichlet_lambdas(R, K, 14))
    schedule = torch.linspace(0.0, 1.0, T, device="cuda") ** 2 if sched else None
    d = M.moq_dense_create(inst.handle, R)
    out = {}
    try:
        for form in ("bf16", "fp8"):
            xo = torch.zeros((R, n), device="cuda")
            yo = torch.zeros((R, n), device="cuda")
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            p = M.moq_default_params(variant="dsb", steps=T, dt=0.5, alpha=alpha, schedule=schedule, x_out=xo, y_out=yo)
            (M.moq_sample_dense if form == "bf16" else M.moq_sample_dense_fp8)(d, lam, R, p, 23, 1, bits)
            M.moq_dense_status(d)
            out[form] = (bits.cpu(), xo.cpu(), yo.cpu())
    finally:
        M.moq_dense_destroy(d)
    for a, b in zip(out["bf16"], out["fp8"]):
        assert torch.equal(a, b)
    assert R == 1 or len(torch.unique(out["fp8"][0], dim=0)) > 1


@pytest.mark.parametrize("n,R,K", [(300, 200, 3), (130, 129, 4), (64, 1, 2)])
def test_dense_fp8_force_within_e4m3_bound(M, P, oracle, n, R, K):
    # the dense workload's weights (|J| up to about 5000): J rounds to E4M3 with a power-of-two
    # row scale (relative error <= 2^-4 per weight, 2^-4 = half an E4M3 ulp), phi = +-1 exact,
    # FP32 accumulation: |f - f64| <= 2^-4 c0 sum_j |J(c)_ij phi_j| against the FP64 oracle
    src = wl.complete_graph(n, 80 + n, K=K)
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, R)
    try:
        lam = wl.dirichlet_lambdas(R, K, 2)
        x0 = np.random.default_rng(3).uniform(-0.5, 0.5, (R, n)).astype(np.float32)
        dt = 2.0 ** -10
        yo = torch.zeros((R, n), device="cuda")
        p = M.moq_default_params(variant="dsb", steps=1, dt=dt, alpha=0.0, schedule=torch.ones(1, device="cuda"),
                                 x_init=_dev(x0), y_init=torch.zeros((R, n), device="cuda"), y_out=yo)
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense_fp8(d, _dev(lam), R, p, 0, 0, bits)
        M.moq_dense_status(d)
        f_gpu = yo.cpu().numpy().astype(np.float64) / dt
    finally:
        M.moq_dense_destroy(d)
    ref = oracle.sb(src, lam.astype(np.float64), variant="dsb", steps=1, dt=dt, alpha=0.0, schedule=[1.0],
                    x_init=x0.astype(np.float64), y_init=np.zeros((R, n)))
    scale = _abs_force_scale(src, lam, np.where(x0 >= 0, 1.0, -1.0), ref["c0"])
    rel = np.abs(f_gpu - ref["y"] / dt) / np.maximum(scale, 1e-30)
    assert rel.max() <= 2.0 ** -4, float(rel.max())
    assert rel.max() > 1e-5  # the weights really are rounded (not the exact path)


def test_dense_fp8_rejects_bsb(M, P):
    src = wl.random_graph(40, 1.0, 3, K=2, wmax=10)
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, 16)
    try:
        p = M.moq_default_params(variant="bsb", steps=3)
        with pytest.raises(M.MoqError) as e:
            M.moq_sample_dense_fp8(d, _dev(np.full((16, 2), 0.5)), 16, p, 0, 0,
                                   torch.zeros((16, 1), dtype=torch.int64, device="cuda"))
        assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    finally:
        M.moq_dense_destroy(d)


@pytest.mark.parametrize("n,R,K", [(300, 200, 3), (130, 129, 4), (64, 1, 2), (257, 70, 3)])
def test_dense_fp8_force_matches_oracle_e4m3_force(M, P, oracle, n, R, K):
    # parity of the FP8 form proper: the oracle's force with the same E4M3 couplings (row
    # scales, nearest-even rounding) in FP64; the E4M3 products are exact and only the FP32
    # accumulation and combination differ, so the 1e-5 normwise FP32 bound applies
    src = wl.complete_graph(n, 90 + n, K=K)
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, R)
    try:
        lam = wl.dirichlet_lambdas(R, K, 6)
        x0 = np.random.default_rng(7).uniform(-0.5, 0.5, (R, n)).astype(np.float32)
        dt = 2.0 ** -10
        yo = torch.zeros((R, n), device="cuda")
        p = M.moq_default_params(variant="dsb", steps=1, dt=dt, alpha=0.0, schedule=torch.ones(1, device="cuda"),
                                 x_init=_dev(x0), y_init=torch.zeros((R, n), device="cuda"), y_out=yo)
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense_fp8(d, _dev(lam), R, p, 0, 0, bits)
        M.moq_dense_status(d)
        f_gpu = yo.cpu().numpy().astype(np.float64) / dt
    finally:
        M.moq_dense_destroy(d)
    phi = np.where(x0 >= 0, 1.0, -1.0)
    c0 = oracle.sb(src, lam.astype(np.float64), steps=0, x_init=np.zeros((R, n)))["c0"]
    f_ref = oracle.force_e4m3(src, lam.astype(np.float64), phi, c0)
    scale = _abs_force_scale(src, lam, phi, c0)
    err = np.abs(f_gpu - f_ref)
    assert np.all(err <= 1e-5 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())


# ---- the split-precision form (BF16(J) + exact residual; bSB: phi_hi + phi_lo) -------------

@pytest.mark.parametrize("n,R,K,alpha,sched", [(300, 300, 3, 0.1, False), (100, 130, 3, 0.15, False), (257, 64, 4, 0.1, True),
                                                (129, 1, 2, 0.0, False)])
def test_dense_split_dsb_matches_fp32_form_bitwise(M, P, n, R, K, alpha, sched):
    # the dense workload's weights (|J| up to about 5000, not exact in BF16): BF16(J) and the
    # residual J - BF16(J) are both exact, so with phi = +-1 every per-objective product is the
    # exact integer the FP32 CUDA-core form computes: same bits, x and y over a noisy trajectory
    src = wl.complete_graph(n, 11 + n + R, K=K)
    inst = P.Instance(src)
    T = 40
    lam = _dev(wl.dirichlet_lambdas(R, K, 15))
    schedule = torch.linspace(0.0, 1.0, T, device="cuda") ** 2 if sched else None
    out = {}
    for form in ("split", "fp32"):
        d = (M.moq_dense_create if form == "split" else M.moq_dense_fp32_create)(inst.handle, R)
        try:
            xo = torch.zeros((R, n), device="cuda")
            yo = torch.zeros((R, n), device="cuda")
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            p = M.moq_default_params(variant="dsb", steps=T, dt=0.5, alpha=alpha, schedule=schedule, x_out=xo, y_out=yo)
            if form == "split":
                M.moq_sample_dense_split(d, lam, R, p, 29, 2, bits)
                M.moq_dense_status(d)
            else:
                M.moq_sample_dense_fp32(d, lam, R, p, 29, 2, bits)
            out[form] = (bits.cpu(), xo.cpu(), yo.cpu())
        finally:
            (M.moq_dense_destroy if form == "split" else M.moq_dense_fp32_destroy)(d)
    for a, b in zip(out["split"], out["fp32"]):
        assert torch.equal(a, b)
    assert R == 1 or len(torch.unique(out["split"][0], dim=0)) > 1


def _force_split(M, P, src, variant, R, seed=1):
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, R)
    try:
        lam = wl.dirichlet_lambdas(R, src.K, seed)
        x0 = np.random.default_rng(seed).uniform(-0.5, 0.5, (R, src.n)).astype(np.float32)
        dt = 2.0 ** -10
        yo = torch.zeros((R, src.n), device="cuda")
        p = M.moq_default_params(variant=variant, steps=1, dt=dt, alpha=0.0, schedule=torch.ones(1, device="cuda"),
                                 x_init=_dev(x0), y_init=torch.zeros((R, src.n), device="cuda"), y_out=yo)
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense_split(d, _dev(lam), R, p, 0, 0, bits)
        M.moq_dense_status(d)
        torch.cuda.synchronize()
    finally:
        M.moq_dense_destroy(d)
    return lam, x0, yo.cpu().numpy().astype(np.float64) / dt


@pytest.mark.parametrize("n,R,K", [(300, 200, 3), (130, 129, 4), (64, 1, 2), (257, 70, 3)])
def test_dense_split_bsb_force_within_1e5(M, P, oracle, n, R, K):
    # bSB on the tensor cores with the FP32 force bound: BF16(J) x_hi + J_res x_hi + BF16(J) x_lo
    # leaves out J_res x_lo (about 2^-18 of each product)
    src = wl.complete_graph(n, 60 + n, K=K)
    lam, x0, f_gpu = _force_split(M, P, src, "bsb", R)
    ref = oracle.sb(src, lam.astype(np.float64), variant="bsb", steps=1, dt=2.0 ** -10, alpha=0.0, schedule=[1.0],
                    x_init=x0.astype(np.float64), y_init=np.zeros((R, n)))
    scale = _abs_force_scale(src, lam, x0.astype(np.float64), ref["c0"])
    err = np.abs(f_gpu - ref["y"] / 2.0 ** -10)
    assert np.all(err <= 1e-5 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())


def test_dense_split_bsb_tracks_fp32_form(M, P):
    # a short noise-free bSB trajectory stays on the FP32 CUDA-core form's
    src = wl.complete_graph(200, 92, K=3)
    inst = P.Instance(src)
    R, T = 192, 8
    lam = _dev(wl.dirichlet_lambdas(R, 3, 6))
    res = {}
    for form in ("split", "fp32"):
        d = (M.moq_dense_create if form == "split" else M.moq_dense_fp32_create)(inst.handle, R)
        try:
            xo = torch.zeros((R, src.n), device="cuda")
            p = M.moq_default_params(variant="bsb", steps=T, dt=0.5, x_out=xo)
            bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
            (M.moq_sample_dense_split if form == "split" else M.moq_sample_dense_fp32)(d, lam, R, p, 4, 0, bits)
            torch.cuda.synchronize()
            res[form] = xo.cpu().numpy()
        finally:
            (M.moq_dense_destroy if form == "split" else M.moq_dense_fp32_destroy)(d)
    assert np.abs(res["split"] - res["fp32"]).max() < 1e-5


def test_dense_split_rejects_large_weights(M, P):
    src = wl.random_graph(40, 1.0, 3, K=2, wmax=10)
    src.w[0, 0] = 70000
    inst = P.Instance(src)
    d = M.moq_dense_create(inst.handle, 16)
    try:
        with pytest.raises(M.MoqError) as e:
            M.moq_sample_dense_split(d, _dev(np.full((16, 2), 0.5)), 16, M.moq_default_params(steps=3), 0, 0,
                                     torch.zeros((16, 1), dtype=torch.int64, device="cuda"))
        assert e.value.code == M.MOQ_ERR_UNSUPPORTED
    finally:
        M.moq_dense_destroy(d)


def test_round_driver_dense_forms(M, P):
    # the round driver runs every operand form; the split form's archive is the one the FP32
    # CUDA-core sampler's samples give (identical dSB samples), and the E4M3 form gives a
    # non-empty mutually non-dominated front
    src = wl.complete_graph(150, 13, K=3)
    inst = P.Instance(src)
    R = 256
    params = M.moq_default_params(variant="dsb", steps=200, dt=0.5, alpha=0.1)
    dh = M.moq_dense_create(inst.handle, R)
    hv = {}
    for form in ("split", "fp8", "bf16"):
        arch = P.Archive(src.n, 3, capacity=1 << 16, max_batch=R)
        buf = P.RoundBuffers(R, src.n, 3)
        for rnd in range(2):
            P.sample_round(inst, arch, buf, params, 7, rnd, dense=dh, dense_form=form)
        M.moq_dense_status(dh)
        hv[form] = arch.hypervolume(inst.ref)
        c, _, _ = arch.copy_out()
        assert len(c) > 0
        arch.close()
    M.moq_dense_destroy(dh)
    d32 = M.moq_dense_fp32_create(inst.handle, R)
    arch = P.Archive(src.n, 3, capacity=1 << 16, max_batch=R)
    buf = P.RoundBuffers(R, src.n, 3)
    for rnd in range(2):
        M.moq_lambda_dirichlet(3, R, 7, rnd, buf.lam)
        M.moq_sample_dense_fp32(d32, buf.lam, R, params, 7, rnd, buf.bits)
        M.moq_evaluate_cuts(inst.handle, buf.bits, R, buf.cuts)
        arch.merge(buf.cuts, buf.bits, R, R * rnd)
    assert arch.hypervolume(inst.ref) == hv["split"]
    arch.close()
    M.moq_dense_fp32_destroy(d32)


def test_dense_forms_edge_cases(M, P, oracle):
    # T = 0 reads out the start state (the same Philox start in every form, the oracle's
    # signs); R = 0 is a no-op; a handle rejects more replicas than it was made for
    src = wl.complete_graph(70, 21, K=2)
    inst = P.Instance(src)
    R = 33
    lam = _dev(wl.dirichlet_lambdas(R, 2, 3))
    d = M.moq_dense_create(inst.handle, R)
    d32 = M.moq_dense_fp32_create(inst.handle, R)
    try:
        want = np.array([[oracle.initial_state(8, 1, r, i)[0] < 0 for i in range(src.n)] for r in range(R)])
        for fn, h in ((M.moq_sample_dense, d), (M.moq_sample_dense_fp8, d), (M.moq_sample_dense_split, d),
                      (M.moq_sample_dense_fp32, d32)):
            bits = torch.full((R, inst.W), -1, dtype=torch.int64, device="cuda")
            fn(h, lam, R, M.moq_default_params(variant="dsb", steps=0), 8, 1, bits)
            torch.cuda.synchronize()
            s = wl.bits_to_signs(bits.cpu().numpy().view(np.uint64), src.n)
            assert np.array_equal(s < 0, want)
            untouched = torch.full((1, inst.W), -1, dtype=torch.int64, device="cuda")
            fn(h, lam, 0, M.moq_default_params(steps=5), 8, 1, untouched)  # R = 0: nothing written
            torch.cuda.synchronize()
            assert int(untouched[0, 0]) == -1
            with pytest.raises(M.MoqError) as e:
                fn(h, _dev(np.full((R + 1, 2), 0.5)), R + 1, M.moq_default_params(steps=2), 0, 0,
                   torch.zeros((R + 1, inst.W), dtype=torch.int64, device="cuda"))
            assert e.value.code == M.MOQ_ERR_ARG
        M.moq_dense_status(d)
    finally:
        M.moq_dense_destroy(d)
        M.moq_dense_fp32_destroy(d32)
    with pytest.raises(M.MoqError) as e:
        M.moq_dense_fp32_create(inst.handle, 0)
    assert e.value.code == M.MOQ_ERR_ARG


@pytest.mark.slow
def test_dense_full_size_sampled_parity(M, P, oracle):
    # the dense benchmark's configuration (complete graph n = 2000, K = 3, R = 8192, the
    # persistent step kernel's launch): one step of every operand form from the same state,
    # checked on sampled replicas against the FP64 oracle with each form's stated bound, and
    # the exact tensor-core cuts of a short run on sampled rows against the oracle's cuts
    n, K, R = 2000, 3, 8192
    src = wl.complete_graph(n, 2000, K=K)
    inst = P.Instance(src)
    lam = wl.dirichlet_lambdas(R, K, 5)
    x0 = np.random.default_rng(11).uniform(-1, 1, (R, n)).astype(np.float32)
    sel = np.random.default_rng(12).choice(R, 12, replace=False)
    sel.sort()
    dt = 2.0 ** -10
    d = M.moq_dense_create(inst.handle, R)
    d32 = M.moq_dense_fp32_create(inst.handle, R)
    ld, xd = _dev(lam), _dev(x0)
    forces = {}
    try:
        for name, variant, fn, h in (("fp32_bsb", "bsb", M.moq_sample_dense_fp32, d32), ("split_bsb", "bsb", M.moq_sample_dense_split, d),
                                     ("bf16_bsb", "bsb", M.moq_sample_dense, d), ("split_dsb", "dsb", M.moq_sample_dense_split, d),
                                     ("fp8_dsb", "dsb", M.moq_sample_dense_fp8, d)):
            yo = torch.zeros((R, n), device="cuda")
            p = M.moq_default_params(variant=variant, steps=1, dt=dt, alpha=0.0, schedule=torch.ones(1, device="cuda"),
                                     x_init=xd, y_init=torch.zeros((R, n), device="cuda"), y_out=yo)
            fn(h, ld, R, p, 0, 0, torch.zeros((R, inst.W), dtype=torch.int64, device="cuda"))
            forces[name] = yo[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.float64) / dt
        bits = torch.zeros((R, inst.W), dtype=torch.int64, device="cuda")
        M.moq_sample_dense(d, ld, R, M.moq_default_params(variant="bsb", steps=20, dt=0.5, alpha=0.1), 3, 0, bits)
        cuts = torch.zeros((R, K), dtype=torch.int64, device="cuda")
        M.moq_dense_evaluate_cuts(d, bits, R, cuts)
        M.moq_dense_status(d)
        rows = bits.cpu().numpy().view(np.uint64)[sel]
        assert np.array_equal(cuts.cpu().numpy()[sel], oracle.cuts(src, rows))
    finally:
        M.moq_dense_destroy(d)
        M.moq_dense_fp32_destroy(d32)
    ls, xs = lam[sel].astype(np.float64), x0[sel].astype(np.float64)
    for variant in ("bsb", "dsb"):
        ref = oracle.sb(src, ls, variant=variant, steps=1, dt=dt, alpha=0.0, schedule=[1.0], x_init=xs, y_init=np.zeros_like(xs))
        phi = xs if variant == "bsb" else np.where(xs >= 0, 1.0, -1.0)
        scale = _abs_force_scale(src, ls, phi, ref["c0"])
        f64 = ref["y"] / dt
        bounds = {"bsb": {"fp32_bsb": 1e-5, "split_bsb": 1e-5, "bf16_bsb": 4e-3}, "dsb": {"split_dsb": 1e-5}}[variant]
        for name, bound in bounds.items():
            err = np.abs(forces[name] - f64)
            assert np.all(err <= bound * scale + 1e-30), (name, float((err / scale).max()))
        if variant == "dsb":
            f8 = oracle.force_e4m3(src, ls, phi, ref["c0"])
            err = np.abs(forces["fp8_dsb"] - f8)
            assert np.all(err <= 1e-5 * scale + 1e-30), float((err / scale).max())
