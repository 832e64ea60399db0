"""Host logic of the round driver that needs no GPU: the weight rescaling for instances whose
objectives were scaled to integers (Appendix E's J2 = 0.2 A - 5 B is stored as A - 25 B), and
the memory layout the round drivers build with."""
import numpy as np
import torch

from paper_2604_26477_b300 import workloads as wl


def test_source_scalarisation_reproduces_the_papers_weighted_sum():
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import pipeline as P
    rng = np.random.default_rng(2)
    src = wl.app_e_correlated(30, 1.0, 7)
    # the source objectives: the stored weights divided by their scale (J2 = 0.2 A - 5 B)
    source_w = src.w.astype(np.float64) / src.objective_scale[:, None]
    assert np.array_equal(source_w[1] * 5, src.w[1])
    lam = torch.from_numpy(rng.dirichlet(np.ones(3), 64))
    stored = P.source_scalarisation(lam.clone(), src.objective_scale).numpy()
    # J(c) on the stored integer weights with the rescaled vectors == the paper's J(c)
    assert np.allclose(stored @ src.w.astype(np.float64), lam.numpy() @ source_w, rtol=1e-12, atol=1e-12)
    assert np.allclose(stored[:, 1] * 5, lam.numpy()[:, 1]) and np.array_equal(stored[:, [0, 2]], lam.numpy()[:, [0, 2]])
    # instances without a scale are left alone
    same = lam.clone()
    assert P.source_scalarisation(same, None) is same and torch.equal(same, lam)


def test_round_layout_policy():
    # the round drivers build float16 rounds and graphs of up to 128 spins with the plain
    # layout, larger FP32 ones with the bank-conflict planner
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import moqaia as M
    from paper_2604_26477_b300 import pipeline as P
    fp32 = M.moq_default_params(steps=10)
    fp16 = M.moq_default_params(steps=10, precision="fp16")
    assert P.round_layout(fp16, 1024) == M.MOQ_LAYOUT_PLAIN
    assert P.round_layout(fp32, 42) == M.MOQ_LAYOUT_PLAIN
    assert P.round_layout(fp32, 128) == M.MOQ_LAYOUT_PLAIN
    assert P.round_layout(fp32, 130) == M.MOQ_LAYOUT_DEFAULT
    assert P.round_layout(fp32) == M.MOQ_LAYOUT_DEFAULT
