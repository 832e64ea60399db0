"""The surrogate MLP on the tensor cores (MOQ_MLP_TENSOR_CORES): forward and gradients against
the FP64 oracle of the same network with BF16 product operands (normwise 1e-4: FP32
accumulation of exact BF16 products), within the stated BF16 distance of the exact network,
deterministic, training, and the proposal on top of it."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DIN, DOUT, H = 12, 4, 128


@pytest.fixture(scope="module")
def M():
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import moqaia
    return moqaia


def _mlp(M, seed=3, max_batch=4096, max_cand=8192, din=DIN, dout=DOUT):
    h = M.moq_mlp_create(din, dout, max_batch, max_cand, seed)
    M.moq_mlp_set_engine(h, "tensor_cores")
    return h


def _data(B, seed, din=DIN, dout=DOUT):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 1, (B, din)).astype(np.float32), rng.normal(0, 1, (B, dout)).astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("din,dout,B", [(12, 4, 1013), (11, 3, 128), (16, 8, 300), (5, 2, 1)])
def test_tc_forward_matches_bf16_oracle(M, oracle, din, dout, B):
    h = _mlp(M, din=din, dout=dout)
    try:
        p = np.random.default_rng(0).normal(0, 0.2, M.moq_mlp_param_count(h)).astype(np.float32)
        M.moq_mlp_set_params(h, p)
        pb = M.moq_mlp_get_params(h, bf16_rounded=True).astype(np.float64)
        X, _ = _data(B, 1, din, dout)  # several 128-row tiles and a ragged tail
        Y = torch.zeros((B, dout), device="cuda")
        M.moq_mlp_forward(h, torch.from_numpy(X).cuda(), B, Y)
        M.moq_mlp_status(h)
        want = oracle.mlp_forward_bf16(pb, X.astype(np.float64), din, H, dout)
        assert _rel(Y.cpu().numpy(), want) <= 1e-4
        exact = oracle.mlp_forward(pb, X.astype(np.float64), din, H, dout)
        assert 1e-5 < _rel(Y.cpu().numpy(), exact) < 8 * 2.0 ** -8
    finally:
        M.moq_mlp_destroy(h)


@pytest.mark.parametrize("din,dout,B", [(12, 4, 32), (12, 4, 777), (12, 4, 4096), (16, 8, 513), (7, 3, 200)])
def test_tc_gradient_matches_bf16_oracle(M, oracle, din, dout, B):
    h = _mlp(M, din=din, dout=dout)
    try:
        X, T = _data(B, B, din, dout)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        P = M.moq_mlp_param_count(h)
        g = torch.zeros(P, device="cuda")
        loss = torch.zeros(1, device="cuda")
        M.moq_mlp_gradient(h, Xd, Td, B, g, loss)
        M.moq_mlp_status(h)
        pb = M.moq_mlp_get_params(h, bf16_rounded=True).astype(np.float64)
        L, gref = oracle.mlp_loss_grad_bf16(pb, X.astype(np.float64), T.astype(np.float64), din, H, dout)
        gg = g.cpu().numpy().astype(np.float64)
        assert abs(loss.item() - L) <= 1e-5 * L
        assert _rel(gg, gref) <= 1e-4
        # every parameter block, not only the norm: W1, b1, W2, b2, W3, b3
        sizes = [H * din, H, H * H, H, dout * H, dout]
        o = 0
        for s in sizes:
            assert _rel(gg[o:o + s], gref[o:o + s]) <= 1e-3, (o, s)
            o += s
        L64, g64 = oracle.mlp_loss_grad(pb, X.astype(np.float64), T.astype(np.float64), din, H, dout)
        assert _rel(gg, g64) < 8 * 2.0 ** -8
        g2 = torch.zeros_like(g)
        M.moq_mlp_gradient(h, Xd, Td, B, g2, None)
        assert torch.equal(g, g2)  # deterministic
    finally:
        M.moq_mlp_destroy(h)


def test_tc_training_fits_a_smooth_map_and_matches_the_split_calls(M):
    ha, hb = _mlp(M, seed=5), _mlp(M, seed=5)
    try:
        rng = np.random.default_rng(7)
        lam = rng.dirichlet(np.ones(DOUT), 4096).astype(np.float32)
        X = np.concatenate([lam, np.tile(rng.normal(0, 1, DIN - DOUT), (4096, 1))], axis=1).astype(np.float32)
        T = np.stack([np.sin(3 * lam[:, 0]), lam[:, 1] ** 2, lam[:, 2] * lam[:, 3], 1 - lam[:, 0]], axis=1).astype(np.float32)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
        M.moq_mlp_gradient(ha, Xd, Td, 4096, None, la)
        first = la.item()
        for s in range(400):
            M.moq_mlp_gradient(ha, Xd, Td, 4096, None, la)
            M.moq_mlp_adam_step(ha, 3e-3)
            M.moq_mlp_train_step(hb, Xd, Td, 4096, 3e-3, lb)
        torch.cuda.synchronize()
        assert torch.equal(la, lb)
        assert np.array_equal(M.moq_mlp_get_params(ha), M.moq_mlp_get_params(hb))
        M.moq_mlp_gradient(ha, Xd, Td, 4096, None, la)
        M.moq_mlp_status(ha)
        assert la.item() < 0.02 * first and la.item() < 2e-3
    finally:
        M.moq_mlp_destroy(ha)
        M.moq_mlp_destroy(hb)


def test_tc_proposal_returns_simplex_vectors_beyond_the_front(M, oracle):
    from paper_2604_26477_b300 import pipeline as P
    K = DOUT
    h = _mlp(M, seed=11)
    arch = P.Archive(42, K, capacity=4096, max_batch=512)
    try:
        rng = np.random.default_rng(5)
        front = rng.integers(0, 100, (300, K)).astype(np.int64)
        arch.merge(torch.from_numpy(front).cuda(), torch.zeros((300, 1), dtype=torch.int64, device="cuda"), 300, 0)
        fc, _, _ = arch.copy_out()
        feats = rng.normal(0, 1, DIN - K).astype(np.float32)
        offset, scale = np.zeros(K, np.int64), np.full(K, 100, np.int64)
        C, R = 2048, 100
        out = torch.zeros((R, K), device="cuda")
        M.moq_lambda_propose(h, arch.handle, feats, offset, scale, C, 21, 3, out, R)
        M.moq_mlp_status(h)
        got = out.cpu().numpy()
        cand = oracle.dirichlet(C, K, 21, 3).astype(np.float32)
        X = np.concatenate([cand, np.tile(feats, (C, 1))], axis=1)
        pred = oracle.mlp_forward_bf16(M.moq_mlp_get_params(h, bf16_rounded=True).astype(np.float64), X.astype(np.float64),
                                       DIN, H, DOUT)
        gap = np.min(np.max(pred[:, None, :] - ((fc - offset) / scale)[None, :, :], axis=2), axis=1)
        order = np.argsort(-gap, kind="stable")
        picked = [int(np.argmin(np.abs(cand - g).sum(axis=1))) for g in got]
        assert np.allclose(cand[picked], got, atol=2e-6)
        assert gap[picked].min() >= gap[order[R - 1]] - 1e-3
        assert np.allclose(got.sum(axis=1), 1, atol=1e-5)
    finally:
        M.moq_mlp_destroy(h)
        arch.close()
