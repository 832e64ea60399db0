"""Pins of the oracle's surrogate MLP (the learned weight-vector proposal; not in the
paper): central finite differences of the loss, the linear regime against plain matrix
products, and the closed form with zero weights."""
import numpy as np

DIN, H, DOUT = 12, 16, 4


def _split(p):
    o = 0
    out = []
    for shape in [(H, DIN), (H,), (H, H), (H,), (DOUT, H), (DOUT,)]:
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape))
        o += size
    return out


def test_param_count(oracle):
    assert oracle.mlp_param_count(DIN, H, DOUT) == H * DIN + H + H * H + H + DOUT * H + DOUT
    assert oracle.mlp_param_count(12, 128, 4) == 18692


def test_linear_regime_matches_matrix_products(oracle):
    # positive weights and inputs keep every pre-activation positive: the network is the
    # affine map W3 (W2 (W1 x + b1) + b2) + b3
    rng = np.random.default_rng(0)
    p = rng.uniform(0.01, 0.1, oracle.mlp_param_count(DIN, H, DOUT))
    W1, b1, W2, b2, W3, b3 = _split(p)
    X = rng.uniform(0.0, 1.0, (9, DIN))
    want = ((X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(oracle.mlp_forward(p, X, DIN, H, DOUT), want, rtol=1e-12)


def test_relu_cuts_negative_preactivations(oracle):
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.5, oracle.mlp_param_count(DIN, H, DOUT))
    W1, b1, W2, b2, W3, b3 = _split(p)
    X = rng.normal(0, 1, (7, DIN))
    h1 = np.maximum(X @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    assert np.allclose(oracle.mlp_forward(p, X, DIN, H, DOUT), h2 @ W3.T + b3, rtol=1e-12)


def test_zero_weights_closed_form(oracle):
    p = np.zeros(oracle.mlp_param_count(DIN, H, DOUT))
    b3 = np.array([0.5, -1.0, 2.0, 0.25])
    p[-DOUT:] = b3
    rng = np.random.default_rng(2)
    X, T = rng.normal(size=(5, DIN)), rng.normal(size=(5, DOUT))
    loss, g = oracle.mlp_loss_grad(p, X, T, DIN, H, DOUT)
    assert np.isclose(loss, np.mean((b3 - T) ** 2))
    assert np.allclose(g[-DOUT:], 2 * (b3 - T).mean(axis=0) / DOUT)


def test_gradient_central_differences(oracle):
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.4, oracle.mlp_param_count(DIN, H, DOUT))
    X, T = rng.normal(size=(11, DIN)), rng.normal(size=(11, DOUT))
    loss, g = oracle.mlp_loss_grad(p, X, T, DIN, H, DOUT)
    hstep = 1e-6
    idx = rng.choice(p.size, 80, replace=False)
    for q in np.concatenate([idx, [0, p.size - 1, H * DIN, H * DIN + H + 5]]):
        pp, pm = p.copy(), p.copy()
        pp[q] += hstep
        pm[q] -= hstep
        fd = (oracle.mlp_loss_grad(pp, X, T, DIN, H, DOUT)[0] - oracle.mlp_loss_grad(pm, X, T, DIN, H, DOUT)[0]) / (2 * hstep)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q])), (q, fd, g[q])
