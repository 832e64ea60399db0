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


# ------------------------------------------------ the BF16-operand variant (tensor-core surrogate)
def test_bf16_rounding_matches_torch(oracle):
    # rho is round to nearest even at 8 significant bits: torch's float32 -> bfloat16 cast on
    # random floats, every midpoint between neighbouring BF16 values of a range, subnormals
    import torch
    rng = np.random.default_rng(3)
    vals = np.concatenate([rng.normal(0, 1, 3000), rng.normal(0, 1e-3, 1000) * 10.0 ** rng.integers(-30, 30, 1000),
                           np.array([0.0, -0.0, 1.0, -1.0, 3.0e-39, -7.1e-40, 2.0 ** -133, 3 * 2.0 ** -134])]).astype(np.float32)
    b = torch.from_numpy(np.arange(0x3F80, 0x4080, dtype=np.int32)).to(torch.int16).view(torch.bfloat16).float().numpy()
    mids = ((b[:-1].astype(np.float64) + b[1:]) / 2).astype(np.float32)  # exact in float32
    vals = np.concatenate([vals, mids, -mids])
    want = torch.from_numpy(vals).to(torch.bfloat16).float().numpy().astype(np.float64)
    got = np.array([oracle.bf16(float(v)) for v in vals])
    assert np.array_equal(got, want)


def _exact_case(seed, din=4, h=8, dout=2, B=4):
    """Weights in {0, +-1/8}, inputs in {-1, 0, 1}, targets y + {0, +-1/8}: with these every
    product operand of the network has at most a few significant bits, so rounding to BF16
    changes nothing."""
    rng = np.random.default_rng(seed)
    P = din * h + h + h * h + h + dout * h + dout
    p = rng.choice([-0.125, 0.0, 0.125], P)
    X = rng.choice([-1.0, 0.0, 1.0], (B, din))
    return p, X


def test_bf16_variant_equals_exact_network_on_exactly_representable_operands(oracle):
    for seed in range(5):
        p, X = _exact_case(seed)
        Y = oracle.mlp_forward(p, X, 4, 8, 2)
        assert np.array_equal(oracle.mlp_forward_bf16(p, X, 4, 8, 2), Y)
        T = Y + np.random.default_rng(seed).choice([-0.125, 0.0, 0.125], Y.shape)
        L, g = oracle.mlp_loss_grad(p, X, T, 4, 8, 2)
        Lb, gb = oracle.mlp_loss_grad_bf16(p, X, T, 4, 8, 2)
        assert Lb == L and np.array_equal(gb, g)
        assert np.abs(g).max() > 0


def test_bf16_variant_rounds_within_its_bound(oracle):
    # on generic values the rounding is active, and the gradient stays within a few BF16
    # units (2^-8) of the exact network's, normwise
    rng = np.random.default_rng(4)
    P = oracle.mlp_param_count(DIN, H, DOUT)
    p = np.array([oracle.bf16(v) for v in rng.normal(0, 0.3, P)])
    X = rng.normal(0, 1, (64, DIN))
    T = rng.normal(0, 1, (64, DOUT))
    L, g = oracle.mlp_loss_grad(p, X, T, DIN, H, DOUT)
    Lb, gb = oracle.mlp_loss_grad_bf16(p, X, T, DIN, H, DOUT)
    rel = np.linalg.norm(gb - g) / np.linalg.norm(g)
    assert 1e-5 < rel < 8 * 2.0 ** -8
    assert 0 < abs(Lb - L) / L < 8 * 2.0 ** -8


def test_gradient_descent_fits_a_tiny_dataset_exactly(oracle):
    # the exact-fit check: 6 points, 4 targets each, and a network with many more parameters
    # than targets; plain gradient descent on the oracle's loss gradient drives the loss to ~0
    # (a sign error or a dropped term in the gradient stalls it far above)
    rng = np.random.default_rng(4)
    X, T = rng.normal(size=(6, DIN)), rng.uniform(-1, 1, size=(6, DOUT))
    p = rng.normal(0, 0.3, oracle.mlp_param_count(DIN, H, DOUT))
    loss0, _ = oracle.mlp_loss_grad(p, X, T, DIN, H, DOUT)
    m, v = np.zeros_like(p), np.zeros_like(p)
    for t in range(1, 3001):  # Adam on the oracle's gradient
        loss, g = oracle.mlp_loss_grad(p, X, T, DIN, H, DOUT)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        p -= 1e-2 * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-12)
    loss, _ = oracle.mlp_loss_grad(p, X, T, DIN, H, DOUT)
    assert loss < 1e-6 * loss0 and loss < 1e-6, (loss0, loss)
    assert np.allclose(oracle.mlp_forward(p, X, DIN, H, DOUT), T, atol=2e-3)
