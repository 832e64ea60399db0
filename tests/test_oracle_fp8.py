"""Pins of the oracle's FP8 (E4M3) force operands: the rounding against torch's
float8_e4m3fn conversion (an independent library routine) and hand values, the row
scales by hand, and the force against the oracle's own SB step where E4M3 is exact."""
import numpy as np
import torch

from paper_2604_26477_b300 import workloads as wl


def _e4m3_values():
    codes = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).double().numpy()
    return np.unique(codes[np.isfinite(codes)])


def test_e4m3_matches_torch_on_every_midpoint_and_random_values(oracle):
    vals = _e4m3_values()
    assert vals.max() == 448.0 and len(vals) == 253  # 126 positive, 126 negative, zero
    mids = (vals[:-1] + vals[1:]) / 2  # exactly halfway: the ties
    rnd = np.random.default_rng(0).uniform(-448, 448, 4000).astype(np.float32).astype(np.float64)
    small = np.random.default_rng(1).uniform(-0.02, 0.02, 2000).astype(np.float32).astype(np.float64)
    m32 = mids.astype(np.float32)  # every midpoint is exact in FP32 (at most 5 significant bits)
    near = np.concatenate([np.nextafter(m32, np.float32(0)), np.nextafter(m32, np.float32(1000))]).astype(np.float64)
    x = np.concatenate([vals, mids, rnd, small, near])  # all exact in FP32, so torch's cast rounds once
    want = torch.from_numpy(x).float().to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(oracle.e4m3(x), want)


def test_e4m3_hand_values(oracle):
    # 17 is halfway between 16 (mantissa 000) and 18 (001): the even mantissa wins; 19 between
    # 18 (001) and 20 (010) goes up; 1 + 1/16 rounds down to 1, 1 + 3/16 up to 1.25; 2^-10 is
    # halfway between 0 and the smallest subnormal 2^-9 (mantissa 001): 0; above 448 saturates
    x = [17, 19, 1.0625, 1.1875, 2.0 ** -10, 3 * 2.0 ** -10, 448, 460, 1e6, -17, 0.3, 240, 232]
    want = [16, 20, 1.0, 1.25, 0.0, 2.0 ** -8, 448, 448, 448, -16, 0.3125, 240, 224]
    assert np.array_equal(oracle.e4m3(x), np.array(want, np.float64))


def test_e4m3_couplings_row_scales(oracle):
    # a path 0-1-2-3-4 with one objective: row maxima 16, 449, 900, 5000, 5000
    ei = np.array([0, 1, 2, 3], np.int32)
    ej = np.array([1, 2, 3, 4], np.int32)
    w = np.array([[16, 449, 900, 5000], [-3, 7, -11, 2]], np.int32)
    inst = wl.Instance(5, ei, ej, w)
    wq_i, wq_j, sc = oracle.e4m3_couplings(inst)
    assert np.array_equal(sc[0], [1, 2, 4, 16, 16])  # 5000 / 16 <= 448 < 5000 / 8
    assert np.array_equal(sc[1], [1, 1, 1, 1, 1])
    assert wq_i[0, 0] == 16 and wq_j[0, 0] == 16  # row 1 (scale 2): 2 * E4M3(16 / 2) = 16
    assert wq_i[0, 1] == 2 * 224 and wq_j[0, 1] == 4 * 112  # 449 / 2 = 224.5 -> 224; 449 / 4 -> 112
    assert np.array_equal(wq_i[1], w[1]) and np.array_equal(wq_j[1], w[1])  # |J| <= 16: exact
    assert np.all(np.abs(wq_i - w) <= 2.0 ** -4 * np.abs(w)) and np.all(np.abs(wq_j - w) <= 2.0 ** -4 * np.abs(w))


def test_force_e4m3_is_the_sb_force_when_weights_are_exact(oracle):
    src = wl.random_graph(40, 0.5, 3, K=3, wmax=16)
    R = 12
    lam = wl.dirichlet_lambdas(R, 3, 1).astype(np.float64)
    x0 = np.random.default_rng(2).uniform(-0.5, 0.5, (R, src.n))
    dt = 2.0 ** -10
    ref = oracle.sb(src, lam, variant="dsb", steps=1, dt=dt, alpha=0.0, schedule=[1.0], x_init=x0, y_init=np.zeros((R, src.n)))
    f = oracle.force_e4m3(src, lam, np.where(x0 >= 0, 1.0, -1.0), ref["c0"])
    assert np.allclose(f, ref["y"] / dt, rtol=1e-9, atol=1e-12)


def test_force_e4m3_within_its_bound(oracle):
    src = wl.complete_graph(30, 5, K=3)
    R = 6
    lam = wl.dirichlet_lambdas(R, 3, 4).astype(np.float64)
    phi = np.where(np.random.default_rng(3).uniform(-1, 1, (R, src.n)) >= 0, 1.0, -1.0)
    c0 = oracle.sb(src, lam, steps=0, x_init=np.zeros((R, src.n)))["c0"]
    f = oracle.force_e4m3(src, lam, phi, c0)
    exact = oracle.force_e4m3(wl.Instance(src.n, src.ei, src.ej, np.zeros_like(src.w)), lam, phi, c0)
    assert np.all(exact == 0)
    Jc = lam @ src.w.astype(np.float64)
    f64 = np.zeros_like(phi)
    scale = np.zeros_like(phi)
    for r in range(R):
        np.add.at(f64[r], src.ei, -Jc[r] * phi[r, src.ej])
        np.add.at(f64[r], src.ej, -Jc[r] * phi[r, src.ei])
        np.add.at(scale[r], src.ei, np.abs(Jc[r]))
        np.add.at(scale[r], src.ej, np.abs(Jc[r]))
    f64 *= c0[:, None]
    scale *= c0[:, None]
    err = np.abs(f - f64)
    assert np.all(err <= 2.0 ** -4 * scale * 1.7)  # per-weight 2^-4 of sum_k c_k |J_k| <= 1.7 sum |J(c)| here
    assert err.max() > 0


def test_split_residual_is_exact_in_bf16():
    # the split-precision dense form rests on this: for every integer |J| <= 65408 (the
    # bound the library enforces, shared with the exact cut evaluation), J = BF16(J) +
    # (J - BF16(J)) with the residual an integer of magnitude <= 128, hence exact in BF16
    J = np.arange(-65408, 65409, dtype=np.float64)
    hi = torch.from_numpy(J).float().to(torch.bfloat16).double().numpy()
    res = J - hi
    assert np.all(np.abs(res) <= 128) and np.all(res == np.round(res))
    assert np.array_equal(torch.from_numpy(res).float().to(torch.bfloat16).double().numpy(), res)
    assert np.array_equal(hi + res, J)
    # the bound is conservative for the residual: between 2^17 and 2^18 an odd residual above
    # 256 needs 9 significant bits and is rounded
    big = np.arange(2 ** 17, 2 ** 17 + 4096, dtype=np.float64)
    r2 = big - torch.from_numpy(big).float().to(torch.bfloat16).double().numpy()
    assert np.any(torch.from_numpy(r2).float().to(torch.bfloat16).double().numpy() != r2)
