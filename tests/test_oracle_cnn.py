"""Pins of the oracle's warm-start network (oracle/cnn.py): the hand-written backward pass must
match central finite differences of the forward pass, the convolution must match a direct
sum over the 3x3 taps, and the BF16 rounding must round to nearest even."""
import numpy as np
import pytest

import workloads as W


def projections(p, s):
    """P_s and its transpose I - Q_s A_s from the oracle's operators."""
    A = p.sub_A(s)

    def P(v):
        return p.sub_apply_P(s, v)

    def PT(v):
        return v - p.sub_apply_Z(s, p.coarse_solve(s, p.sub_apply_Zt(s, A @ v)))
    return P, PT


def _batch(oracle_mod):
    p = oracle_mod.Problem(11, 7.0)
    p.setup_dd(2, 1, 1, [0, 5, 11], [0, 11])
    p.setup_deflation()
    out = []
    for s in range(p.nsub):
        b = p.box(s)
        f = W.random_complex(p.sub_n(s), 40 + s)
        out.append((f, (b["ny"], b["nx"]), p.sub_A(s)) + projections(p, s))
    return out, p


def test_transpose_projection(oracle_mod):
    """<P u, v> = <u, Pᵀ v> for the transpose used by the gradient."""
    batch, p = _batch(oracle_mod)
    f, shape, A, P, PT = batch[0]
    u, v = W.random_complex(f.size, 1), W.random_complex(f.size, 2)
    assert abs(np.sum(P(u) * v) - np.sum(u * PT(v))) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(v)


def test_conv_matches_direct_sum():
    from oracle import cnn
    rng = np.random.default_rng(0)
    img = rng.standard_normal((5, 6, 4))
    Wt = rng.standard_normal((3, 9, 4))
    b = rng.standard_normal(3)
    y = cnn.conv(img, Wt, b)
    for (yy, xx) in [(0, 0), (2, 3), (4, 5), (1, 0)]:
        for co in range(3):
            ref = b[co]
            for k in range(9):
                sy, sx = yy + k // 3 - 1, xx + k % 3 - 1
                if 0 <= sy < 5 and 0 <= sx < 6:
                    ref += Wt[co, k] @ img[sy, sx]
            assert y[yy, xx, co] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_bf16_rounding():
    from oracle import cnn
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -3.140625, 1e-3], dtype=np.float32)
    r = cnn.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie → even mantissa
    assert r[2] == 1.0 + 2 ** -6           # tie → even (rounds up)
    assert r[3] == -3.140625
    assert abs(r[4] - 1e-3) <= 2 ** -9 * 1e-3


def test_gradient_matches_finite_differences(oracle_mod):
    from oracle import cnn
    batch, _ = _batch(oracle_mod)
    rng = np.random.default_rng(1)
    params = rng.standard_normal(cnn.NPARAM) * 0.2
    L, g = cnn.loss_and_grad(params, batch, kh=0.5)
    idx = rng.choice(cnn.NPARAM, 24, replace=False)
    off = cnn.offsets()
    idx = np.concatenate([idx, [off[1] - 1, off[3] + 5, off[4] - 1]])   # biases and last layer
    eps = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (cnn.loss_and_grad(pp, batch, 0.5, False)[0] - cnn.loss_and_grad(pm, batch, 0.5, False)[0]) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(L)))


def test_zero_network_gives_zero_guess(oracle_mod):
    from oracle import cnn
    batch, _ = _batch(oracle_mod)
    f, shape = batch[0][0], batch[0][1]
    x0 = cnn.guess(np.zeros(cnn.NPARAM), f, shape, 0.5)
    assert np.all(x0 == 0)
    L, _ = cnn.loss_and_grad(np.zeros(cnn.NPARAM), batch, 0.5, False)
    # with a zero guess the loss is mean_t ||P f̂_t||²/||P f̂_t||² = 1 exactly
    assert L == pytest.approx(1.0, rel=1e-12)


def test_bf16_activation_forward():
    """With act_bf16 every hidden activation is a BF16 value (low 16 bits of its FP32 pattern
    zero) and the output stays within the BF16 rounding (2^-9 relative per activation) of the
    unrounded forward, amplified by three layers."""
    from oracle import cnn
    rng = np.random.default_rng(5)
    params = rng.standard_normal(cnn.NPARAM) * 0.15
    img = rng.standard_normal((9, 11, 4))
    img[..., 3] = 0.0
    a = cnn.forward(params, img, act_bf16=True)
    b = cnn.forward(params, img)
    for l in (1, 2, 3):
        bits = a[l].astype(np.float32).view(np.uint32)
        assert np.all(bits & 0xFFFF == 0)
        assert np.array_equal(a[l].astype(np.float32).astype(np.float64), a[l])
    rel = np.linalg.norm(a[4] - b[4]) / np.linalg.norm(b[4])
    assert 0 < rel < 3 * 2.0 ** -9 * 8
