"""CPU oracle of the learned warm start (TEST INFRASTRUCTURE ONLY), numpy FP64.

Network: four 3x3 convolutions (zero padding) 4->32, 32->32, 32->32 with ReLU, then 32->2;
input image of a subdomain right-hand side f: channels (Re f/σ, Im f/σ, k·h, 0) with
σ = sqrt(mean |f|²); output (a, b), guess x0 = σ(a + i b).  Loss of a batch of subdomains:
mean_t ||P_t(f̂_t - A_t y_t)||² / ||P_t f̂_t||², f̂ = f/σ, y = a + i b, with A_t and the
deflation projection P_t = I - A_t Z_t E_t⁻¹ Z_tᵀ (Eq. 4) of the oracle; its transpose is
Pᵀ = I - Q_t A_t (A_t, Q_t = Z_t E_t⁻¹ Z_tᵀ symmetric), so dL/dy_t = -2 A_t Pᵀ P r / (T ||P f̂||²).
Parameters: one flat array, per layer W[cout][ky*3+kx][cin] then b[cout].

The backward pass is written out by hand (chain rule through the loss, the convolutions and the
ReLUs); it is pinned against central finite differences of the forward pass in
tests/test_oracle_cnn.py.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(4, 32, True), (32, 32, True), (32, 32, True), (32, 2, False)]


def offsets():
    off = [0]
    for cin, cout, _ in LAYERS:
        off.append(off[-1] + cout * 9 * cin + cout)
    return off


NPARAM = offsets()[-1]


def unpack(params):
    off = offsets()
    out = []
    for l, (cin, cout, _) in enumerate(LAYERS):
        p = np.asarray(params[off[l]:off[l + 1]], dtype=np.float64)
        out.append((p[:cout * 9 * cin].reshape(cout, 9, cin), p[cout * 9 * cin:]))
    return out


def bf16_round(params):
    """Round FP32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    x = np.ascontiguousarray(params, dtype=np.float32).view(np.uint32).astype(np.uint64)
    x = (x + 0x7FFF + ((x >> 16) & 1)) & 0xFFFF0000
    return x.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(img, dy, dx):
    """out[y, x] = img[y + dy, x + dx] with zeros outside."""
    ny, nx = img.shape[:2]
    out = np.zeros_like(img)
    ys, yd = (slice(dy, ny), slice(0, ny - dy)) if dy >= 0 else (slice(0, ny + dy), slice(-dy, ny))
    xs, xd = (slice(dx, nx), slice(0, nx - dx)) if dx >= 0 else (slice(0, nx + dx), slice(-dx, nx))
    out[yd, xd] = img[ys, xs]
    return out


def conv(img, W, b):
    """y[y, x, co] = b[co] + Σ_k Σ_ci W[co, k, ci] img[y + dy_k, x + dx_k, ci]."""
    out = np.broadcast_to(b, img.shape[:2] + (W.shape[0],)).copy()
    for k in range(9):
        sh = _shift(img, k // 3 - 1, k % 3 - 1)
        out += sh @ W[:, k, :].T
    return out


def input_image(f, shape, kh):
    ny, nx = shape
    f = np.asarray(f, dtype=np.complex128).reshape(ny, nx)
    sigma = np.sqrt(np.mean(np.abs(f) ** 2))
    sigma = sigma if sigma > 0 else 1.0
    img = np.zeros((ny, nx, 4))
    img[..., 0] = f.real / sigma
    img[..., 1] = f.imag / sigma
    img[..., 2] = kh
    return img, sigma


def forward(params, img, act_bf16=False):
    """Activations of every layer.  act_bf16: the inputs of layers 2-4 (the ReLU outputs) are
    rounded to BF16, the storage format of the tensor-core inference; sums stay FP64."""
    acts = [img]
    for (W, b), (_, _, relu) in zip(unpack(params), LAYERS):
        y = conv(acts[-1], W, b)
        if relu:
            y = np.maximum(y, 0.0)
            if act_bf16:
                y = bf16_round(y).reshape(y.shape)
        acts.append(y)
    return acts


def guess(params, f, shape, kh, act_bf16=False):
    img, sigma = input_image(f, shape, kh)
    out = forward(params, img, act_bf16)[-1]
    return (sigma * (out[..., 0] + 1j * out[..., 1])).reshape(-1)


def loss_and_grad(params, batch, kh, with_grad=True):
    """batch: list of (f, (ny, nx), A, P, PT): local matrix A (scipy sparse, real) and callables
    applying the deflation projection P and its transpose to complex vectors."""
    T = len(batch)
    L = 0.0
    grad = np.zeros(NPARAM)
    Ws = unpack(params)
    off = offsets()
    for f, shape, A, P, PT in batch:
        ny, nx = shape
        img, _ = input_image(f, shape, kh)
        acts = forward(params, img)
        out = acts[-1]
        fh = img[..., 0].reshape(-1) + 1j * img[..., 1].reshape(-1)
        y = out[..., 0].reshape(-1) + 1j * out[..., 1].reshape(-1)
        Pf = P(fh)
        q = P(fh - A @ y)
        den = np.vdot(Pf, Pf).real
        L += np.vdot(q, q).real / den / T
        if not with_grad:
            continue
        g = (-2.0 / (T * den)) * (A.T @ PT(q))
        dY = np.zeros((ny, nx, 2))
        dY[..., 0] = g.real.reshape(ny, nx)
        dY[..., 1] = g.imag.reshape(ny, nx)
        for l in range(3, -1, -1):
            W, _ = Ws[l]
            if LAYERS[l][2]:
                dY = dY * (acts[l + 1] > 0)
            X = acts[l]
            cout, _, cin = W.shape
            gW = np.zeros_like(W)
            for k in range(9):
                sh = _shift(X, k // 3 - 1, k % 3 - 1)
                gW[:, k, :] = dY.reshape(-1, cout).T @ sh.reshape(-1, cin)
            grad[off[l]:off[l] + cout * 9 * cin] += gW.reshape(-1)
            grad[off[l] + cout * 9 * cin:off[l + 1]] += dY.reshape(-1, cout).sum(axis=0)
            if l > 0:
                dX = np.zeros_like(X)
                for k in range(9):
                    dX += _shift(dY, -(k // 3 - 1), -(k % 3 - 1)) @ W[:, k, :]
                dY = dX
    return L, grad
