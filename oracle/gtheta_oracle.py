"""CPU oracle of the learned coarse propagator G_theta (numpy, FP64). TEST INFRASTRUCTURE ONLY.

G_theta(U) = U + R(U): R is six 3x3 convolutions with zero padding (the field is zero outside
the interior grid, as u = 0 on the boundary of Section 2.1), channels 1 -> 32 -> 32 -> 32 -> 32 ->
32 -> 1, ReLU after the first five. The paper has no learned propagator; this network replaces
the plain coarse step of Eq. 2.2 and is trained on pairs (U(t), U(t + Delta T)) of the fine
solver. Fields are [H][W] arrays, activations [H][W][C] (channels last).

Weights: W[l] has shape [3][3][Cout][Cin] (tap (dy, dx) in 0..2 for offsets -1..1), b[l] [Cout].

Functions: ``forward`` (with the activations for backpropagation), ``backward`` (gradients of a
scalar loss through all layers), ``mse_crop_loss`` (mean squared error over a central window),
``adam_step`` (Kingma and Ba, 2015, with bias correction). Pinned in tests/test_oracle_gtheta.py
by central finite differences of the loss in every layer, by the convolution of a delta image,
and by the shift structure of zero padding.

Storage precision. The network is specified with BF16 weights and activations and FP32
accumulation. ``forward(..., bf16=True)`` / ``backward(..., bf16=True)`` evaluate that storage
model in FP64 arithmetic: the hidden activations a1..a5, the weights of the four 32 -> 32 layers
and the hidden-layer gradients are rounded to BF16 (round to nearest, ties to even) where they
are stored; the input, the first and last layers' weights, R and dLoss/dR stay unrounded.
``bf16_round`` is pinned against torch's own float32 -> bfloat16 conversion.
"""
from __future__ import annotations

import numpy as np

CHANNELS = [1, 32, 32, 32, 32, 32, 1]


def init_params(seed: int = 0, scale_last: float = 0.1):
    """He-normal weights from a seeded numpy generator (training initialisation only)."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for l in range(6):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        std = np.sqrt(2.0 / (9 * cin))
        w = rng.standard_normal((3, 3, cout, cin)) * std
        if l == 5:
            w *= scale_last
        W.append(w)
        b.append(np.zeros(cout))
    return W, b


def conv3(x: np.ndarray, w: np.ndarray, bias: np.ndarray) -> np.ndarray:
    """y[i,j,co] = b[co] + sum_{dy,dx,ci} w[dy,dx,co,ci] x[i+dy-1, j+dx-1, ci] (zero outside)."""
    H, Wd, _ = x.shape
    xp = np.zeros((H + 2, Wd + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    y = np.zeros((H, Wd, w.shape[2])) + bias
    for dy in range(3):
        for dx in range(3):
            y += xp[dy:dy + H, dx:dx + Wd] @ w[dy, dx].T
    return y


def conv3_backward(x: np.ndarray, w: np.ndarray, gy: np.ndarray):
    """Gradients of conv3 w.r.t. x, w and b for the output gradient gy."""
    H, Wd, _ = x.shape
    xp = np.zeros((H + 2, Wd + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            patch = xp[dy:dy + H, dx:dx + Wd]
            gw[dy, dx] = np.einsum("ijo,ijc->oc", gy, patch)
            gxp[dy:dy + H, dx:dx + Wd] += gy @ w[dy, dx]
    return gxp[1:-1, 1:-1], gw, gy.sum(axis=(0, 1))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Nearest BF16 value (ties to even) of each entry, returned as float64. BF16 keeps the top
    16 bits of the IEEE float32 pattern; the input is first rounded to float32."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def _stored_weights(W, bf16: bool):
    return [bf16_round(w) if (bf16 and 0 < l < 5) else w for l, w in enumerate(W)]


def forward(u: np.ndarray, W, b, bf16: bool = False):
    """Returns (G(U), [a0, a1, ..., a6]) with a0 = U[..., None] and a6 = R(U)."""
    Ws = _stored_weights(W, bf16)
    a = [u[..., None].astype(np.float64)]
    for l in range(6):
        z = conv3(a[-1], Ws[l], b[l])
        if l < 5:
            z = np.maximum(z, 0.0)
            if bf16:
                z = bf16_round(z)
        a.append(z)
    return u + a[-1][..., 0], a


def backward(acts, W, grad_r: np.ndarray, bf16: bool = False):
    """Gradients of a loss with dLoss/dR = grad_r ([H][W]) through the six layers."""
    Ws = _stored_weights(W, bf16)
    gW, gb = [None] * 6, [None] * 6
    g = grad_r[..., None]
    for l in range(5, -1, -1):
        gx, gW[l], gb[l] = conv3_backward(acts[l], Ws[l], g)
        if l > 0:
            g = gx * (acts[l] > 0)  # ReLU of layer l (activation a_l = relu(z_l))
            if bf16:
                g = bf16_round(g)
    return gW, gb


def mse_crop_loss(r: np.ndarray, target: np.ndarray, margin: int, relative: bool = False):
    """Mean of (r - target)^2 over the window [margin, H - margin) x [margin, W - margin); the
    gradient with respect to r is zero outside it. relative: the sum of (r - target)^2 over the
    window divided by E = sum of target^2 there + 1e-12 per window pixel (one crop's relative
    squared error; a batch's loss is the mean of its crops')."""
    H, Wd = r.shape
    m = np.zeros_like(r)
    m[margin:H - margin, margin:Wd - margin] = 1.0
    cnt = m.sum()
    d = (r - target) * m
    if relative:
        e = float((target * target * m).sum()) + 1e-12 * cnt
        return float((d * d).sum() / e), 2.0 * d / e
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (in place on p, m, v) with bias correction at step t (1-based)."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p -= lr * mh / (np.sqrt(vh) + eps)
