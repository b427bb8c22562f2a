"""Plain FP64 definition of the learned mode-table surrogate.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: tests may import it,
the product path never does, and it shares no code with the CUDA library.

The paper tabulates its kernel exactly and has no learned model; this file
writes out, as plainly as numpy allows, the network the library's surrogate
evaluates, so that the CUDA forward pass, loss and gradients can be compared
with it element by element:

* ``features``  -- x = (ln(q r) / 4, d_x / r, d_y / r, ln(r) / 5) with
                   r = |d| and q = 2 pi k / (L c), the wavenumber of mode k of
                   the line DFT (Sec. 3.2, Eqs. 37-38).
* ``scale``     -- s(q, r) = exp(-q r) / (c sqrt(1 + q r)), zero beyond
                   q r = 16: the decay the line sum of the Green function
                   (Sec. 3.1, Eqs. 32-36) takes for k >= 1.
* ``forward``   -- y = W4^T h3 + b4 with h_l = silu(W_l^T h_{l-1} + b_l),
                   widths 4 -> H -> H -> H -> 6, parameters packed as
                   W1 [4][H], b1, W2 [H][H], b2, W3 [H][H], b3, W4 [H][6], b4.
* ``loss_grad`` -- loss = sum (y - t)^2 / (6 n) and its exact gradient by
                   the chain rule (pinned by central differences in
                   ``tests/test_oracle_mlp.py``).
* ``round_bf16`` -- float32 -> bfloat16 (round to nearest, ties to even) ->
                   float32, the rounding the inference weights get.
"""

from __future__ import annotations

import numpy as np

QR_CUT = 16.0


def n_params(H: int) -> int:
    return 4 * H + H + 2 * (H * H + H) + H * 6 + 6


def unpack(p: np.ndarray, H: int):
    """Weights and biases of the four layers, as views into ``p``."""
    p = np.asarray(p, dtype=np.float64)
    shapes = [(4, H), (H,), (H, H), (H,), (H, H), (H,), (H, 6), (6,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    assert o == p.size, (o, p.size)
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, H: int, x):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p, H)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1 + b1
    a1 = silu(z1)
    z2 = a1 @ W2 + b2
    a2 = silu(z2)
    z3 = a2 @ W3 + b3
    a3 = silu(z3)
    y = a3 @ W4 + b4
    return y, (x, z1, a1, z2, a2, z3, a3)


def loss_grad(p, H: int, x, t):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p, H)
    y, (x, z1, a1, z2, a2, z3, a3) = forward(p, H, x)
    t = np.asarray(t, dtype=np.float64)
    n = x.shape[0]
    diff = y - t
    loss = float(np.sum(diff * diff) / (6 * n))
    dy = 2.0 * diff / (6 * n)
    gW4, gb4 = a3.T @ dy, dy.sum(0)
    dz3 = (dy @ W4.T) * silu_grad(z3)
    gW3, gb3 = a2.T @ dz3, dz3.sum(0)
    dz2 = (dz3 @ W3.T) * silu_grad(z2)
    gW2, gb2 = a1.T @ dz2, dz2.sum(0)
    dz1 = (dz2 @ W2.T) * silu_grad(z1)
    gW1, gb1 = x.T @ dz1, dz1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])
    return loss, g


def round_bf16(a) -> np.ndarray:
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def features(d, k, L: int, c: float = 1.0) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64).reshape(-1, 2)
    k = np.asarray(k, dtype=np.float64).reshape(-1)
    r = np.hypot(d[:, 0], d[:, 1])
    qr = 2.0 * np.pi * k / (L * c) * r
    return np.stack([np.log(qr) / 4.0, d[:, 0] / r, d[:, 1] / r, np.log(r) / 5.0], axis=1)


def scale(d, k, L: int, c: float = 1.0) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64).reshape(-1, 2)
    k = np.asarray(k, dtype=np.float64).reshape(-1)
    qr = 2.0 * np.pi * k / (L * c) * np.hypot(d[:, 0], d[:, 1])
    return np.where(qr > QR_CUT, 0.0, np.exp(-np.minimum(qr, QR_CUT)) / (c * np.sqrt(1.0 + qr)))
