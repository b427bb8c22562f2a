"""Pins of the FP64 surrogate reference (``oracle/mlp.py``) on the CPU.

The gradient is checked against central finite differences of the loss in
FP64 (a dropped term, a transposed weight or a wrong activation derivative
each fail it), the BF16 rounding against hand-worked bit patterns, and the
features and scale against their definitions at special points.
"""

import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_central_differences():
    H, n = 8, 11
    rng = np.random.default_rng(5)
    p = rng.normal(0, 0.5, mlp.n_params(H))
    x = rng.normal(0, 1, (n, 4))
    t = rng.normal(0, 1, (n, 6))
    loss, g = mlp.loss_grad(p, H, x, t)
    assert g.shape == p.shape
    h = 1e-6
    num = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (mlp.loss_grad(p + e, H, x, t)[0] - mlp.loss_grad(p - e, H, x, t)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-8 * max(1.0, np.max(np.abs(g)))
    y, _ = mlp.forward(p, H, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)


def test_forward_of_a_hand_built_network():
    # W1 passes x0 through unit 0, later layers copy unit 0 forward: y_j = silu(silu(silu(x0))) * (j + 1) + j
    H = 8
    W1, b1, W2, b2, W3, b3, W4, b4 = (np.zeros(s) for s in [(4, H), (H,), (H, H), (H,), (H, H), (H,), (H, 6), (6,)])
    W1[0, 0] = 1.0
    W2[0, 0] = 1.0
    W3[0, 0] = 1.0
    W4[0, :] = np.arange(1, 7)
    b4[:] = np.arange(6)
    p = np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3, W4, b4)])
    x = np.array([[0.7, 5.0, -3.0, 2.0]])
    s = lambda z: z / (1 + np.exp(-z))
    y, _ = mlp.forward(p, H, x)
    np.testing.assert_allclose(y[0], s(s(s(0.7))) * np.arange(1, 7) + np.arange(6), rtol=1e-15)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, 1.0 + 2**-9, -2.5, 3.0e-3], dtype=np.float32)
    r = mlp.round_bf16(vals)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1; 1 + 3*2^-9 rounds up to 1 + 2^-7
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == np.float32(1.0 + 2**-7) and r[3] == 1.0 and r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2**-8
    assert (r.view(np.uint32) & 0xFFFF).max() == 0


def test_features_and_scale():
    d = np.array([[3, 4], [-8, 0]])
    k = np.array([2, 1])
    x = mlp.features(d, k, L=64, c=2.0)
    q0 = 2 * np.pi * 2 / (64 * 2.0) * 5
    np.testing.assert_allclose(x[0], [np.log(q0) / 4, 0.6, 0.8, np.log(5) / 5], rtol=1e-15)
    np.testing.assert_allclose(x[1, 1:], [-1.0, 0.0, np.log(8) / 5], rtol=1e-15)
    s = mlp.scale(d, k, L=64, c=2.0)
    assert s[0] == pytest.approx(np.exp(-q0) / (2.0 * np.sqrt(1 + q0)), rel=1e-15)
    assert mlp.scale([[100, 0]], [32], L=64)[0] == 0.0  # q r = 100 pi > 16
