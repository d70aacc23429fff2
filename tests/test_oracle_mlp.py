"""Pins of the FP64 surrogate-network reference: backpropagation against
central finite differences, GELU against its integral definition, and the
bfloat16 rounding against torch's conversion."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_definition_and_derivative():
    from scipy.stats import norm
    z = np.linspace(-6, 6, 241)
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), rtol=0, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(2)
    theta = mlp.init(7)
    x = rng.uniform(-1, 1, size=(6, 4))
    t = rng.standard_normal(6)
    loss, g = mlp.loss_and_grad(theta, x, t)
    # every bias and a spread of weights, central differences in FP64
    idx = list(range(0, mlp.SIZE, 997)) + [1024 + 5, 1024 + 256 + 65536 + 3, mlp.SIZE - 1, mlp.SIZE - 2]
    for i in idx:
        h = 1e-6
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        lp, _ = mlp.loss_and_grad(tp, x, t)
        lm, _ = mlp.loss_and_grad(tm, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
    assert loss == pytest.approx(float(np.mean((mlp.forward(theta, x)[0] - t) ** 2)), rel=1e-15)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 3.0e38]])
    ours = mlp.bf16(v)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_packed_layout():
    theta = np.arange(mlp.SIZE, dtype=np.float64)
    parts = mlp.unpack(theta)
    assert [p.shape for p in parts] == mlp.SHAPES
    assert np.array_equal(mlp.pack(parts), theta)
    assert mlp.SIZE == 256 * 4 + 256 + 2 * (256 * 256 + 256) + 256 + 1


def test_bf16_activations_option():
    """forward(..., act_round=bf16): every hidden activation is the BF16
    rounding of the exact GELU of its FP64 pre-activation (which sees the
    rounded activations of the layer below); without rounding it is the FP64
    network, and the BF16 network's output stays within the rounding's reach."""
    rng = np.random.default_rng(6)
    theta = mlp.init(3)
    x = rng.uniform(-1, 1, size=(64, 4))
    y64, _ = mlp.forward(theta, x)
    assert np.array_equal(mlp.forward(theta, x, act_round=None)[0], y64)
    y16, (x0, z1, h1, z2, h2, z3, h3) = mlp.forward(theta, x, act_round=mlp.bf16)
    W1, b1, W2, b2, W3, b3, W4, b4 = mlp.unpack(theta)
    assert np.array_equal(h1, mlp.bf16(mlp.gelu(x @ W1.T + b1)))
    assert np.array_equal(h2, mlp.bf16(mlp.gelu(h1 @ W2.T + b2)))
    assert np.array_equal(h3, mlp.bf16(mlp.gelu(h2 @ W3.T + b3)))
    assert np.array_equal(y16, (h3 @ W4.T + b4)[:, 0])
    assert np.all(mlp.bf16(h3) == h3)
    # each activation moves by at most 2^-9 of itself; the output by a few 1e-3
    assert 0 < np.abs(y16 - y64).max() < 1e-2 * np.abs(y64).max()
