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
