"""FP64 reference of the surrogate network (test infrastructure only).

MLP 4 -> 256 -> 256 -> 256 -> 1 with GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2
on the hidden layers, a linear output and the mean-squared-error loss
L = mean_b (y_b - t_b)^2.  Inputs are normalised to [-1, 1] by the training box
[lo, hi] before the first layer.  Backpropagation written out layer by layer;
pinned by central finite differences in tests/test_oracle_mlp.py.

Parameter vector (the library's packed layout): W1 (256 x 4), b1 (256),
W2 (256 x 256), b2 (256), W3 (256 x 256), b3 (256), W4 (1 x 256), b4 (1),
each matrix row-major [out][in].
"""
import math

import numpy as np

IN, HID = 4, 256
SHAPES = [(HID, IN), (HID,), (HID, HID), (HID,), (HID, HID), (HID,), (1, HID), (1,)]
SIZE = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])


def normalise(x, lo, hi):
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * (x - lo) / (hi - lo) - 1.0


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, xn, act_round=None):
    """xn: normalised inputs (B, 4).  Returns y (B,) and the cache.
    act_round: None for FP64 activations, or a rounding applied to every
    hidden activation (``bf16``: the network with BF16 activations, as the
    surrogate's specification states them; products and sums stay FP64)."""
    r = (lambda h: h) if act_round is None else act_round
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    z1 = xn @ W1.T + b1
    h1 = r(gelu(z1))
    z2 = h1 @ W2.T + b2
    h2 = r(gelu(z2))
    z3 = h2 @ W3.T + b3
    h3 = r(gelu(z3))
    y = (h3 @ W4.T + b4)[:, 0]
    return y, (xn, z1, h1, z2, h2, z3, h3)


def loss_and_grad(theta, xn, t):
    """MSE loss and its gradient with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    y, (x0, z1, h1, z2, h2, z3, h3) = forward(theta, xn)
    B = y.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(d * d))
    dy = (2.0 / B) * d[:, None]                 # dL/dy, (B, 1)
    gW4 = dy.T @ h3
    gb4 = dy.sum(0)
    dz3 = (dy @ W4) * gelu_grad(z3)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ x0
    gb1 = dz1.sum(0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


def init(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (numpy RNG)."""
    rng = np.random.default_rng(seed)
    out = []
    fans = [IN, IN, HID, HID, HID, HID, HID, HID]
    for s, fan in zip(SHAPES, fans):
        a = 1.0 / math.sqrt(fan)
        out.append(rng.uniform(-a, a, size=s))
    return pack(out)


def bf16(x):
    """Round FP64/FP32 values to bfloat16 (round to nearest even), as floats."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
