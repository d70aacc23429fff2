"""Surrogate network on the tensor cores (wlb_mlp_*) against the FP64 oracle
network: forward values and backpropagated gradients for the same BF16-rounded
weights and inputs, and training on a smooth target."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu

LO = np.array([0.1, 0.0, 0.2, 0.8])
HI = np.array([1.2, np.pi, 1.6, 2.0])


@pytest.fixture(scope="module")
def wlb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2404_02346_gb300 import build as B
    B.build()
    import paper_2404_02346_gb300 as W
    W.lib()
    return W


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    return LO + (HI - LO) * rng.uniform(size=(n, 4))


def _bf16_theta(theta):
    return ref.bf16(theta)


def _gpu_theta(theta):
    """The parameters the GPU network computes with: BF16 weight matrices, FP32
    biases (added in the FP32 epilogue)."""
    return ref.pack([ref.bf16(p) if p.ndim == 2 else p.astype(np.float32).astype(np.float64)
                     for p in ref.unpack(theta)])


def test_forward_matches_oracle(wlb):
    import torch
    net = wlb.MLP(LO, HI, batch_max=1024)
    net.init_weights(11)
    w = net.get_weights().astype(np.float64)
    x = _inputs(1000, 1)  # 1000 queries: a ragged last tile of 128 rows
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    y, inside = net.predict(xt)
    y = y.cpu().numpy().astype(np.float64)
    assert inside.cpu().numpy().all()
    xn = ref.bf16(ref.normalise(x.astype(np.float32).astype(np.float64), LO.astype(np.float32), HI.astype(np.float32)))
    # the network as specified: BF16 weights, inputs and activations, FP32
    # biases; the GPU accumulates in FP32 and evaluates GELU with a 1.5e-7 erf,
    # so only activations within that distance of a BF16 rounding boundary can
    # round the other way (each such flip moves one activation by 2^-8 of
    # itself): most queries agree to FP32 rounding, a few by such flips
    y_ref, _ = ref.forward(_gpu_theta(w), xn, act_round=ref.bf16)
    scale = np.abs(y_ref).max()
    err = np.abs(y - y_ref)
    assert np.median(err) <= 1e-4 * scale, (np.median(err), scale)
    assert err.max() <= 5e-3 * scale, (err.max(), scale)
    # against the FP64-activation network: the BF16 activations' own effect
    y_64, _ = ref.forward(_gpu_theta(w), xn)
    assert np.abs(y - y_64).max() <= 2e-2 * scale, (np.abs(y - y_64).max(), scale)
    # outside the box: flagged
    xo = x[:4].copy()
    xo[0, 0] = 5.0
    xo[1, 3] = 0.1
    _, ins = net.predict(torch.tensor(xo, dtype=torch.float32, device="cuda"))
    assert list(ins.cpu().numpy()) == [0, 0, 1, 1]
    net.close()


def test_fused_forward_bit_identical_to_layer_by_layer(wlb):
    """The one-launch fused forward (activations kept on the chip, weights
    streamed) against the layer-by-layer GEMM launches: the same products,
    epilogues and roundings, hence the same bits.  One query, a ragged single
    tile, several tiles per CTA with a ragged end, queries outside the box,
    again after training changed the weights (the stream is repacked), and
    n = 0."""
    import torch
    net = wlb.MLP(LO, HI, batch_max=4096)
    net.init_weights(11)

    def both(x):
        xt = torch.tensor(x, dtype=torch.float32, device="cuda")
        net.set_fused(True)
        yf, inf = net.predict(xt)
        net.set_fused(False)
        yl, inl = net.predict(xt)
        net.set_fused(True)
        return yf, inf, yl, inl

    for n, seed in [(1, 5), (1000, 1), (300_001, 2)]:
        x = _inputs(n, seed)
        x[3::7, 0] = 5.0
        x[5::11, 3] = 0.1
        yf, inf, yl, inl = both(x)
        assert torch.equal(yf, yl), (n, (yf - yl).abs().max().item())
        assert torch.equal(inf, inl), n
        assert torch.isfinite(yf).all()
    x = _inputs(4096, 8)
    t = torch.tensor(np.sin(2 * x[:, 1]), dtype=torch.float32, device="cuda")
    y0, _, _, _ = both(x)
    net.train(torch.tensor(x, dtype=torch.float32, device="cuda"), t, epochs=2, batch=512, lr=2e-3, lr_final=1e-3)
    yf, inf, yl, inl = both(x)
    assert torch.equal(yf, yl) and torch.equal(inf, inl)
    assert not torch.equal(yf, y0)
    y, ins = net.predict(torch.empty((0, 4), dtype=torch.float32, device="cuda"))
    assert y.numel() == 0 and ins.numel() == 0
    assert wlb.lib().wlb_mlp_set_fused(net._h, 2) == wlb.WLB_ERR_ARG
    net.close()


def test_gradients_match_oracle(wlb):
    """Loss and gradients of a 384-sample batch (three 128-row tiles) against
    FP64 backpropagation with the same BF16 weights and inputs; the GPU keeps
    activations and activation gradients in BF16, hence the per-block bound."""
    import torch
    net = wlb.MLP(LO, HI, batch_max=512)
    net.init_weights(5)
    w = net.get_weights().astype(np.float64)
    x = _inputs(384, 2)
    rng = np.random.default_rng(3)
    t = rng.standard_normal(384) * 0.5
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    loss, g = net.loss_grad(xt, tt)
    xn = ref.bf16(ref.normalise(x.astype(np.float32).astype(np.float64), LO.astype(np.float32), HI.astype(np.float32)))
    loss_ref, g_ref = ref.loss_and_grad(_bf16_theta(w), xn, t.astype(np.float32).astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    parts, parts_ref = ref.unpack(g.astype(np.float64)), ref.unpack(g_ref)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"], parts, parts_ref):
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert err < 5e-2, (name, err)
    net.close()


def test_training_fits_a_smooth_target(wlb):
    import torch
    x = _inputs(8192, 4)
    t = np.sin(2 * x[:, 1]) * (1 - 1 / x[:, 3] ** 2) + 0.3 * x[:, 0]
    net = wlb.MLP(LO, HI, batch_max=512)
    net.init_weights(1)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    hist = net.train(xt, tt, epochs=40, batch=512, lr=2e-3, lr_final=1e-4, seed=9)
    assert hist[-1] < 0.05 * hist[0]
    y, _ = net.predict(xt)
    rms = float(np.sqrt(np.mean((y.cpu().numpy() - t) ** 2)))
    assert rms < 0.05 * float(np.std(t)) + 0.02
    net.close()
