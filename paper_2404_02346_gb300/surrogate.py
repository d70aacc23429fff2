"""Learned surrogate of the radiation force, trained on the batched lattice runs.

Orchestration over the C ABI only: the lattice forces come from the batched
kernels (wlb_batch_*), the network runs on the tensor-core kernels (wlb_mlp_*).
Features are (k R_p, k z0, kappa~, c~); the target is the force along the wave
divided by the 2D force scale F0 = pi R^2 p_a^2 k / (4 rho0 c0^2), so that
Wei's closed form reads (1 - kappa~) sin(2 k z0).  Queries outside the training
box are answered by the lattice method itself.
"""
import math

import numpy as np

from . import Batch, MLP


def force_scale(prob):
    k = 2.0 * math.pi / prob["wavelength"]
    return math.pi * prob["radius"] ** 2 * prob["p_a"] ** 2 * k / (4.0 * prob["rho0"] * prob["c0"] ** 2)


def lattice_targets(problems, chunk=512, stream=None):
    """Normalised forces of the problems, computed by the batched lattice
    kernels in chunks of `chunk` lattices."""
    out = np.zeros(len(problems))
    ax = problems[0]["wave_axis"]
    for i in range(0, len(problems), chunk):
        part = problems[i:i + chunk]
        with Batch(part, stream=stream) as b:
            F = b.run()
        out[i:i + len(part)] = [F[j, ax] / force_scale(p) for j, p in enumerate(part)]
    return out


class Surrogate:
    """Tensor-core MLP over the features, with lattice fallback outside the box."""

    def __init__(self, box, batch_max=65536, stream=None):
        (a0, a1), (z0, z1), (c0, c1) = box["ka"], box["kz"], box["c_ratio"]
        self.lo = np.array([a0, z0, 1.0 / c1 ** 2, c0], dtype=np.float32)
        self.hi = np.array([a1, z1, 1.0 / c0 ** 2, c1], dtype=np.float32)
        self.net = MLP(self.lo, self.hi, batch_max=batch_max, stream=stream)
        self.stream = stream

    def fit(self, features, targets, epochs, batch=512, lr=2e-3, lr_final=2e-5, seed=1):
        import torch
        x = torch.tensor(np.asarray(features, dtype=np.float32), device="cuda")
        t = torch.tensor(np.asarray(targets, dtype=np.float32), device="cuda")
        self.net.init_weights(seed)
        return self.net.train(x, t, epochs=epochs, batch=batch, lr=lr, lr_final=lr_final, seed=seed)

    def predict(self, features):
        """Network outputs and inside-the-box flags (torch CUDA tensors)."""
        import torch
        x = features if hasattr(features, "data_ptr") else torch.tensor(
            np.asarray(features, dtype=np.float32), device="cuda")
        return self.net.predict(x)

    def normalised_forces(self, problems):
        """Normalised force for each problem: the network inside the box, the
        batched lattice method outside.  Returns (values, used_lattice)."""
        feats = np.array([p["features"] for p in problems], dtype=np.float32)
        y, inside = self.predict(feats)
        y = y.cpu().numpy().astype(np.float64)
        inside = inside.cpu().numpy().astype(bool)
        out = ~inside
        if out.any():
            y[out] = lattice_targets([p for p, o in zip(problems, out) if o], stream=self.stream)
        return y, out

    def close(self):
        self.net.close()
