"""The seeded synthetic workloads stand in for the paper's Table I style runs:
their sizes, wavelengths, radii, point counts, periods and parameter ranges
are pinned here, so that a change to a preset cannot silently change what the
benchmarks and parity tests measure."""
import math

import numpy as np

import workloads


def _on_grid(v, q=2.0 ** -10):
    return abs(v / q - round(v / q)) == 0.0


def test_cylinder_2d_workload():
    seen = set()
    for seed in range(1, 6):
        p = workloads.cylinder_2d(seed=seed)
        T = p["period"]
        assert p["dim"] == 2 and tuple(p["n"][:2]) == (128, 128) and p["wave_axis"] == 1
        assert p["wavelength"] == 64.0 and p["p_a"] == 1e-3 and p["radius"] == 8.0 and p["c0"] == 0.25
        assert p["cp"] == 1.5 * p["c0"] and p["n_surface"] == 64 and p["precision"] == "f64"
        assert p["n_steps"] == 20 * T and p["n_window"] == 5 * T and T == 256
        x, y = p["center"][:2]
        assert abs(x - 64.0) <= 0.5 and abs(y - 8.0) <= 0.5 and _on_grid(x) and _on_grid(y)
        seen.add((x, y))
    assert len(seen) == 5  # the seed draws the jitter


def test_sphere_3d_workload():
    kappas = set()
    for seed in range(1, 6):
        p = workloads.sphere_3d(seed=seed)
        T = p["period"]
        assert p["dim"] == 3 and tuple(p["n"]) == (256, 256, 256) and p["wave_axis"] == 2
        assert p["wavelength"] == 128.0 and p["radius"] == 16.0 and p["p_a"] == 1e-3
        assert p["center"] == (128.0, 128.0, 16.0) and p["n_surface"] == 2000 and p["precision"] == "f32"
        assert p["n_steps"] == 30 * T and p["n_window"] == 10 * T and T == 512
        assert 0.2 <= p["kappa"] <= 0.8 and math.isclose(p["cp"], p["c0"] / math.sqrt(p["kappa"]))
        assert math.isclose(2 * math.pi / p["wavelength"] * p["radius"], 0.785, abs_tol=1e-3)
        kappas.add(p["kappa"])
    assert len(kappas) == 5


def test_sphere_3d_large_sweep_positions():
    zs = []
    for j in range(16):
        p = workloads.sphere_3d_large(position=j)
        assert tuple(p["n"]) == (512, 512, 512) and p["wavelength"] == 256.0 and p["radius"] == 24.0
        assert p["n_surface"] == 4096 and p["kappa"] == 0.5
        z0 = p["center"][2]
        exact = j * math.pi / 15 * 256.0 / (2 * math.pi)
        assert _on_grid(z0) and 0.0 <= exact - z0 < 2.0 ** -10  # rounded down to the 2^-10 grid
        zs.append(z0)
    assert zs[0] == 0.0 and np.all(np.diff(zs) > 0) and 128.0 - zs[-1] <= 2.0 ** -10  # k z from 0 to pi


def test_ensembles():
    e3 = workloads.ensemble_3d(seed=1)
    assert len(e3) == 64 and {p["n"][0] for p in e3} == {96, 128, 160}
    for p in e3:
        edge = p["n"][0]
        assert tuple(p["n"]) == (edge, edge, edge) and p["wavelength"] == edge / 2
        assert 4.0 <= p["radius"] <= 12.0 and 0.0 <= p["kz"] <= math.pi and 0.8 <= p["c_ratio"] <= 2.0
        assert math.isclose(p["kappa"], 1.0 / p["c_ratio"] ** 2) and p["n_surface"] == 1000
        assert p["n_steps"] == 25 * p["period"] and p["n_window"] == 10 * p["period"]
    e2 = workloads.ensemble_2d(seed=1)
    assert len(e2) == 512
    assert all(tuple(p["n"][:2]) == (192, 192) and p["wavelength"] == 96.0 and p["dim"] == 2 for p in e2)


def test_surrogate_samples_are_a_latin_hypercube():
    n = 200
    u = np.array(workloads.latin_hypercube(n, 3, seed=7))
    assert u.shape == (n, 3) and np.all((u >= 0) & (u < 1))
    for a in range(3):
        assert sorted(np.floor(u[:, a] * n).astype(int)) == list(range(n))  # one per stratum
    probs = workloads.surrogate_problems(50, seed=3)
    box = workloads.SURROGATE_BOX
    for p in probs:
        ka, kz, kappa, c = p["features"]
        # k R is quantised with the radius (2^-10 cells), so it may sit a hair outside
        assert box["ka"][0] - 1e-3 <= ka <= box["ka"][1] + 1e-3
        assert box["kz"][0] <= kz <= box["kz"][1] and box["c_ratio"][0] <= c <= box["c_ratio"][1]
        assert math.isclose(kappa, 1.0 / c ** 2) and tuple(p["n"][:2]) == (192, 192)
