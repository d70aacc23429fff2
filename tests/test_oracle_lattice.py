"""Pins of the oracle's lattice Boltzmann step (Sec. V) against invariants and
closed forms that do not come from the oracle itself."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import theory


def _velocities(dim):
    v = [np.zeros(dim, dtype=int)]
    for a in range(dim):
        for s in (1, -1):
            e = np.zeros(dim, dtype=int)
            e[a] = s
            v.append(e)
    return np.array(v)


def _small(dim, cp=0.375, n=None):
    if n is None:
        n = (20, 18, 16) if dim == 3 else (24, 20)
    center = tuple(v / 2 + 0.25 for v in n[:dim])
    return workloads.problem(dim, n[:dim], dim - 1, float(n[dim - 1]), 3.0, center, cp=cp,
                             c0=0.25, n_surface=8, n_periods=1, n_avg_periods=1)


@pytest.mark.parametrize("dim", [2, 3])
def test_collision_conserves_moments_and_is_an_involution(dim):
    """Eq. (63) with tau = 1/2 keeps rho1 = sum f and J1 = sum v f (the moments of
    Eq. (71) equal those of f), so applying it twice returns the input."""
    p = _small(dim)
    c2 = oracle.sound_speed_sq(p)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((oracle.Q(p),) + oracle.shape(p)) * 1e-3
    g = oracle.collide(p, c2, f)
    r0, J0 = oracle.macroscopic(p, f)
    r1, J1 = oracle.macroscopic(p, g)
    assert np.abs(r1 - r0).max() <= 1e-17
    assert np.abs(J1 - J0).max() <= 1e-17
    h = oracle.collide(p, c2, g)
    assert np.abs(h - f).max() <= 1e-17
    # an equilibrium state is a fixed point
    e = oracle.initial_populations(p, c2)
    assert np.abs(oracle.collide(p, c2, e) - e).max() <= 1e-15 * np.abs(e).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_moments(dim):
    """Eq. (72) initial state: rho1 = p1/c^2, J1 = 0 and the momentum flux of
    Eq. (66) is diagonal with entries c^2 rho1 = p1 (Eq. 67)."""
    p = _small(dim)
    c2 = oracle.sound_speed_sq(p)
    f = oracle.initial_populations(p, c2)
    rho, J = oracle.macroscopic(p, f)
    s = np.arange(p["n"][dim - 1]) - p["antinode"]
    p_inc = p["p_a"] * np.cos(2 * math.pi * s / p["wavelength"])
    shp = [1, 1, 1]
    shp[2 - (dim - 1)] = -1
    p_inc = p_inc.reshape(shp) * np.ones(oracle.shape(p))
    assert np.allclose(rho * c2, p_inc, rtol=0, atol=1e-18)
    assert np.abs(J).max() == 0.0
    V = _velocities(dim)
    for a in range(dim):
        for b in range(dim):
            Pi = sum(V[i, a] * V[i, b] * f[i] for i in range(len(V)))
            want = c2 * rho if a == b else 0.0
            assert np.allclose(Pi, want, rtol=0, atol=1e-18)


@pytest.mark.parametrize("dim", [2, 3])
def test_advection_moves_each_population_by_its_velocity(dim):
    """Eq. (64), periodic: a lone value of population i at x arrives at x + v_i."""
    p = _small(dim)
    shp = oracle.shape(p)
    V = _velocities(dim)
    corner = (0,) * 3  # exercises the wrap on every axis
    for i in range(oracle.Q(p)):
        f = np.zeros((oracle.Q(p),) + shp)
        f[(i,) + corner] = 1.0
        g = oracle.advect(p, f)
        # array order is (z, y, x)
        target = [0, 0, 0]
        for a in range(dim):
            target[2 - a] = V[i, a] % p["n"][a]
        assert g[(i,) + tuple(target)] == 1.0
        assert g.sum() == 1.0


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 2)])
def test_uniform_medium_follows_closed_form_mode(dim, axis):
    """With c = c0 everywhere the standing wave of Eq. (38) evolves as one mode of
    the scheme: p1(x, t) = p_a cos(k s) cos(w t), sin^2(w/2) = c^2 sin^2(k/2).
    The equilibrium initial state excites no other eigenmode."""
    n = [24, 20, 16][:dim]
    lam = 16.0 if axis != 1 else 20.0
    n[axis] = int(lam) * (2 if axis == 0 else 1)
    center = tuple(v / 2 for v in n)
    p = workloads.problem(dim, n, axis, lam, 2.0, center, cp=0.25, c0=0.25, n_surface=0,
                          n_periods=3, n_avg_periods=0)
    p["antinode"] = 3.0
    out = oracle.run(p, fields=True)
    k = 2 * math.pi / lam
    kv = [0.0] * dim
    kv[axis] = k
    w = theory.lattice_omega(kv, 0.0625)
    s = np.arange(n[axis]) - p["antinode"]
    shp = [1, 1, 1]
    shp[2 - axis] = -1
    want = p["p_a"] * np.cos(k * s).reshape(shp) * math.cos(w * p["n_steps"]) * np.ones(oracle.shape(p))
    assert np.abs(out["p1"] - want).max() <= 1e-14 * p["p_a"]


def test_lattice_sound_speed_limit():
    """The dispersion of the scheme tends to w = c k for long waves (Eq. 68)."""
    c2 = 0.0625
    for lam in (64, 256, 1024):
        k = 2 * math.pi / lam
        w = theory.lattice_omega([k], c2)
        assert abs(w / k - 0.25) < 0.25 * (k * k / 6 + 1e-12)
    assert theory.lattice_omega([2 * math.pi / 128, 0, 0], 0.0625) == pytest.approx(
        theory.lattice_omega([2 * math.pi / 128], 0.0625), rel=1e-15)


def test_velocity_set_moment_conditions():
    """Eqs. (69)-(70) with the c_s^2 printed after Eq. (71): the weights the
    oracle's equilibrium implies satisfy the moment conditions."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    for dim, key in ((2, "D2Q5_cs2"), (3, "D3Q7_cs2")):
        cs2 = gold["velocity_sets"][key]
        # weights from the equilibrium of a unit-density rest state with c^2 = c_s^2:
        # f^eq_i = w_i exactly when c^2 = c_s^2 (Eq. 71)
        p = _small(dim, cp=0.25)
        V = _velocities(dim)
        f = np.zeros((oracle.Q(p),) + oracle.shape(p))
        c2 = np.full(oracle.shape(p), cs2)
        # collide a state with rho1 = 1, J1 = 0 concentrated in the rest population
        f[0] = 1.0
        w = oracle.collide(p, c2, f)  # = 2 f^eq - f
        weq = (w + f)[:, 0, 0, 0] / 2.0
        assert weq.sum() == pytest.approx(1.0, abs=1e-15)
        for a in range(dim):
            assert (weq * V[:, a]).sum() == pytest.approx(0.0, abs=1e-15)
            for b in range(dim):
                m2 = (weq * V[:, a] * V[:, b]).sum()
                assert m2 == pytest.approx(cs2 if a == b else 0.0, abs=1e-15)
