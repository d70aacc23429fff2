"""Pins of the oracle's driven cavity (Sec. VII): damped bounce-back walls
(Eq. 73), the source sheet imposing fields (Eq. 72), and the cavity of the
paper's results section reproducing Wei's force at steady state."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import theory


def _cavity(n=(12, 16), lam=16.0, amp=0.0, phi=0.9, R=1.0, s0=8.0, periods=1, avg=0, N=0, cp=0.25):
    p = workloads.problem(2, n, 1, lam, R, (n[0] / 2, s0), cp=cp, n_surface=N, n_periods=periods,
                          n_avg_periods=avg, interface_d=0.25)
    p.update(boundary="driven", wall_damping=phi, source_amplitude=amp)
    return p


def test_walls_bounce_back_damped_and_drop_outward():
    p = _cavity()
    shp = oracle.shape(p)
    c2 = oracle.sound_speed_sq(p)
    ny = p["n"][1]
    f = np.zeros((5,) + shp)
    f[4, 0, 0, 3] = 1.0       # -y arriving at the low wall
    f[3, 0, ny - 1, 7] = 2.0  # +y arriving at the high wall
    f[1, 0, 0, 5] = 3.0       # +x arriving at the low wall
    g = oracle.apply_boundaries(p, c2, f, np.full_like(f, 7.0), 0)
    assert g[3, 0, 0, 3] == pytest.approx(0.9)        # reflected into the domain
    assert g[4, 0, 0, 3] == 0.0                       # outward value dropped
    assert g[4, 0, ny - 1, 7] == pytest.approx(1.8)
    assert g[3, 0, ny - 1, 7] == 0.0
    assert g[2, 0, 0, 5] == pytest.approx(2.7)        # lateral directions reversed too
    assert np.all(g[:, 0, 2:ny - 1, :] == 7.0)       # interior untouched


def test_source_sheet_imposes_the_equilibrium():
    p = _cavity(amp=2e-3)
    T = p["period"]
    c2 = oracle.sound_speed_sq(p)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((5,) + oracle.shape(p)) * 1e-3
    for t in (0, 3, T + 5):
        g = oracle.apply_boundaries(p, c2, f, np.zeros_like(f), t)
        rho_src = 2e-3 * math.sin(2 * math.pi * (t % T) / T)
        sheet = g[:, 0, 1, :]
        assert np.allclose(sheet.sum(0), rho_src, rtol=0, atol=1e-18)
        Jx = f[1, 0, 1, :] - f[2, 0, 1, :]
        Jy = f[3, 0, 1, :] - f[4, 0, 1, :]
        assert np.allclose(sheet[1] - sheet[2], Jx, rtol=0, atol=1e-18)
        assert np.allclose(sheet[3] - sheet[4], Jy, rtol=0, atol=1e-18)
        assert np.allclose(sheet[1] + sheet[2], 0.0625 * rho_src, rtol=0, atol=1e-18)  # Pi_xx = c^2 rho


def test_cavity_of_the_results_section_reproduces_wei():
    """Sec. VII: box lambda/2 + 3 cells along the wave (lambda = 400), 64-cell
    periodic lateral box, source at s = 1, damped walls (Phi = 0.99): a standing
    wave of amplitude rho_a c0^2 with its node at L/2 + 1; a cylinder at lambda/8
    from the source-side antinode feels Wei's force at steady state, and none at
    the node."""
    lam, lat = 400.0, 64
    L = int(lam / 2 + 3)
    p_a = 1e-3

    def run(s0, cp, periods=12, avg=4):
        p = workloads.problem(2, (lat, L), 1, lam, 8.0, (lat / 2, s0), cp=cp, n_surface=64,
                              n_periods=periods, n_avg_periods=avg, surface_radius=10.0)
        p.update(boundary="driven", wall_damping=0.99, source_amplitude=p_a / 0.0625)
        return p

    wei = theory.wei_force_2d(8.0, p_a, lam, lam / 8, 0.25, 0.375)
    F = oracle.run(run(2 + lam / 8, 0.375))["force"][1]
    assert abs(F / wei - 1) < 0.03
    Fn = oracle.run(run(L / 2 + 0.5, 0.375))["force"][1]
    assert abs(Fn) < 0.03 * abs(F)
    # empty cavity: envelope of p1 over one period after 8 periods
    p = run(L / 2, 0.25, periods=1, avg=0)
    c2 = oracle.sound_speed_sq(p)
    f = oracle.run(dict(p, n_steps=8 * p["period"]), populations=True)["f"]
    env = np.zeros(L)
    for t in range(p["period"]):
        g = oracle.collide(p, c2, f)
        g = oracle.apply_boundaries(p, c2, f, g, 8 * p["period"] + t)
        f = oracle.advect(p, g)
        rho, _ = oracle.macroscopic(p, f)
        env = np.maximum(env, np.abs(rho[0, :, lat // 2]) * 0.0625)
    assert abs(env[2:].max() / p_a - 1) < 0.02
    node = 2 + int(np.argmin(env[2:L - 1]))
    assert abs(node - (L / 2 + 1)) <= 1.5
