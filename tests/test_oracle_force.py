"""Pins of the oracle's force functional, Eq. (14), against the divergence
theorem and exact symmetries."""
import math

import numpy as np
import pytest

import oracle
import workloads


def _surface(dim, N, Rs, center):
    n = (64, 64, 64)[:dim]
    p = workloads.problem(dim, n, dim - 1, 64.0, Rs - 2, center, cp=0.375, n_surface=N,
                          n_periods=1, n_avg_periods=1, surface_radius=Rs)
    return p, oracle.surface_points(p)


CASES = [(2, 4096, 9.0, (30.5, 33.25)), (3, 40000, 12.0, (31.0, 33.5, 29.75))]


@pytest.mark.parametrize("dim,N,Rs,center", CASES)
def test_pressure_term_divergence_theorem(dim, N, Rs, center):
    """<p1^2> = a^2 x^2 and u1 = 0 on the surface: Eq. (14) equals
    -int d_x(a^2 x^2)/(2 rho0 c0^2) dV = -a^2 x_c V/(rho0 c0^2) along x and 0 else."""
    p, pts = _surface(dim, N, Rs, center)
    a, rho0, c0, nw = 3e-4, 1.3, 0.25, 7.0
    x = pts[:, 0]
    Spp = nw * a * a * x * x
    F = oracle.force(dim, pts, Spp, np.zeros(N), np.zeros((N, 3)), nw, rho0, c0)
    V = math.pi * Rs ** 2 if dim == 2 else 4 / 3 * math.pi * Rs ** 3
    want = -a * a * center[0] * V / (rho0 * c0 * c0)
    assert F[0] == pytest.approx(want, rel=2e-4)
    assert np.all(np.abs(F[1:dim]) < 2e-4 * abs(want))
    # same along the second axis (exercises the y components)
    y = pts[:, 1]
    F = oracle.force(dim, pts, nw * a * a * y * y, np.zeros(N), np.zeros((N, 3)), nw, rho0, c0)
    want = -a * a * center[1] * V / (rho0 * c0 * c0)
    assert F[1] == pytest.approx(want, rel=2e-4)
    assert abs(F[0]) < 2e-4 * abs(want)


@pytest.mark.parametrize("dim,N,Rs,center", CASES)
def test_velocity_terms_divergence_theorem(dim, N, Rs, center):
    """u1 = (b x, 0, 0): the tensor -rho0 u^2/2 I + rho0 u u of Eq. (14) has
    divergence (rho0 b^2 x, 0, 0), so F = (-rho0 b^2 x_c V, 0, 0)."""
    p, pts = _surface(dim, N, Rs, center)
    b, rho0, c0, nw = 2e-3, 0.9, 0.25, 3.0
    x = pts[:, 0]
    u = b * x
    Suu = nw * u * u
    Snu = np.zeros((N, 3))
    Snu[:, 0] = nw * u * (u * pts[:, 3])
    F = oracle.force(dim, pts, np.zeros(N), Suu, Snu, nw, rho0, c0)
    V = math.pi * Rs ** 2 if dim == 2 else 4 / 3 * math.pi * Rs ** 3
    want = -rho0 * b * b * center[0] * V
    assert F[0] == pytest.approx(want, rel=2e-4)
    assert np.all(np.abs(F[1:dim]) < 2e-4 * abs(want))


def test_uniform_fields_give_zero_force():
    """Constant <p1^2>, <u1^2> and <u1 (u1.n)> from a constant u1: the closed
    surface integral vanishes (2D arcs: to rounding; 3D Fibonacci: to the
    quadrature residual sum n dS)."""
    for dim, N in ((2, 64), (3, 2000)):
        p, pts = _surface(dim, N, 8.0, (32.0, 32.0, 32.0)[:dim])
        P0, u0 = 1e-3, np.array([3e-3, -2e-3, 1e-3])[:3]
        Snu = np.outer(pts[:, 3:6] @ u0, u0)
        F = oracle.force(dim, pts, np.full(N, P0 * P0), np.full(N, u0 @ u0), Snu, 1.0, 1.0, 0.25)
        scale = P0 * P0 / (2 * 0.0625) * 2 * math.pi * 8.0 * (1 if dim == 2 else 8.0 * 2)
        if dim == 2:
            assert np.abs(F).max() < 1e-15 * scale
        else:
            resid = np.abs((pts[:, 3:6] * pts[:, 6:7]).sum(0)).max() / (4 * math.pi * 64)
            assert np.abs(F).max() < 4 * resid * scale + 1e-18


def test_pressure_amplitude_scaling_is_exact():
    """Doubling p_a doubles every population exactly (the scheme is linear and a
    power-of-two scale commutes with rounding), so the force scales by exactly 4;
    the paper measures an exponent of 1.9999 (Table II) and 1.9994 (Table III)."""
    base = workloads.problem(2, (48, 32), 1, 32.0, 4.0, (24.0, 4.5), cp=0.375, n_surface=32,
                             n_periods=2, n_avg_periods=1)
    F1 = oracle.run(base)["force"]
    dbl = dict(base, p_a=2 * base["p_a"])
    F2 = oracle.run(dbl)["force"]
    assert np.array_equal(F2, 4 * F1)
    tri = dict(base, p_a=3 * base["p_a"])
    F3 = oracle.run(tri)["force"]
    assert F3[1] == pytest.approx(9 * F1[1], rel=1e-12)
    assert abs(F3[0] - 9 * F1[0]) < 1e-12 * abs(F3[1])  # lateral: rounding noise only
    assert abs(F1[1]) > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_window_samples_the_last_steps(dim):
    """The averaged steps are the last n_window of n_steps (Sec. VII: average
    once the signal is established), each sampled before its collision; the
    fields after the run are those at t = n_steps."""
    n = (24, 20, 16)[:dim]
    lam = float(n[dim - 1])
    p = workloads.problem(dim, n, dim - 1, lam, 3.0, tuple(v / 2 + 0.25 for v in n), cp=0.4,
                          n_surface=12, n_periods=1, n_avg_periods=1)
    p["n_steps"], p["n_window"] = 9, 3
    out = oracle.run(p, fields=True, populations=True)
    c2 = oracle.sound_speed_sq(p)
    f = oracle.initial_populations(p, c2)
    pts = oracle.surface_points(p)
    sums = np.zeros((12, 5))
    for t in range(9):
        if t >= 6:
            rho, J = oracle.macroscopic(p, f)
            P, U = oracle.interpolate(p, pts, c2, rho, J)
            un = (U * pts[:, 3:6]).sum(1)
            sums[:, 0] += P * P
            sums[:, 1] += (U * U).sum(1)
            sums[:, 2:] += U * un[:, None]
        f = oracle.advect(p, oracle.collide(p, c2, f))
    assert np.allclose(out["sums"], sums, rtol=1e-13, atol=0)
    assert np.array_equal(out["f"], f)
    rho, J = oracle.macroscopic(p, f)
    assert np.allclose(out["p1"], c2 * rho, rtol=1e-15, atol=0)
