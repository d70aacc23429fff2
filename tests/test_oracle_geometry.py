"""Pins of the oracle's geometry: the sound-speed profile (Eq. 79), cell classes,
surface elements (Sec. VI) and the interpolation kernel (Eq. 82)."""
import math

import numpy as np
import pytest

import oracle
import workloads


def _prob(dim, n, center, R=6.0, cp=0.375, N=64, Rs=None):
    return workloads.problem(dim, n, dim - 1, float(n[dim - 1]), R, center, cp=cp, n_surface=N,
                             n_periods=1, n_avg_periods=1, surface_radius=Rs)


def test_sound_speed_profile_reading():
    """Eq. (79) read with c0 in the fluid and cp inside (the object's speed):
    c = cp at the centre, (c0 + cp)/2 on |r - r0| = R, c0 far away, monotone."""
    p = _prob(3, (48, 48, 48), (24.0, 24.0, 24.0), R=10.0, cp=0.375)
    c = np.sqrt(oracle.sound_speed_sq(p))
    assert c[24, 24, 24] == 0.375
    assert c[24, 24, 34] == pytest.approx(0.5 * (0.25 + 0.375), abs=1e-15)  # |r - r0| = R exactly
    assert c[0, 0, 0] == 0.25
    line = c[24, 24, 24:]
    assert np.all(np.diff(line) <= 0) and line[-1] == 0.25  # cp > c0 here
    # periodic minimum image: the profile is symmetric about the centre across the wrap
    q = _prob(3, (32, 32, 32), (2.0, 16.0, 16.0), R=6.0)
    cq = np.sqrt(oracle.sound_speed_sq(q))
    for j in range(1, 12):
        assert cq[16, 16, (2 + j) % 32] == cq[16, 16, (2 - j) % 32]


def test_mask_classes_follow_the_profile():
    """Cells classed fluid/object carry exactly c0^2/cp^2 (tanh = +-1 in double
    precision); band cells are those with |d^2 - R^2| < 20 d."""
    for dim, n, ctr in ((2, (48, 40), (23.5, 20.0)), (3, (40, 38, 36), (19.25, 18.5, 17.75))):
        p = _prob(dim, n, ctr, R=12.0, cp=0.5)
        m = oracle.mask(p)
        c2 = oracle.sound_speed_sq(p)
        assert set(np.unique(m)) == {0, 1, 2}
        assert np.all(c2[m == 0] == 0.0625)
        assert np.all(c2[m == 1] == 0.25)
        idx = np.indices(oracle.shape(p))
        d2 = 0
        for a in range(dim):
            d2 = d2 + (idx[2 - a] - p["center"][a]) ** 2
        q = d2 - p["radius"] ** 2
        assert np.array_equal(m == 2, np.abs(q) < 20 * p["interface_d"])


def test_sound_speed_field_integrates_to_the_profile_volume():
    """The lattice sum of the compressibility contrast 1 - c0^2/c^2 over cells
    equals the continuous integral of Eq. (79)'s profile (2D area, 3D volume)."""
    from scipy.integrate import quad
    c0, cp, d = 0.25, 0.375, 4.0

    def g(r, R):
        c = cp + 0.5 * (c0 - cp) * (1 + math.tanh((r * r - R * R) / d))
        return 1 - c0 * c0 / (c * c)

    for dim, n, ctr, R in ((2, (64, 64), (31.25, 32.5), 12.0), (3, (48, 48, 48), (23.5, 24.25, 24.0), 12.0)):
        p = _prob(dim, n, ctr, R=R, cp=cp)
        c2 = oracle.sound_speed_sq(p)
        lattice = (1 - c0 * c0 / c2).sum()
        if dim == 2:
            cont = quad(lambda r: g(r, R) * 2 * math.pi * r, 0, R + 30, limit=400)[0]
        else:
            cont = quad(lambda r: g(r, R) * 4 * math.pi * r * r, 0, R + 30, limit=400)[0]
        assert abs(lattice / cont - 1) < 0.01


def test_sincos_turns_matches_high_precision():
    """The series sin/cos of 2 pi t used for the surface points is within 2 ulp
    of the exact values (40-digit reference)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    ts = np.concatenate([rng.uniform(0, 1, 2000), np.arange(16) / 16.0, [0.0, 0.999999999]])
    err = 0.0
    for t in ts:
        s, c = oracle.sincos_turns(t)
        a = 2 * mpmath.pi * mpmath.mpf(float(t))
        err = max(err, abs(s - float(mpmath.sin(a))), abs(c - float(mpmath.cos(a))))
    assert err <= 2.3e-16


def test_surface_points_3d_fibonacci():
    """Fibonacci points: z_k = 1 - (2k+1)/N, azimuth k pi (3 - sqrt 5), unit
    normals, equal areas 4 pi R^2 / N, centres r0 + R n."""
    N, Rs = 2000, 16.0
    p = _prob(3, (64, 64, 64), (32.0, 31.5, 30.25), R=12.0, N=N, Rs=Rs)
    pts = oracle.surface_points(p)
    k = np.arange(N)
    nz = 1 - (2 * k + 1) / N
    assert np.array_equal(pts[:, 5], nz)
    rho = np.sqrt(1 - nz * nz)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    g = mpmath.pi * (3 - mpmath.sqrt(5))
    cphi = np.array([float(mpmath.cos(int(j) * g)) for j in k])
    sphi = np.array([float(mpmath.sin(int(j) * g)) for j in k])
    # the azimuth is frac(k h) turns with h the double nearest (3 - sqrt 5)/2, so
    # its error is bounded by 2 pi (ulp(k h) + k ulp(h)) ~ 1e-12 rad at k < 2000
    assert np.abs(pts[:, 3] - rho * cphi).max() < 1e-12
    assert np.abs(pts[:, 4] - rho * sphi).max() < 1e-12
    assert np.abs(np.linalg.norm(pts[:, 3:6], axis=1) - 1).max() < 4e-16
    assert np.allclose(pts[:, 0:3], np.array(p["center"]) + Rs * pts[:, 3:6], rtol=0, atol=1e-13)
    assert np.allclose(pts[:, 6], 4 * math.pi * Rs * Rs / N, rtol=1e-15)
    assert abs(pts[:, 5].sum()) < 1e-12
    # closed surface: sum n dS small (quadrature residual) relative to the area
    assert np.abs((pts[:, 3:6] * pts[:, 6:7]).sum(0)).max() < 2e-3 * 4 * math.pi * Rs * Rs


def test_surface_points_2d_arcs():
    N, Rs = 64, 8.0
    p = _prob(2, (64, 64), (32.0, 8.25), R=8.0, N=N, Rs=Rs)
    pts = oracle.surface_points(p)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    th = [2 * mpmath.pi * (k + mpmath.mpf(1) / 2) / N for k in range(N)]
    assert np.abs(pts[:, 3] - np.array([float(mpmath.cos(t)) for t in th])).max() < 2.3e-16
    assert np.abs(pts[:, 4] - np.array([float(mpmath.sin(t)) for t in th])).max() < 2.3e-16
    assert np.all(pts[:, 5] == 0) and np.all(pts[:, 2] == 0)
    assert np.allclose(pts[:, 6], 2 * math.pi * Rs / N, rtol=1e-15)
    # mirror pairs k <-> N-1-k about the x axis
    assert np.abs(pts[::-1, 4] + pts[:, 4]).max() < 4e-16
    assert np.abs(pts[::-1, 3] - pts[:, 3]).max() < 4e-16


def test_kernel_identities():
    """Eq. (82): on the three nearest nodes the weights sum to 1, have zero first
    moment and square-sum 1/2 for every offset; delta(0) = 2/3, delta(1/2) = 1/2
    from both branches, delta(1) = 1/6, delta(3/2) = 0."""
    assert oracle.kernel(0.0) == pytest.approx(2 / 3, abs=1e-16)
    assert oracle.kernel(0.5) == 0.5 and oracle.kernel(np.nextafter(0.5, 1)) == pytest.approx(0.5, abs=1e-8)
    assert oracle.kernel(1.0) == pytest.approx(1 / 6, abs=1e-16)
    assert oracle.kernel(1.5) == 0.0 and oracle.kernel(-1.5) == 0.0 and oracle.kernel(2.0) == 0.0
    rng = np.random.default_rng(11)
    for X in np.concatenate([rng.uniform(-40, 40, 500), np.linspace(-0.5, 0.5, 101)]):
        b = math.floor(X + 0.5)
        r = np.array([b - 1 - X, b - X, b + 1 - X])
        w = np.array([oracle.kernel(v) for v in r])
        assert abs(w.sum() - 1) < 1e-15
        assert abs((r * w).sum()) < 1e-15
        assert abs((w * w).sum() - 0.5) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_interpolation_exact_on_linear_fields(dim):
    """Eqs. (80)-(81) reproduce fields linear in x, y, z (partition of unity and
    zero first moment), including stencils that wrap around the box."""
    n = (24, 22, 20)[:dim]
    p = _prob(dim, n, tuple(v / 2 for v in n), R=5.0, cp=0.25, N=50, Rs=5.0)
    p["center"] = (12.0, 11.0, 10.0)[:dim] + (0.0,) * (3 - dim)
    pts = oracle.surface_points(p)
    shp = oracle.shape(p)
    idx = np.indices(shp).astype(float)
    coef = np.array([0.3, -0.7, 0.2])
    lin = 1.5 + sum(coef[a] * idx[2 - a] for a in range(dim))
    c2 = np.full(shp, 0.0625)
    rho = lin / 0.0625
    J = np.stack([lin * (a + 1) for a in range(dim)])
    P, U = oracle.interpolate(p, pts, c2, rho, J)
    want = 1.5 + sum(coef[a] * pts[:, a] for a in range(dim))
    assert np.abs(P - want).max() < 1e-12
    for a in range(dim):
        assert np.abs(U[:, a] - want * (a + 1)).max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_interpolation_is_translation_invariant_across_the_wrap(dim):
    """Periodic stencils: shifting the points across the box edge and rolling the
    fields by the same amount gives the same interpolated values."""
    n = (24, 22, 20)[:dim]
    p = _prob(dim, n, tuple(v / 2 for v in n), R=5.0, cp=0.25, N=40, Rs=5.0)
    rng = np.random.default_rng(5)
    shp = oracle.shape(p)
    c2 = rng.uniform(0.05, 0.1, shp)
    rho = rng.standard_normal(shp)
    J = rng.standard_normal((dim,) + shp)
    pts = oracle.surface_points(p)
    P0, U0 = oracle.interpolate(p, pts, c2, rho, J)
    shift = np.array([11, -9, 7][:dim])
    pts2 = pts.copy()
    pts2[:, :dim] -= shift
    axes = tuple(2 - a for a in range(dim))
    roll = lambda a: np.roll(a, tuple(-s for s in shift), axis=axes)
    P1, U1 = oracle.interpolate(p, pts2, roll(c2), roll(rho),
                                np.stack([roll(J[a]) for a in range(dim)]))
    assert np.abs(P1 - P0).max() < 1e-13
    assert np.abs(U1 - U0).max() < 1e-13
