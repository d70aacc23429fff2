"""Seeded synthetic problem sets shared by the library's tests, the oracle's tests
and the benchmark.

This module only builds parameter dictionaries (lattice size, wave, object,
surface sampling, averaging window) and draws the seeded random parameters; it
holds none of the method's arithmetic.  The paper uses no dataset: the problems
below are shaped like its Table I setups and the workloads the benchmark runs.

Problem keys (all lattice units, dx = dt = 1):
    dim            2 (D2Q5) or 3 (D3Q7)
    n              (nx, ny, nz); nz = 1 in 2D
    wave_axis      axis of the standing wave
    c0, cp, rho0   fluid and object sound speeds, mean density
    p_a            pressure amplitude of the standing wave
    wavelength     lambda (cells); the box along wave_axis holds whole wavelengths
    antinode       coordinate of a pressure antinode along wave_axis
    center         object centre, quantised to multiples of 2^-10 cells
    radius         object radius R_p
    interface_d    "square thickness" d of the sound-speed profile (4)
    surface_radius radius of the integration surface (defaults to R_p)
    n_surface      number of surface elements
    n_steps        total LB steps  (n_periods * T, T = lambda / c0)
    n_window       averaged steps  (n_avg_periods * T)
    precision      population storage of the GPU path: "f32" or "f64"
"""
import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014), the published 64-bit mixer."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self):
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def quantise(v, bits=10):
    """Round down to a multiple of 2^-bits (keeps |r - r0|^2 exact in FP64)."""
    s = float(1 << bits)
    return math.floor(v * s) / s


def problem(dim, n, wave_axis, wavelength, radius, center, cp, c0=0.25, p_a=1e-3,
            n_surface=64, n_periods=20, n_avg_periods=5, precision="f32",
            antinode=0.0, interface_d=4.0, surface_radius=None, rho0=1.0):
    n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
    T = wavelength / c0
    if abs(T - round(T)) > 1e-9:
        raise ValueError("period lambda/c0 must be a whole number of steps")
    T = int(round(T))
    center = tuple(quantise(float(c)) for c in center) + (0.0,) * (3 - len(center))
    return {
        "dim": int(dim), "n": n, "wave_axis": int(wave_axis),
        "c0": float(c0), "cp": float(cp), "rho0": float(rho0), "p_a": float(p_a),
        "wavelength": float(wavelength), "antinode": float(antinode),
        "center": center, "radius": float(radius), "interface_d": float(interface_d),
        "surface_radius": float(radius if surface_radius is None else surface_radius),
        "n_surface": int(n_surface), "n_steps": int(n_periods * T),
        "n_window": int(n_avg_periods * T), "precision": precision, "period": T,
    }


def cylinder_2d(seed=1, n_periods=20, n_avg_periods=5):
    """2D infinite cylinder, FP64 populations: 128 x 128 D2Q5, standing wave along y
    with lambda = 64, p_a = 1e-3, R = 8 at y = lambda/8 (x = 64), sound-speed ratio
    1.5, 64 surface points, 20 periods averaged over the last 5.  The seed draws
    the centre jitter U[-1/2, 1/2) per axis."""
    g = SplitMix64(seed)
    jx = g.uniform() - 0.5
    jy = g.uniform() - 0.5
    lam = 64.0
    return problem(2, (128, 128), 1, lam, 8.0, (64.0 + jx, lam / 8 + jy), cp=1.5 * 0.25,
                   n_surface=64, n_periods=n_periods, n_avg_periods=n_avg_periods,
                   precision="f64")


def sphere_3d(seed=1, n=256, wavelength=128.0, radius=16.0, n_surface=2000,
              n_periods=30, n_avg_periods=10, kappa=None, z0=None, precision="f32"):
    """3D sphere, FP32 populations: n^3 D3Q7, standing wave along z, p_a = 1e-3,
    sphere at z = lambda/8 (x = y = n/2), compressibility ratio kappa~ = c0^2/cp^2
    drawn from U[0.2, 0.8] by the seed unless given, Fibonacci surface points.
    Default: 256^3, lambda = 128, R = 16, 2000 points, 30 periods, last 10 averaged."""
    if kappa is None:
        kappa = 0.2 + 0.6 * SplitMix64(seed).uniform()
    c0 = 0.25
    cp = c0 / math.sqrt(kappa)
    if z0 is None:
        z0 = wavelength / 8.0
    p = problem(3, (n, n, n), 2, wavelength, radius, (n / 2, n / 2, z0), cp=cp, c0=c0,
                n_surface=n_surface, n_periods=n_periods, n_avg_periods=n_avg_periods,
                precision=precision)
    p["kappa"] = kappa
    return p


def sphere_3d_large(position=0, n_periods=30, n_avg_periods=10, precision="f32"):
    """512^3 D3Q7, lambda = 256, R = 24, 4096 points, kappa~ = 0.5; one of the 16
    positions k z_j = j pi / 15 of the force-vs-position sweep."""
    lam = 256.0
    kz = position * math.pi / 15.0
    z0 = kz * lam / (2.0 * math.pi)
    return sphere_3d(n=512, wavelength=lam, radius=24.0, n_surface=4096, kappa=0.5,
                     z0=z0, n_periods=n_periods, n_avg_periods=n_avg_periods,
                     precision=precision)


def _ensemble_member(g, dim, edge, n_surface, n_periods, n_avg_periods, precision):
    """One ensemble lattice: lambda = edge/2, R ~ U[4, 12], k z0 ~ U[0, pi],
    sound-speed ratio c~ ~ U[0.8, 2.0] (density matched, so kappa~ = 1/c~^2)."""
    lam = edge / 2.0
    R = quantise(4.0 + 8.0 * g.uniform())
    kz = math.pi * g.uniform()
    c_ratio = 0.8 + 1.2 * g.uniform()
    z0 = kz * lam / (2.0 * math.pi)
    center = (edge / 2.0,) * (dim - 1) + (z0,)
    n = (edge,) * dim
    p = problem(dim, n, dim - 1, lam, R, center, cp=c_ratio * 0.25, n_surface=n_surface,
                n_periods=n_periods, n_avg_periods=n_avg_periods, precision=precision)
    p.update({"kz": kz, "c_ratio": c_ratio, "kappa": 1.0 / c_ratio ** 2,
              "ka": 2.0 * math.pi / lam * R})
    return p


def ensemble_3d(seed=1, count=64, n_surface=1000, n_periods=25, n_avg_periods=10, precision="f32"):
    """Batched ensemble: count independent 3D lattices with edge uniform in
    {96, 128, 160}, lambda = edge/2, R ~ U[4, 12], k z0 ~ U[0, pi], c~ ~ U[0.8, 2.0],
    1000 surface points, 25 periods (last 10 averaged)."""
    g = SplitMix64(seed)
    out = []
    for _ in range(count):
        edge = (96, 128, 160)[min(2, int(3 * g.uniform()))]
        out.append(_ensemble_member(g, 3, edge, n_surface, n_periods, n_avg_periods, precision))
    return out


def ensemble_2d(seed=1, count=512, edge=192, n_surface=1000, n_periods=25, n_avg_periods=10,
                precision="f32"):
    """2D variant: count cylinders on edge^2 lattices (192^2), lambda = edge/2."""
    g = SplitMix64(seed)
    return [_ensemble_member(g, 2, edge, n_surface, n_periods, n_avg_periods, precision)
            for _ in range(count)]


# Learned-surrogate inputs: k R_p, k z0, sound-speed ratio (kappa~ = 1/c~^2).
SURROGATE_BOX = {"ka": (0.1, 1.2), "kz": (0.0, math.pi), "c_ratio": (0.8, 2.0)}


def latin_hypercube(n, dims, seed):
    """n points in [0, 1)^dims, one per stratum on every axis (SplitMix64)."""
    g = SplitMix64(seed)
    cols = []
    for _ in range(dims):
        perm = list(range(n))
        for i in range(n - 1, 0, -1):
            j = int(g.uniform() * (i + 1))
            perm[i], perm[j] = perm[j], perm[i]
        cols.append([(perm[i] + g.uniform()) / n for i in range(n)])
    return [[cols[d][i] for d in range(dims)] for i in range(n)]


def surrogate_problem(ka, kz, c_ratio, edge=192, n_surface=1000, n_periods=25, n_avg_periods=10,
                      precision="f32"):
    """2D cylinder on an edge^2 lattice (lambda = edge/2) for the given features."""
    lam = edge / 2.0
    k = 2.0 * math.pi / lam
    R = quantise(ka / k)
    z0 = kz / k
    p = problem(2, (edge, edge), 1, lam, R, (edge / 2.0, z0), cp=c_ratio * 0.25, n_surface=n_surface,
                n_periods=n_periods, n_avg_periods=n_avg_periods, precision=precision)
    p.update({"ka": k * R, "kz": kz, "c_ratio": c_ratio, "kappa": 1.0 / c_ratio ** 2,
              "features": (k * R, kz, 1.0 / c_ratio ** 2, c_ratio)})
    return p


def surrogate_problems(n, seed, **kw):
    """Seeded Latin-hypercube sample of the surrogate's input box."""
    (a0, a1), (z0, z1), (c0, c1) = (SURROGATE_BOX[k] for k in ("ka", "kz", "c_ratio"))
    return [surrogate_problem(a0 + (a1 - a0) * u[0], z0 + (z1 - z0) * u[1], c0 + (c1 - c0) * u[2], **kw)
            for u in latin_hypercube(n, 3, seed)]


def surrogate_queries(n, seed, outside_fraction=0.0):
    """n feature rows (k R, k z0, kappa~, c~) drawn uniformly in the box; a
    fraction of them pushed outside (k R beyond the trained range)."""
    g = SplitMix64(seed)
    (a0, a1), (z0, z1), (c0, c1) = (SURROGATE_BOX[k] for k in ("ka", "kz", "c_ratio"))
    rows = []
    for i in range(n):
        ka = a0 + (a1 - a0) * g.uniform()
        kz = z0 + (z1 - z0) * g.uniform()
        c = c0 + (c1 - c0) * g.uniform()
        if g.uniform() < outside_fraction:
            ka = a1 + 0.1 + 0.2 * g.uniform()
        rows.append((ka, kz, 1.0 / c ** 2, c))
    return rows
