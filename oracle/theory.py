"""Closed forms from the paper, used to pin the oracle (test infrastructure only).

Sign convention: the standing wave is p1 = P_a cos(k s) cos(w t) with s measured
from a pressure antinode (Eq. 38).  With that phase, F = -dU/ds of the Gor'kov
potential (Eq. 40) is

    F_s = + pi R^3 P_a^2 k Psi / (3 rho0)  sin(2 k s)     (sphere, Eq. 83a)
    F_s = + pi R^2 P_a^2 k Psi / (4 rho0)  sin(2 k s)     (cylinder, Eq. 83b)

with Psi = 1/c0^2 - 1/cp^2 (Eq. 84): positive Psi pushes the object toward the
pressure node at k s = pi/2, as Sec. VII states.  Eqs. (41), (60) and (83) print
a leading minus sign that belongs to the sin(k x) phase of the incident wave;
the magnitude is the same.
"""
import math


def psi(c0, cp):
    """Contrast factor of Eq. (84)."""
    return 1.0 / c0 ** 2 - 1.0 / cp ** 2


def gorkov_phi(rho_ratio, kappa_ratio):
    """Phi(rho~, kappa~) of Eq. (42) (sphere)."""
    return (5.0 * rho_ratio - 2.0) / (2.0 * rho_ratio + 1.0) - kappa_ratio


def wei_phi(rho_ratio, kappa_ratio):
    """Phi(rho~, kappa~) of Eq. (61) (cylinder)."""
    return (3.0 - rho_ratio) / (1.0 + rho_ratio) - kappa_ratio


def gorkov_force_3d(R, p_a, wavelength, s, c0, cp, rho0=1.0):
    """Sphere force along the wave axis, Eq. (83a) (density matched)."""
    k = 2.0 * math.pi / wavelength
    return math.pi * R ** 3 * p_a ** 2 * k * psi(c0, cp) / (3.0 * rho0) * math.sin(2.0 * k * s)


def wei_force_2d(R, p_a, wavelength, s, c0, cp, rho0=1.0):
    """Cylinder force per length along the wave axis, Eq. (83b) (density matched)."""
    k = 2.0 * math.pi / wavelength
    return math.pi * R ** 2 * p_a ** 2 * k * psi(c0, cp) / (4.0 * rho0) * math.sin(2.0 * k * s)


def lattice_omega(k, c2):
    """Angular frequency of the propagating mode of the tau = 1/2 wave scheme of
    Eqs. (62)-(64), (71) with wave vector k (one entry per axis), from the
    eigenvalues of its one-step amplification matrix:
        sin^2(w/2) = c^2 sum_a sin^2(k_a/2).
    For k -> 0 this gives w = c |k| (Eq. 68 with the local sound speed)."""
    s = c2 * sum(math.sin(0.5 * ka) ** 2 for ka in k)
    return 2.0 * math.asin(math.sqrt(s))


def volume_ratio(dim, R, c0, cp, d=4.0):
    """Compressibility volume of the smooth object of Eq. (79) over that of the
    sharp one: int (1 - kappa(r)/kappa0) dV / ((1 - kappa~) V_R), with
    kappa = 1/c^2 (density matched).  The monopole strength of Eq. (24)
    integrated over a graded object is proportional to the numerator, so the
    closed forms of Eqs. (83a, b) for the smooth object carry this factor."""
    from scipy.integrate import quad

    def g(r):
        c = cp + 0.5 * (c0 - cp) * (1 + math.tanh((r * r - R * R) / d))
        return 1 - c0 * c0 / (c * c)

    kap = c0 * c0 / (cp * cp)
    if dim == 2:
        return quad(lambda r: g(r) * 2 * math.pi * r, 0, R + 30, limit=400)[0] / ((1 - kap) * math.pi * R * R)
    return quad(lambda r: g(r) * 4 * math.pi * r * r, 0, R + 30, limit=400)[0] / ((1 - kap) * 4 / 3 * math.pi * R ** 3)
