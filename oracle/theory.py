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
