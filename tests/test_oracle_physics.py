"""Physics pins of the whole oracle protocol against the paper's closed forms:
Wei's cylinder force (Eq. 83b) and Gor'kov's sphere force (Eq. 83a) at the
paper's small kR = 0.125 (Table I), their linearity in Psi (Eq. 84, Sec. VII)
and the sin(2 k s) position dependence (Sec. VII).

Setup as in Sec. VII (lambda >> R, 64-cell periodic lateral box, object at
lambda/8 from a pressure antinode), resized so the periodic box along the wave
holds one wavelength.  The integration surface sits R_p + 2 outside the
interface band, where the time-averaged momentum flux is that of the
homogeneous fluid; the average is taken over the second period.  In a closed
lossless periodic box the object couples the degenerate cos(ks)/sin(ks) modes
and the force drifts slowly over tens of periods, so early periods are the ones
comparable with the single-mode closed forms.

Two tolerances per case: against the sharp-object closed form (the paper's own
agreement is a few per cent, Tables II-III), and against the closed form with
the object's volume replaced by the compressibility volume of the smooth
profile of Eq. (79), int (1 - kappa(r)/kappa0) dV / (1 - kappa~) (the monopole
strength of Eq. 24 integrated over a graded object).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from oracle import theory

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _volume_ratio(dim, R, c0, cp, d=4.0):
    return theory.volume_ratio(dim, R, c0, cp, d)


def _cyl(cp, s0, R=8.0, lam=400.0, lateral=64, N=64):
    return workloads.problem(2, (lateral, int(lam)), 1, lam, R, (lateral / 2, s0), cp=cp, c0=0.25,
                             n_surface=N, n_periods=2, n_avg_periods=1, surface_radius=R + 2)


def test_wei_cylinder_force():
    c0, cp, lam, R = 0.25, 0.375, 400.0, 8.0
    F = oracle.run(_cyl(cp, lam / 8))["force"]
    wei = theory.wei_force_2d(R, 1e-3, lam, lam / 8, c0, cp)
    assert wei > 0 and F[1] > 0  # toward the node at lambda/4 for Psi > 0 (Sec. VII)
    assert abs(F[1] / wei - 1) < 0.05
    assert abs(F[1] / (wei * _volume_ratio(2, R, c0, cp)) - 1) < 0.02
    assert abs(F[0]) < 1e-6 * abs(F[1])


@pytest.mark.slow
def test_gorkov_sphere_force():
    c0, cp, lam, R = 0.25, 0.375, 160.0, 4.0
    p = workloads.problem(3, (40, 40, int(lam)), 2, lam, R, (20.0, 20.0, lam / 8), cp=cp, c0=c0,
                          n_surface=400, n_periods=2, n_avg_periods=1, surface_radius=R + 2)
    F = oracle.run(p)["force"]
    gk = theory.gorkov_force_3d(R, 1e-3, lam, lam / 8, c0, cp)
    assert gk > 0 and F[2] > 0
    assert abs(F[2] / gk - 1) < 0.15  # R = 4 cells: smooth-profile volume is 13 % larger
    assert abs(F[2] / (gk * _volume_ratio(3, R, c0, cp)) - 1) < 0.03
    assert np.all(np.abs(F[:2]) < 1e-2 * abs(F[2]))


def test_force_is_linear_in_contrast_factor():
    """Sec. VII: <F> linear in Psi = 1/c0^2 - 1/cp^2 with R^2 = 0.999 in 2D."""
    c0, lam = 0.25, 400.0
    ratios = [0.8, 1.2, 1.5, 2.0]
    psi = np.array([theory.psi(c0, r * c0) for r in ratios])
    F = np.array([oracle.run(_cyl(r * c0, lam / 8))["force"][1] for r in ratios])
    A = np.vstack([psi, np.ones_like(psi)]).T
    coef, res, *_ = np.linalg.lstsq(A, F, rcond=None)
    r2 = 1 - ((F - A @ coef) ** 2).sum() / ((F - F.mean()) ** 2).sum()
    assert r2 >= GOLD["contrast_linearity_R2"]["2d"]
    slope = theory.wei_force_2d(8.0, 1e-3, lam, lam / 8, c0, 2 * c0) / theory.psi(c0, 2 * c0)
    assert abs(coef[0] / slope - 1) < 0.06
    assert np.all(np.sign(F) == np.sign(psi))


def test_force_follows_sin_2ks_and_vanishes_at_the_node():
    """Sec. VII: F proportional to sin(2 k s), zero at the node s = lambda/4.
    Mirror symmetry s -> lambda/2 - s of the lattice flips p1, so F(3 lambda/8)
    = -F(lambda/8) and F(lambda/4) = 0 to rounding."""
    lam, cp = 400.0, 0.375
    F = {s: oracle.run(_cyl(cp, s))["force"][1] for s in (lam / 16, lam / 8, lam / 4, 3 * lam / 8)}
    top = F[lam / 8]
    assert abs(F[lam / 4]) < 1e-9 * abs(top)
    assert abs(F[3 * lam / 8] + top) < 1e-9 * abs(top)
    assert F[lam / 16] / top == pytest.approx(math.sin(math.pi / 4), rel=0.03)


def test_radius_exponent_2d():
    """Table III: F ~ R^2 for the cylinder (measured 2.0127).  The smooth
    profile's extra volume shrinks as R grows, so the exponent of the raw
    forces sits slightly below 2; corrected by that volume it is 2."""
    c0, cp, lam = 0.25, 0.375, 400.0
    Rs = np.array([6.0, 8.0, 10.0])
    F = np.array([oracle.run(_cyl(cp, lam / 8, R=R))["force"][1] for R in Rs])
    raw = np.polyfit(np.log(Rs), np.log(F), 1)[0]
    vr = np.array([_volume_ratio(2, R, c0, cp) for R in Rs])
    corr = np.polyfit(np.log(Rs), np.log(F / vr), 1)[0]
    want = GOLD["table_III_exponents_2d"]["R_p"]["expected"]
    assert abs(raw - want) < 0.1
    assert abs(corr - want) < 0.03
