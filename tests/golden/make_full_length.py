"""Write the full-length oracle goldens of the two 3D benchmark lattices.

Calls only the FP64 oracle (``oracle.run``) on the seeded problems of
``workloads``; nothing here touches the GPU library.  Each golden holds the
oracle's result of the whole protocol (Sec. V steps, Eqs. 62-64 and 71; the
surface average of Eqs. 80-82; King's integral, Eq. 14):

  force        (3,) FP64, Eq. (14) over the averaging window
  sums         (N, 5) FP64 running sums of p1^2, u1.u1, (n.u1) u1
  p1_x, p1_y, p1_z
               p1 = c^2 rho1 at the last step on the three lattice planes
               through the object's centre (x = xc: [z][y]; y = yc: [z][x];
               z = zc: [y][x]), stored as FP32 (the rounding, at most
               2^-24 |p1| < 1e-7 p_a, is far below the 1e-4 p_a parity bar)
  u1_y         u1 = J1 / rho0 on the plane y = yc, [a][z][x], FP32
  plane_index  (xc, yc, zc)
  params       the problem dictionary as JSON (the test rebuilds the problem
               from ``workloads`` and checks that it is this one)

Workloads:
  sphere256        256^3 D3Q7, lambda = 128, R = 16 at lambda/8, seeded
                   kappa~, 2000 points, 30 periods with the last 10 averaged
                   (15360 steps): the whole benchmark protocol.
  sphere512_kz_pi4 512^3 D3Q7, lambda = 256, R = 24, kappa~ = 0.5, 4096
                   points, k z0 = pi/4 (z0 = 32): the first 2 periods
                   (2048 steps) with the second averaged.

Usage: python tests/golden/make_full_length.py [sphere256] [sphere512_kz_pi4]
(about 1.5 h each on 8 host cores; OMP_NUM_THREADS sets the threads).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def problem(name):
    if name == "sphere256":
        return workloads.sphere_3d(seed=1)
    if name == "sphere512_kz_pi4":
        # k z0 = pi/4 with lambda = 256: z0 = lambda/8 = 32 cells
        return workloads.sphere_3d(n=512, wavelength=256.0, radius=24.0, n_surface=4096, kappa=0.5,
                                   z0=32.0, n_periods=2, n_avg_periods=1)
    raise KeyError(name)


def path(name):
    return os.path.join(HERE, "full_length_%s.npz" % name)


def plane_index(prob):
    return tuple(int(round(c)) for c in prob["center"][:3])


def write(name):
    prob = problem(name)
    t0 = time.perf_counter()
    o = oracle.run(prob, fields=True)
    dt = time.perf_counter() - t0
    xc, yc, zc = plane_index(prob)
    p1, u1 = o["p1"], o["u1"]
    np.savez_compressed(
        path(name),
        force=o["force"], sums=o["sums"],
        p1_x=p1[:, :, xc].astype(np.float32), p1_y=p1[:, yc, :].astype(np.float32),
        p1_z=p1[zc, :, :].astype(np.float32), u1_y=u1[:, :, yc, :].astype(np.float32),
        plane_index=np.array([xc, yc, zc]), params=json.dumps(prob, sort_keys=True),
        oracle_seconds=dt, oracle_threads=oracle.threads())
    print("%s: force %s, %.0f s on %d threads" % (name, o["force"], dt, oracle.threads()), flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or ["sphere256", "sphere512_kz_pi4"]
    oracle.build.build()
    for n in names:
        write(n)
