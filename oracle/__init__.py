"""FP64 CPU oracle for the wave lattice Boltzmann acoustic radiation force.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and
by the CPU-baseline leg of ``bench.py``.  The library (``paper_2404_02346_gb300``)
never imports it, and this package imports nothing from the library.

``problem`` dictionaries are the plain parameter sets produced by ``workloads``
(keys: dim, n, wave_axis, c0, cp, rho0, p_a, wavelength, antinode, center,
radius, interface_d, surface_radius, n_surface, n_steps, n_window).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("wave_axis", ctypes.c_int),
        ("c0", ctypes.c_double),
        ("cp", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("p_a", ctypes.c_double),
        ("wavelength", ctypes.c_double),
        ("antinode", ctypes.c_double),
        ("center", ctypes.c_double * 3),
        ("radius", ctypes.c_double),
        ("interface_d", ctypes.c_double),
        ("surface_radius", ctypes.c_double),
        ("n_surface", ctypes.c_int),
        ("n_steps", ctypes.c_long),
        ("n_window", ctypes.c_long),
        ("driven", ctypes.c_int),
        ("wall_damping", ctypes.c_double),
        ("source_amplitude", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        L.orc_run.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.orc_run.restype = ctypes.c_int
        L.orc_kernel.argtypes = [ctypes.c_double]
        L.orc_kernel.restype = ctypes.c_double
        L.orc_sincos_turns.argtypes = [ctypes.c_double, dp, dp]
        L.orc_sound_speed_sq_field.argtypes = [pp, dp]
        L.orc_mask.argtypes = [pp, ctypes.POINTER(ctypes.c_ubyte)]
        L.orc_surface_points.argtypes = [pp, dp]
        L.orc_initial_populations.argtypes = [pp, dp, dp]
        L.orc_macroscopic.argtypes = [pp, dp, dp, dp]
        L.orc_collide.argtypes = [pp, dp, dp, dp]
        L.orc_advect.argtypes = [pp, dp, dp]
        L.orc_apply_boundaries.argtypes = [pp, dp, dp, dp, ctypes.c_long]
        L.orc_interpolate.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.orc_force.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _struct(prob):
    s = _Problem()
    s.dim = int(prob["dim"])
    n = list(prob["n"]) + [1] * (3 - len(prob["n"]))
    for a in range(3):
        s.n[a] = int(n[a])
    s.wave_axis = int(prob["wave_axis"])
    for k in ("c0", "cp", "rho0", "p_a", "wavelength", "antinode", "radius",
              "interface_d", "surface_radius"):
        setattr(s, k, float(prob[k]))
    c = list(prob["center"]) + [0.0] * (3 - len(prob["center"]))
    for a in range(3):
        s.center[a] = float(c[a])
    s.n_surface = int(prob["n_surface"])
    s.n_steps = int(prob["n_steps"])
    s.n_window = int(prob["n_window"])
    s.driven = 1 if prob.get("boundary", "periodic") == "driven" else 0
    s.wall_damping = float(prob.get("wall_damping", 0.99))
    s.source_amplitude = float(prob.get("source_amplitude", 0.0))
    return s


def shape(prob):
    """Lattice shape (nz, ny, nx), the layout of every per-cell array."""
    n = list(prob["n"]) + [1] * (3 - len(prob["n"]))
    return (n[2], n[1], n[0])


def Q(prob):
    return 2 * int(prob["dim"]) + 1


def threads():
    return lib().orc_threads()


def run(prob, fields=False, populations=False):
    """Run the whole protocol.  Returns a dict with 'force' (3,), 'sums' (N, 5),
    'points' (N, 7) and, on request, 'p1' (nz, ny, nx), 'u1' (dim, nz, ny, nx) and
    'f' (Q, nz, ny, nx) at t = n_steps."""
    s = _struct(prob)
    shp = shape(prob)
    N = s.n_surface
    F = np.zeros(3)
    sums = np.zeros((max(N, 1), 5))
    pts = np.zeros((max(N, 1), 7))
    p1 = np.zeros(shp) if fields else None
    u1 = np.zeros((s.dim,) + shp) if fields else None
    f = np.zeros((Q(prob),) + shp) if populations else None
    null = ctypes.POINTER(ctypes.c_double)()
    rc = lib().orc_run(ctypes.byref(s), _p(F), _p(p1) if fields else null,
                       _p(u1) if fields else null, _p(f) if populations else null,
                       _p(sums), _p(pts))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out = {"force": F, "sums": sums[:N], "points": pts[:N]}
    if fields:
        out["p1"], out["u1"] = p1, u1
    if populations:
        out["f"] = f
    return out


def sound_speed_sq(prob):
    s = _struct(prob)
    c2 = np.zeros(shape(prob))
    lib().orc_sound_speed_sq_field(ctypes.byref(s), _p(c2))
    return c2


def mask(prob):
    s = _struct(prob)
    m = np.zeros(shape(prob), dtype=np.uint8)
    lib().orc_mask(ctypes.byref(s), m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return m


def surface_points(prob):
    s = _struct(prob)
    pts = np.zeros((max(s.n_surface, 1), 7))
    lib().orc_surface_points(ctypes.byref(s), _p(pts))
    return pts[: s.n_surface]


def initial_populations(prob, c2=None):
    s = _struct(prob)
    if c2 is None:
        c2 = sound_speed_sq(prob)
    f = np.zeros((Q(prob),) + shape(prob))
    lib().orc_initial_populations(ctypes.byref(s), _p(np.ascontiguousarray(c2)), _p(f))
    return f


def macroscopic(prob, f):
    s = _struct(prob)
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros(shape(prob))
    J = np.zeros((s.dim,) + shape(prob))
    lib().orc_macroscopic(ctypes.byref(s), _p(f), _p(rho), _p(J))
    return rho, J


def collide(prob, c2, f):
    s = _struct(prob)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    lib().orc_collide(ctypes.byref(s), _p(np.ascontiguousarray(c2)), _p(f), _p(out))
    return out


def advect(prob, fnew):
    s = _struct(prob)
    fnew = np.ascontiguousarray(fnew, dtype=np.float64)
    out = np.zeros_like(fnew)
    lib().orc_advect(ctypes.byref(s), _p(fnew), _p(out))
    return out


def interpolate(prob, pts, c2, rho, J):
    s = _struct(prob)
    N = s.n_surface
    P = np.zeros(max(N, 1))
    U = np.zeros((max(N, 1), 3))
    lib().orc_interpolate(ctypes.byref(s), _p(np.ascontiguousarray(pts)),
                          _p(np.ascontiguousarray(c2)), _p(np.ascontiguousarray(rho)),
                          _p(np.ascontiguousarray(J)), _p(P), _p(U))
    return P[:N], U[:N]


def force(dim, pts, Spp, Suu, Snu, n_window, rho0, c0):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    F = np.zeros(3)
    lib().orc_force(int(dim), int(pts.shape[0]), _p(pts),
                    _p(np.ascontiguousarray(Spp, dtype=np.float64)),
                    _p(np.ascontiguousarray(Suu, dtype=np.float64)),
                    _p(np.ascontiguousarray(Snu, dtype=np.float64)),
                    float(n_window), float(rho0), float(c0), _p(F))
    return F


def kernel(r):
    return lib().orc_kernel(float(r))


def sincos_turns(t):
    s = ctypes.c_double()
    c = ctypes.c_double()
    lib().orc_sincos_turns(float(t), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def apply_boundaries(prob, c2, f, fnew, t):
    """Driven-wall boundary step on post-collision values (in place copy)."""
    s = _struct(prob)
    out = np.ascontiguousarray(fnew, dtype=np.float64).copy()
    lib().orc_apply_boundaries(ctypes.byref(s), _p(np.ascontiguousarray(c2)),
                               _p(np.ascontiguousarray(f, dtype=np.float64)), _p(out), int(t))
    return out
