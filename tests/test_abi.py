"""The C-ABI library builds, loads and exports what include/wlb.h declares, and
its host-side parameter checks behave as documented.  No GPU needed: only
calls that do no CUDA work are made here."""
import ctypes
import os
import re

import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wlb():
    from paper_2404_02346_gb300 import build as B
    B.build()
    import paper_2404_02346_gb300 as W
    W.lib()
    return W


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(wlb_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_function(wlb):
    declared = _declared()
    assert {"wlb_create", "wlb_init", "wlb_step", "wlb_force", "wlb_run", "wlb_fields",
            "wlb_surface", "wlb_mask", "wlb_destroy", "wlb_status_str"} <= declared
    L = ctypes.CDLL(wlb.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(L, name), name
    # the binding wraps every declared function
    assert declared <= set(wlb._SIGNATURES)


def test_status_strings(wlb):
    L = wlb.lib()
    for s in range(6):
        assert L.wlb_status_str(s)
    assert L.wlb_status_str(99) == b"unknown status"


def _valid():
    return workloads.sphere_3d(seed=3, n=64, wavelength=32.0, radius=6.0, n_surface=100,
                               n_periods=3, n_avg_periods=1)


def test_parameter_validation(wlb):
    ok = wlb.params_from_problem(_valid())
    assert wlb.validate(ok) == wlb.WLB_OK
    assert wlb.workspace_bytes(ok) > 2 * 7 * 64 ** 3 * 4

    def bad(**kw):
        p = wlb.params_from_problem(_valid())
        for k, v in kw.items():
            setattr(p, k, v)
        return wlb.validate(p)

    E = wlb.WLB_ERR_ARG
    assert bad(lattice=5) == E
    assert bad(precision=7) == E
    assert bad(nx=0) == E
    assert bad(wave_axis=3) == E
    assert bad(c0=0.6) == E            # 3 c0^2 >= 1: f_0^eq < 0, unstable
    assert bad(cp=0.58) == E           # 3 cp^2 >= 1
    assert bad(cp=-0.1) == E
    assert bad(rho0=0.0) == E
    assert bad(wavelength=30.0) == E   # 64 cells is not a whole number of wavelengths
    assert bad(c0=0.3) == E            # T = 32/0.3 not whole
    assert bad(radius=30.0) == E       # object + band wider than half the box
    assert bad(surface_radius=40.0) == E
    assert bad(n_surface=-1) == E
    assert bad(n_periods=0) == E
    assert bad(n_avg_periods=4) == E
    assert bad(interface_d=0.0) == E
    assert bad(p_a=float("nan")) == E
    p2 = wlb.params_from_problem(workloads.cylinder_2d(1))
    assert wlb.validate(p2) == wlb.WLB_OK
    p2.nz = 2
    assert wlb.validate(p2) == E


def test_workspace_size_is_checked_before_any_cuda_call(wlb):
    L = wlb.lib()
    p = wlb.params_from_problem(_valid())
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)  # aligned, never dereferenced: too small -> rejected first
    assert L.wlb_create(ctypes.byref(p), fake, 16, None, ctypes.byref(h)) in (wlb.WLB_ERR_OOM, wlb.WLB_ERR_CUDA)
    assert not h.value
    mis = ctypes.c_void_p((1 << 20) + 8)
    assert L.wlb_create(ctypes.byref(p), mis, 1 << 40, None, ctypes.byref(h)) == wlb.WLB_ERR_ARG
    assert not h.value


def test_null_arguments(wlb):
    L = wlb.lib()
    assert L.wlb_validate(None) == wlb.WLB_ERR_ARG
    assert L.wlb_init(None) == wlb.WLB_ERR_ARG
    assert L.wlb_step(None, 1, 0) == wlb.WLB_ERR_ARG
    assert L.wlb_destroy(None) == wlb.WLB_ERR_ARG
    assert L.wlb_set_two_step(None, 1, 0) == wlb.WLB_ERR_ARG
    assert L.wlb_set_two_step_tiles(None, 0) == wlb.WLB_ERR_ARG
    assert L.wlb_set_two_step_staging(None, 0) == wlb.WLB_ERR_ARG
    assert L.wlb_set_two_step_c2(None, 0) == wlb.WLB_ERR_ARG
    assert L.wlb_average_noalloc(None, 1, None) == wlb.WLB_ERR_ARG
    assert L.wlb_last_error(None) == b""


def test_batch_workspace_validation(wlb):
    """wlb_batch_workspace_bytes checks the batch on the host: mixed lattice
    types or precisions and rows the batched update does not cover are rejected."""
    L = wlb.lib()
    a = _valid()
    b = workloads.problem(2, (48, 32), 1, 16.0, 3.0, (24.0, 2.0), cp=0.3, n_surface=8,
                          n_periods=2, n_avg_periods=1)
    nb = ctypes.c_size_t()

    def arr(*probs):
        return (wlb.Params * len(probs))(*[wlb.params_from_problem(p) for p in probs])

    assert L.wlb_batch_workspace_bytes(arr(a, a), 2, ctypes.byref(nb)) == wlb.WLB_OK
    single = wlb.workspace_bytes(wlb.params_from_problem(a))
    assert nb.value >= 2 * single
    assert L.wlb_batch_workspace_bytes(arr(a, b), 2, ctypes.byref(nb)) == wlb.WLB_ERR_ARG
    assert L.wlb_batch_workspace_bytes(arr(a, dict(a, precision="f64")), 2, ctypes.byref(nb)) == wlb.WLB_ERR_ARG
    wide = workloads.problem(2, (1024, 32), 1, 16.0, 3.0, (512.0, 2.0), cp=0.3, n_surface=8,
                             n_periods=2, n_avg_periods=1)
    assert L.wlb_batch_workspace_bytes(arr(wide), 1, ctypes.byref(nb)) == wlb.WLB_ERR_ARG
    assert L.wlb_batch_workspace_bytes(arr(a), 0, ctypes.byref(nb)) == wlb.WLB_ERR_ARG


def test_driven_geometry_validation(wlb):
    p = workloads.problem(2, (32, 35), 1, 64.0, 3.0, (16.0, 14.0), cp=0.375, n_surface=8,
                          n_periods=2, n_avg_periods=1)
    p.update(boundary="driven", wall_damping=0.99, source_amplitude=0.016)
    assert wlb.validate(wlb.params_from_problem(p)) == wlb.WLB_OK   # box need not hold whole wavelengths
    near_wall = dict(p, center=(16.0, 8.0, 0.0))
    assert wlb.validate(wlb.params_from_problem(near_wall)) == wlb.WLB_ERR_ARG
    bad_phi = dict(p, wall_damping=1.5)
    assert wlb.validate(wlb.params_from_problem(bad_phi)) == wlb.WLB_ERR_ARG
    q = wlb.params_from_problem(p)
    q.boundary = 7
    assert wlb.validate(q) == wlb.WLB_ERR_ARG
    # batches are periodic only
    nb = ctypes.c_size_t()
    arr = (wlb.Params * 1)(wlb.params_from_problem(p))
    assert wlb.lib().wlb_batch_workspace_bytes(arr, 1, ctypes.byref(nb)) == wlb.WLB_ERR_ARG
