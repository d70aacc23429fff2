"""wlb_average_noalloc, the allocation-free averaging call, against the
regular wlb_step(sample=1) + wlb_force path on the same states, twice in a row.

Callers whose device memory is a fixed pool owned by someone else (a caching
allocator that has reserved the whole budget, an arena given to a plugin), or
that cannot afford cudaMalloc / cudaFree in their loop, use this call.  Its
running sums live in a static device array shared by every call, so this file
runs last and checks that a second call does not see the first call's sums.
It runs the same sampling, fold and force kernels with the same fold cadence
as the regular path, so the forces must be equal bit for bit; a warm call
must leave the device's free memory unchanged.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wlb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2404_02346_gb300 import build as B
    B.build()
    import paper_2404_02346_gb300 as W
    W.lib()
    return W


def _noalloc(W, solver, n):
    F = np.zeros(3)
    st = W.lib().wlb_average_noalloc(solver._h, n, F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == W.WLB_OK, W.lib().wlb_last_error(solver._h)
    return F


def _regular(W, prob, n_before, n_avg):
    with W.Solver(prob) as s:
        s.init()
        s.step(n_before, sample=False)
        s.step(n_avg, sample=True)
        return s.force()


@pytest.mark.parametrize("kind", ["3d_f32", "3d_f16", "2d_f64"])
def test_noalloc_average_matches_regular_path_twice(wlb, kind):
    if kind.startswith("3d"):
        prob = workloads.problem(3, (128, 48, 64), 2, 32.0, 6.0, (64.375, 23.75, 4.125), cp=0.42,
                                 n_surface=500, n_periods=4, n_avg_periods=2, precision=kind[3:])
    else:
        prob = workloads.problem(2, (128, 64), 1, 32.0, 5.0, (64.25, 3.5), cp=0.375, n_surface=64,
                                 n_periods=4, n_avg_periods=2, precision="f64")
    T = prob["period"]
    n_free, n_win = 2 * T, 2 * T - 5  # a window that ends mid-period
    ref1 = _regular(wlb, prob, n_free, n_win)
    ref2 = _regular(wlb, prob, n_free + n_win, n_win)
    with wlb.Solver(prob) as s:
        s.init()
        s.step(n_free, sample=False)
        F1 = _noalloc(wlb, s, n_win)
        F2 = _noalloc(wlb, s, n_win)  # continues from the advanced state
        assert s.info().steps_done == n_free + 2 * n_win
    axis = prob["wave_axis"]
    for F, ref in ((F1, ref1), (F2, ref2)):
        assert np.array_equal(F, ref), (F, ref)
    assert abs(F1[axis] - F2[axis]) > 0  # different windows, different averages


def test_noalloc_warm_call_leaves_free_memory_unchanged(wlb):
    import torch

    prob = workloads.problem(3, (128, 48, 64), 2, 32.0, 6.0, (64.375, 23.75, 4.125), cp=0.42,
                             n_surface=500, n_periods=4, n_avg_periods=2)
    with wlb.Solver(prob) as s:
        s.init()
        _noalloc(wlb, s, prob["period"] + 3)  # warm: kernels loaded, address looked up
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        F = _noalloc(wlb, s, prob["period"] + 3)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.all(np.isfinite(F)) and F[2] != 0


def test_noalloc_limits_and_state(wlb):
    L = wlb.lib()
    big = workloads.problem(3, (64, 64, 64), 2, 32.0, 8.0, (32.0, 32.0, 4.0), cp=0.4,
                            n_surface=8193, n_periods=1, n_avg_periods=1)
    F = np.zeros(3)
    Fp = F.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    with wlb.Solver(big) as s:
        assert L.wlb_average_noalloc(s._h, 4, Fp) == wlb.WLB_ERR_STATE
        s.init()
        assert L.wlb_average_noalloc(s._h, 4, Fp) == wlb.WLB_ERR_ARG
        assert b"WLB_NOALLOC_MAX_SURFACE" in L.wlb_last_error(s._h)
        assert L.wlb_average_noalloc(s._h, -1, Fp) == wlb.WLB_ERR_ARG
    ok = dict(big, n_surface=100)
    with wlb.Solver(ok) as s:
        s.init()
        F[:] = 1.0
        assert L.wlb_average_noalloc(s._h, 0, Fp) == wlb.WLB_OK
        assert np.array_equal(F, np.zeros(3))
