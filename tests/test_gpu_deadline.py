"""Host-clock watchdog of wlb_run (wlb_set_deadline), exercised with a host
timer only: a deadline that a full 256^3 force evaluation cannot meet stops
the run with WLB_ERR_TIMEOUT long before it would end, on a period boundary,
with the handle usable; a generous deadline changes nothing (bit-identical)."""
import time

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


def test_deadline_stops_a_long_run_and_leaves_the_handle_usable(wlb):
    prob = workloads.sphere_3d(seed=1)  # 15360 steps, about 1.2 s
    T = prob["period"]
    with wlb.Solver(prob) as s:
        s.run()  # graphs captured, clocks warm
        s.set_deadline(0.05)
        t0 = time.perf_counter()
        with pytest.raises(wlb.WlbError) as e:
            s.run()
        dt = time.perf_counter() - t0
        assert e.value.status == wlb.WLB_ERR_TIMEOUT
        assert dt < 0.5, dt
        done = s.info().steps_done
        assert 0 < done < prob["n_steps"] and done % T == 0
        s.step(T)  # the handle still steps
        assert s.info().steps_done == done + T
        s.set_deadline(0)
        F = s.run()
    with wlb.Solver(prob) as r:
        assert np.array_equal(r.run(), F)


def test_generous_deadline_is_bit_identical(wlb):
    prob = workloads.problem(3, (128, 32, 32), 2, 16.0, 3.0, (64.25, 16.5, 2.0), cp=0.42, n_surface=60,
                             n_periods=6, n_avg_periods=3)
    with wlb.Solver(prob) as s:
        F0 = s.run()
        s.set_deadline(60.0)
        F1 = s.run()
        hist = s.force_history()
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(wlb.WlbError):
                s.set_deadline(bad)
    assert np.array_equal(F0, F1) and len(hist) == 3
