"""Checkpoint and resume (wlb_save_state / wlb_load_state): a run stopped at
any step, saved, and continued in a fresh handle gives the force and fields of
the uninterrupted run bit for bit.  Cuts fall inside the unsampled phase and
inside a sampled period (an odd number of samples into it), on the two-step
3D path (FP32, FP16), the 2D path (FP64) and the driven cavity (source phase
follows the restored step index)."""
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


def _problem(case):
    if case == "3d_f32":
        return workloads.problem(3, (128, 32, 32), 2, 16.0, 3.0, (64.25, 16.5, 2.0), cp=0.42, n_surface=60,
                                 n_periods=6, n_avg_periods=3)
    if case == "3d_f16":
        return workloads.problem(3, (256, 24, 32), 2, 16.0, 3.0, (128.25, 12.5, 2.0), cp=0.42, n_surface=60,
                                 n_periods=6, n_avg_periods=3, precision="f16")
    if case == "2d_f64":
        return workloads.problem(2, (128, 128), 1, 64.0, 8.0, (64.25, 8.5), cp=0.375, n_surface=64,
                                 n_periods=4, n_avg_periods=2, precision="f64")
    prob = workloads.problem(2, (128, 35), 1, 64.0, 3.0, (64.0, 14.0), cp=0.375, n_surface=48,
                             n_periods=4, n_avg_periods=2, precision="f64", surface_radius=4.0)
    prob.update(boundary="driven", wall_damping=0.99, source_amplitude=1e-3 / 0.0625)
    return prob


def _schedule(prob):
    """Calls of the whole protocol with two cut points: (steps, sampled) pieces
    and the indices after which a state is saved."""
    T, n_free, n_win = prob["period"], prob["n_steps"] - prob["n_window"], prob["n_window"]
    a = n_free // 2 + 1                      # inside the unsampled phase (odd)
    b = T + 7 if n_win > T + 7 else n_win // 2 + 1  # into a sampled period, odd
    pieces = [(a, False), (n_free - a, False), (b, True), (n_win - b, True)]
    return pieces, (0, 2)                    # save after pieces 0 and 2


@pytest.mark.parametrize("case", ["3d_f32", "3d_f16", "2d_f64", "driven_2d_f64"])
def test_resume_is_bit_identical(wlb, case):
    prob = _problem(case)
    pieces, cuts = _schedule(prob)
    states = {}
    with wlb.Solver(prob) as s:
        s.init()
        for i, (n, smp) in enumerate(pieces):
            s.step(n, sample=smp)
            if i in cuts:
                states[i] = s.save_state()
        F = s.force()
        p1, u1 = s.fields()
        hist = s.force_history()
    assert np.any(F != 0) and len(hist) == prob["n_window"] // prob["period"]
    for cut, state in states.items():
        with wlb.Solver(prob) as r:  # never initialised: the load runs the setup
            r.load_state(state)
            assert r.info().steps_done == sum(n for n, _ in pieces[:cut + 1])
            for n, smp in pieces[cut + 1:]:
                r.step(n, sample=smp)
            assert np.array_equal(r.force(), F), (case, cut)
            q1, v1 = r.fields()
            assert np.array_equal(q1, p1) and np.array_equal(v1, u1), (case, cut)
            assert np.array_equal(r.force_history(), hist), (case, cut)


def test_state_is_checked(wlb):
    prob = _problem("3d_f32")
    with wlb.Solver(prob) as s:
        with pytest.raises(wlb.WlbError):
            s.save_state()  # before wlb_init
        s.init()
        s.step(10)
        state = s.save_state()
    other = dict(prob, radius=prob["radius"] + 0.5)
    with wlb.Solver(other) as r:
        with pytest.raises(wlb.WlbError):
            r.load_state(state)  # saved for other parameters
    with wlb.Solver(prob) as r:
        with pytest.raises(wlb.WlbError):
            r.load_state(state[:-8])  # short
        bad = state.copy()
        bad[0] ^= 1
        with pytest.raises(wlb.WlbError):
            r.load_state(bad)  # foreign format
        r.load_state(state)
        assert r.info().steps_done == 10
