"""Batched ensembles (wlb_batch_*) against single-lattice runs and the oracle."""
import math

import numpy as np
import pytest

import oracle
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


def _members_3d(precision="f32"):
    # ragged rows (40, 96, 64, 160 cells): the widest needs two 128-cell chunks,
    # so every row runs the two-chunk code with idle lanes; uneven periods and
    # run lengths (the longest lattice keeps stepping after the others stop)
    specs = [((40, 36, 32), 16.0, 4.0, 30, 10), ((96, 24, 32), 16.0, 3.0, 20, 5),
             ((64, 24, 24), 24.0, 3.5, 12, 4), ((160, 24, 32), 32.0, 3.0, 6, 2)]
    out = []
    for i, (n, lam, R, per, avg) in enumerate(specs):
        c = (n[0] / 2 + 0.25, n[1] / 2 - 0.5, lam / 8 + 0.125 * i)
        out.append(workloads.problem(3, n, 2, lam, R, c, cp=0.25 * (0.8 + 0.3 * i), n_surface=100 + 50 * i,
                                     n_periods=per, n_avg_periods=avg, precision=precision))
    return out


def test_batch_3d_matches_single_and_oracle(wlb):
    probs = _members_3d()
    with wlb.Batch(probs) as b:
        info = b.info()
        assert info.count == 4 and info.row_chunks == 2
        F = b.run()
        F2 = b.run()  # a second run from a fresh setup gives the same forces
    assert np.array_equal(F, F2)
    for i, p in enumerate(probs):
        with wlb.Solver(p) as s:
            Fs = s.run()
        assert np.array_equal(F[i], Fs), (i, F[i], Fs)
    o = oracle.run(probs[0])["force"]
    assert abs(F[0, 2] - o[2]) <= 1e-3 * abs(o[2])


@pytest.mark.parametrize("precision", ["f32", "f64", "f16"])
def test_batch_2d_ragged(wlb, precision):
    specs = [((48, 32), 16.0, 3.0, 8), ((192, 96), 48.0, 6.0, 4), ((24, 64), 32.0, 4.0, 5)]
    if precision == "f16":  # 16-byte rows of FP16 need nx % 8 == 0
        specs[2] = ((32, 64), 32.0, 4.0, 5)
    probs = [workloads.problem(2, n, 1, lam, R, (n[0] / 2 + 0.25, lam / 8), cp=0.32, n_surface=40,
                               n_periods=per, n_avg_periods=2, precision=precision)
             for (n, lam, R, per) in specs]
    with wlb.Batch(probs) as b:
        # even lengths and rows of at most 64 vectors: two steps per launch,
        # except FP64, whose 192-cell rows need three chunks per lane
        two = b.info().steps_per_launch == 2
        assert two == (precision != "f64")
        F = b.run()
        if two:
            # the autotuner times several rows-per-warp chunk heights; any gives the same bits
            best = b.autotune(steps_per_trial=4)
            assert best["plans_tried"] >= 2 and 1 <= best["z_chunk"] <= 32
            assert np.array_equal(b.run(), F)
            b.set_two_step(False)
            assert np.array_equal(b.run(), F)
    # the batch samples 2D points one thread each, summing the stencil in the
    # order of the single-lattice warp reduction: the same bits
    for i, p in enumerate(probs):
        with wlb.Solver(p) as s:
            Fs = s.run()
        assert np.array_equal(F[i], Fs), (i, F[i], Fs)
    if precision == "f32":  # the two-step 2D batch against the FP64 oracle directly
        o = oracle.run(probs[1])["force"]
        assert abs(F[1, 1] - o[1]) <= 1e-3 * abs(o[1]), (F[1], o)


def test_batch_autotune_and_member_without_window(wlb):
    probs = _members_3d()
    probs[1] = dict(probs[1], n_window=0)  # no averaging window: zero force, still stepped
    with wlb.Batch(probs) as b:
        best = b.autotune(steps_per_trial=8)
        assert best["threads_per_block"] in (128, 256) and best["blocks_per_sm"] in (2, 4, 8, 16)
        info = b.info()
        assert info.threads_per_block == best["threads_per_block"]
        F = b.run()
    assert np.array_equal(F[1], np.zeros(3))
    with wlb.Solver(probs[0]) as s:
        Fs = s.run()
    assert abs(F[0, 2] - Fs[2]) <= 1e-6 * abs(Fs[2])


def _members_two_step(precision="f32"):
    # rows of 96, 64, 160 and 128 cells (multiples of 16: two steps per launch),
    # uneven periods and run lengths, one member without an averaging window
    specs = [((96, 24, 32), 16.0, 3.0, 20, 5), ((64, 24, 24), 24.0, 3.5, 12, 4),
             ((160, 24, 32), 32.0, 3.0, 6, 2), ((128, 40, 32), 16.0, 4.0, 16, 0)]
    out = []
    for i, (n, lam, R, per, avg) in enumerate(specs):
        c = (n[0] / 2 + 0.25, n[1] / 2 - 0.5, lam / 8 + 0.125 * i)
        out.append(workloads.problem(3, n, 2, lam, R, c, cp=0.25 * (0.8 + 0.3 * i), n_surface=100 + 50 * i,
                                     n_periods=per, n_avg_periods=avg, precision=precision))
    return out


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_batch_two_steps_per_launch_bit_identical(wlb, precision):
    """The batched two-step launch (one slab launch over every lattice, batched
    sampling of both steps) gives the same bits as one step per launch and as
    every lattice run alone."""
    probs = _members_two_step(precision)
    with wlb.Batch(probs) as b:
        info = b.info()
        assert info.steps_per_launch == 2 and info.total_ctas > 0
        F2 = b.run()
        b.set_two_step(False)
        assert b.info().steps_per_launch == 1
        F1 = b.run()
        b.set_two_step(True)
        best = b.autotune(steps_per_trial=8)
        assert best["blocks_per_sm"] == 1 and best["ms_per_step"] > 0
        # plans tried: z-chunk length x slab-height cap x lane layout, fastest kept
        assert best["plans_tried"] > 4
        assert best["z_chunk"] in (16, 24, 32, 48, 64, 96, 1 << 20) and best["slab_rows_cap"] in (0, 8, 5)
        assert best["one_chunk_per_lane"] in (0, 1) and best["staging_warp"] in (0, 1)
        F2b = b.run()
    assert np.array_equal(F2, F1) and np.array_equal(F2, F2b)
    assert np.array_equal(F2[3], np.zeros(3))  # no averaging window
    for i, p in enumerate(probs[:3]):
        with wlb.Solver(p) as s:
            Fs = s.run()
        assert np.array_equal(F2[i], Fs), (i, F2[i], Fs)
    if precision == "f32":  # and against the FP64 oracle directly (one- and two-chunk lattices)
        for i in (0, 2):
            o = oracle.run(probs[i])["force"]
            ax = probs[i]["wave_axis"]
            assert abs(F2[i, ax] - o[ax]) <= 1e-3 * abs(o[ax]), (i, F2[i], o)


def test_batch_two_step_unavailable(wlb):
    probs = _members_3d()  # a 40-cell row: not a whole number of 16 cells
    with wlb.Batch(probs) as b:
        assert b.info().steps_per_launch == 1
        with pytest.raises(wlb.WlbError):
            b.set_two_step(True)


def test_batch_rejects_mixed_or_unsupported(wlb):
    p3 = _members_3d()[0]
    p2 = workloads.problem(2, (48, 32), 1, 16.0, 3.0, (24.0, 2.0), cp=0.3, n_surface=8,
                           n_periods=2, n_avg_periods=1)
    with pytest.raises(wlb.WlbError):
        wlb.Batch([p3, p2])
    with pytest.raises(wlb.WlbError):
        wlb.Batch([p3, dict(p3, precision="f64")])
    wide = workloads.problem(2, (1024, 32), 1, 16.0, 3.0, (512.0, 2.0), cp=0.3, n_surface=8,
                             n_periods=2, n_avg_periods=1)  # 1024 FP32 cells > 4 chunks
    with pytest.raises(wlb.WlbError):
        wlb.Batch([wide])
