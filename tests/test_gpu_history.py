"""Force history (wlb_force_history): the force of every fold of the running
sums (each full sampled period, and a partial one wlb_force folds).  Pinned
against the oracle without a history of its own: a run averaging the last k
periods gives F(k), so the j-th period from the end has the force
j F(j) - (j - 1) F(j - 1) (Eq. 14 is linear in the sums).  Also: the
sample-weighted mean of the history is the force, also with a partial fold in
the middle of a run, and the call is refused before wlb_init."""
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


def test_history_matches_oracle_periods_2d_fp64(wlb):
    n_avg = 4
    prob = workloads.problem(2, (128, 128), 1, 64.0, 8.0, (64.25, 8.5), cp=0.375, n_surface=64,
                             n_periods=6, n_avg_periods=n_avg, precision="f64")
    with wlb.Solver(prob) as s:
        F = s.run()
        hist = s.force_history()
    assert hist.shape == (n_avg, 3)
    Fk = [oracle.run(dict(prob, n_window=k * prob["period"]))["force"] for k in range(1, n_avg + 1)]
    per = [Fk[0]] + [(j + 1) * Fk[j] - j * Fk[j - 1] for j in range(1, n_avg)]  # j-th from the end
    ref = np.array(per[::-1])
    scale = np.abs(ref[:, 1]).max()
    assert np.abs(hist - ref).max() <= 1e-9 * scale, np.abs(hist - ref).max() / scale
    assert np.allclose(hist.mean(axis=0), F, rtol=1e-12, atol=1e-15 * scale)


def test_history_mean_is_the_force_3d_two_step(wlb):
    prob = workloads.problem(3, (128, 32, 32), 2, 16.0, 3.0, (64.25, 16.5, 2.0), cp=0.42, n_surface=60,
                             n_periods=8, n_avg_periods=5)
    with wlb.Solver(prob) as s:
        assert s.info().steps_per_launch == 2
        with pytest.raises(wlb.WlbError):
            s.force_history()  # before wlb_init
        F = s.run()
        hist = s.force_history()
        assert hist.shape == (5, 3)
        scale = np.abs(F).max()
        assert np.abs(hist.mean(axis=0) - F).max() <= 1e-12 * scale
        # partial folds (force() inside a period) are rows with their own counts
        T = prob["period"]
        s.init()
        s.step(prob["n_steps"] - prob["n_window"], sample=False)
        s.step(2 * T + 11, sample=True)
        assert len(s.force_history()) == 2
        s.force()
        s.step(T + 5, sample=True)
        F2 = s.force()
        hist, n = s.force_history(with_samples=True)
        assert list(n) == [T, T, 11, T, 5]
        mean = (hist * n[:, None]).sum(axis=0) / n.sum()
        assert np.abs(mean - F2).max() <= 1e-12 * np.abs(F2).max()
