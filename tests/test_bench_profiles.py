"""bench.py reports the update kernel's DRAM traffic from the committed ncu
summaries only when they were taken on the current kernel source.  These
checks fail when a kernel changes without a new capture, and check the lookup
itself (a foreign source hash gives no traffic)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

@pytest.mark.parametrize("steps_per_launch,edge", [(1, 256), (2, 256), (2, 512)])
def test_committed_profile_matches_current_kernel(steps_per_launch, edge):
    traffic = bench._traffic(bench._kernel_sha(steps_per_launch), steps_per_launch, edge)
    assert traffic is not None, "kernel source changed since its profile was captured"
    # every population read and written once per launch, plus the class byte:
    # the measured bytes lie within a few per cent of 57 B per cell
    algorithmic = 57.0 * edge ** 3
    assert 0.9 * algorithmic < traffic < 1.1 * algorithmic


@pytest.mark.parametrize("edge", [256, 512])
def test_committed_fp16_profile_matches_current_kernel(edge):
    traffic = bench._traffic(bench._kernel_sha(2), name=bench._profile_name(2, edge, "f16"))
    assert traffic is not None, "kernel source changed since its profile was captured"
    algorithmic = 29.0 * edge ** 3  # FP16 populations read and written once per launch, plus the class byte
    assert 0.85 * algorithmic < traffic < 1.1 * algorithmic


def test_committed_ensemble_profile_matches_current_kernel():
    traffic = bench._traffic(bench._kernel_sha(2), name="batch_update2_d3q7_f32_ensemble64.md")
    assert traffic is not None, "kernel source changed since its profile was captured"
    assert 0.95 * 7.9287e9 < traffic < 1.1 * 7.9287e9  # 57 B x 139.1 M cells per two-step pass


def test_committed_ensemble2d_profile_matches_current_kernel():
    traffic = bench._traffic(bench._kernel_sha(2, "wlb_two_step_2d.cu"), name="batch2d_update2_d2q5_f32_ensemble512.md")
    assert traffic is not None, "kernel source changed since its profile was captured"
    assert 0.9 * 7.738e8 < traffic < 1.1 * 7.738e8  # 41 B x 512 x 192^2 cells per two-step launch


def test_foreign_source_hash_gives_no_traffic():
    assert bench._traffic("0" * 64, 2) is None
    assert bench._traffic("0" * 64, 1) is None
