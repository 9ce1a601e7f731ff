"""Host-side pieces of bench.py that need no GPU: the launch and byte counts
behind the roofline line, and the committed DRAM-traffic record that the
headline's roofline quotes (it must have been taken on the kernels' current
source, or the bench line reports its traffic as null)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("K, fuse, launches", [(25, 1, 25), (25, 2, 13), (24, 2, 12), (25, 3, 9), (25, 4, 7)])
def test_smoothing_launch_count(K, fuse, launches):
    assert bench.smoothing_launches(K, fuse) == launches


def test_diffusion_launch_reads_and_writes_the_mesh_once():
    P = 128 ** 3
    per_launch, n = bench.algorithmic_bytes("smooth", 4, P, 32768, 25, fuse=2)
    assert per_launch == 2 * 4 * P and n == 13


@pytest.mark.parametrize("kernel", ["k_diffuse4", "k_diffuse4x2"])
def test_headline_traffic_record_matches_the_kernel_source(kernel):
    assert bench.kernel_source_sha(kernel) is not None
    t = bench.recorded_traffic(kernel, "nacl_32k", "mixed")
    assert t is not None, f"recapture the DRAM traffic of {kernel}: its source changed"
    # one 8.4 MB FP32 mesh read per launch at 128^3 (the other stays in L2)
    assert 0.9 * 4 * 128 ** 3 < t < 1.1 * 4 * 128 ** 3
