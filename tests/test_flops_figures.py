"""The algorithmic flop figures the bench's roofline uses are the oracle's counts.

bench.py divides RHS_FLOPS_PER_POINT + RK_FLOPS_PER_POINT interior-point flops
by the measured k_rhs time; both constants must be what the flop-counting
build of the oracle reports for one substep of the 128^3 star workload (a
24^3 sub-box at the same grid spacing).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def counts():
    from oracle import count_flops
    return count_flops.count(24)


def test_bench_constants_are_the_oracle_counts(counts):
    import bench
    assert counts["rhs_local_per_interior_point"] == bench.RHS_FLOPS_PER_POINT
    # RK4: stages 0-2 form acc += b k and the next stage input (128 flops per
    # point over 32 fields), the last stage only the final combination (64).
    assert counts["rk_stage0_per_interior_point"] == 128.0
    assert bench.RK_FLOPS_PER_POINT == (3 * 128.0 + 64.0) / 4.0


def test_pointwise_and_interface_counts(counts):
    # The pointwise flux of one direction is data independent; con2prim and
    # MP5 depend on the data (Brent's iterations, limiter branches).
    assert counts["flux_per_point_direction"] == 433.0
    assert 300.0 < counts["c2p_per_ghosted_point"] < 600.0
    assert 600.0 < counts["iflux_per_interface"] < 1000.0
