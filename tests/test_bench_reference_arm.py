"""bench.py --impl reference: the oracle sample is sized to the time budget and reports the contract's
keys (host logic only, small grids, runs on the CPU)."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_sizes_the_sample_to_the_budget():
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(steps=3, warmup=1, oracle_n=24, op="AFB_R", n=256, gpus=1)
    line = bench.reference_arm(args, budget_s=1e-6)   # nothing fits: the smallest grid is taken
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1
    assert "16^3" in line["config"]["workload"] and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    line = bench.reference_arm(args, budget_s=1e6)    # everything fits: the largest allowed grid
    assert "24^3" in line["config"]["workload"]
