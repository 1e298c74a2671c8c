"""The ncu records bench.py reports (profiles/traffic.json) belong to the
kernels as they are: each record's sources hash to the value stored with it,
so the benchmark line carries the measured DRAM traffic of the dominant
kernel rather than null.  The recorded traffic per cell also stays within a
few percent of the kernels' algorithmic bytes (FP32, 10 fields), the figure
the roofline divides by.
"""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# algorithmic bytes per cell at F = 10, 4-byte values (the split column pass):
# stage 1 (2F+3) s; stage 2 (3F+3) s + 3 doubles; stage 3 (2F+4) s + F doubles;
# back substitution (F+1) doubles + F s
F, S = 10, 4
ALGO = {"stage": (2 * F + 3) * S, "stage2_factor": (3 * F + 3) * S + 24,
        "stage3_column": (2 * F + 4) * S + 8 * F, "column": (F + 1) * 8 + F * S}


def _records():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        return {k: v for k, v in json.load(fh).items() if k != "about"}


@pytest.mark.parametrize("kernel", sorted(_records()))
def test_record_matches_the_current_sources(kernel):
    key = "bytes_per_cell" if "bytes_per_cell" in _records()[kernel] else "fp64_inst_per_cell"
    assert bench._recorded(kernel, key, 1) is not None, f"{kernel}: sources changed since the capture"


@pytest.mark.parametrize("kernel", sorted(ALGO))
def test_recorded_traffic_is_close_to_the_algorithmic_bytes(kernel):
    per_cell = bench._recorded_traffic(kernel, 1)
    assert per_cell is not None
    assert 0.95 * ALGO[kernel] <= per_cell <= 1.1 * ALGO[kernel], (kernel, per_cell, ALGO[kernel])
