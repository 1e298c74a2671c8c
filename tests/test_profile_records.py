"""The ncu records bench.py reports (profiles/traffic.json) belong to the
kernels as they are: each record's sources hash to the value stored with it,
so the benchmark line carries the measured DRAM traffic of the dominant
kernel rather than null.  The recorded traffic per cell also stays within a
few percent of the kernels' algorithmic bytes (FP32, 10 fields), the figure
the roofline divides by.  The benchmark's compulsory-floor fraction and its
DRAM rate from the recorded traffic are checked on a report of known figures.
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


def test_floor_and_dram_fractions():
    """The compulsory-floor fraction and the DRAM rate from the recorded
    traffic, on a report shaped like the benchmark's (100 steps of the
    1024x1024x58 workload in 828.7 ms against a 6770.5 GB/s peak)."""
    C, peak, ms = 60817408, 6770.5, 828.7393
    per_cell = {"stage": (92, 96.42), "stage2_factor": (156, 157.18), "stage3_column": (176, 175.81),
                "column": (128, 126.43)}
    kern = {k: {"launches": 100, "algo_bytes_per_launch": a * C, "traffic_bytes_per_launch": t * C}
            for k, (a, t) in per_cell.items()}
    kern["budget_reduce"] = {"launches": 100, "algo_bytes_per_launch": 0.0, "traffic_bytes_per_launch": None}
    out = bench._floor_and_dram(kern, 10, 4, C, ms, 100, peak)
    assert out["floor_bytes_per_cell"] == 92
    assert abs(out["floor_frac"] - 92 * C * 100 / (ms * 1e-3) / 1e9 / peak) < 1e-12
    dram = sum(t for _, t in per_cell.values()) * C * 100 / (ms * 1e-3) / 1e9
    assert abs(out["dram_gbs_ncu"] - dram) < 1e-6 * dram and abs(out["dram_frac_ncu"] - dram / peak) < 1e-12
    kern["stage"]["traffic_bytes_per_launch"] = None          # a kernel without a current record
    assert bench._floor_and_dram(kern, 10, 4, C, ms, 100, peak)["dram_gbs_ncu"] is None
    assert bench._floor_and_dram({}, 10, 4, C, 0.0, 100, peak)["floor_frac"] is None
