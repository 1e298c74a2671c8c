"""Autotuner bookkeeping on the CPU: cache keys and the JSON round trip."""
import os

from paper_1710_08616_gb300 import autotune


class _G:
    def __init__(self, nx, ny, nz, F, prec):
        self.nx, self.ny, self.nz, self.nfields, self.prec = nx, ny, nz, F, prec


def test_keys_identify_gpu_sizes_fields_and_precision():
    k1 = autotune.step_key("NVIDIA GB300", _G(1024, 1024, 58, 10, 1))
    k2 = autotune.step_key("NVIDIA GB300", _G(1024, 1024, 58, 10, 0))
    k3 = autotune.step_key("Other", _G(1024, 1024, 58, 10, 1))
    assert len({k1, k2, k3}) == 3 and "1024x1024x58" in k1 and "F10" in k1
    e = autotune.ensemble_key("NVIDIA GB300", [_G(64, 64, 58, 6, 1), _G(80, 80, 58, 6, 1)])
    assert "64x64,80x80" in e and "ensemble" in e


def test_cache_round_trip(tmp_path, monkeypatch):
    path = str(tmp_path / "sub" / "tuning.json")
    monkeypatch.setenv("ASUCA_TUNE_CACHE", path)
    assert autotune.load_cache() == {}
    d = {"a|step|x": {"best": {"stage_tile_rows": 8, "col_blocks_per_sm": 3, "ms_per_step": 1.0}}}
    autotune.save_cache(d)
    assert os.path.exists(path)
    assert autotune.load_cache() == d
    with open(path, "w") as fh:
        fh.write("not json")
    assert autotune.load_cache() == {}


def test_candidates():
    c32 = autotune.step_candidates(_G(64, 64, 10, 5, 1))
    c64 = autotune.step_candidates(_G(64, 64, 10, 5, 0))
    assert {c["stage_tile_rows"] for c in c32} == {4, 8, 16}
    assert {c["stage_tile_rows"] for c in c64} == {8}
    assert {c["col_blocks_per_sm"] for c in c32} == {1, 2, 3, 4}
    assert {c["step_mode"] for c in c32} == {0, 1}
    assert {c["fused_column"] for c in c32} == {0, 1}
    assert all(c["stage_tile_rows"] == 8 and c["step_mode"] == 0 for c in c32 if c["fused_column"])
