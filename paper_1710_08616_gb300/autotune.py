"""Autotuner for the launch shapes of the step and ensemble kernels.

It times candidate shapes through the public C ABI on the caller's grid and
state (CUDA events, best of a few repetitions) and keeps the fastest per
(GPU name, operation, domain sizes, field count, precision) in a JSON cache:
  step:      one launch per stage and column pass, with the stage tile rows
             (32 x 4 / 8 / 16 for FP32, 8 for FP64) and the column kernel's
             resident blocks per SM (1..4), the third stage fused with the
             top-down column pass or not; or the persistent dataflow kernel;
  ensemble:  ensemble tile rows (32 x 4 / 8 for FP32, 8 for FP64).
Every shape computes the same arithmetic per cell, so results do not depend
on the choice (a GPU test checks this bit for bit).  The cache file is
$ASUCA_TUNE_CACHE, else ~/.cache/asuca_gb300/tuning.json.
"""
from __future__ import annotations

import json
import os

from . import (FP64, TUNE_COL_BLOCKS_PER_SM, TUNE_ENSEMBLE_TILE_ROWS, TUNE_FUSED_COLUMN, TUNE_STAGE_TILE_ROWS,
               TUNE_STEP_MODE, ensemble_step, ensemble_workspace_bytes, get_tuning, set_tuning, step)

TUNE_STAGE_TILE_ROWS_FP32 = (4, 8, 16)
TUNE_ENS_TILE_ROWS_FP32 = (4, 8)
COL_BLOCKS = (1, 2, 3, 4)


def cache_path() -> str:
    p = os.environ.get("ASUCA_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "asuca_gb300", "tuning.json")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(d: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def step_key(gpu: str, grid) -> str:
    return f"{gpu}|step|{grid.nx}x{grid.ny}x{grid.nz}|F{grid.nfields}|{'fp64' if grid.prec == FP64 else 'fp32'}"


def ensemble_key(gpu: str, grids) -> str:
    sizes = ",".join(f"{g.nx}x{g.ny}" for g in grids)
    g0 = grids[0]
    return f"{gpu}|ensemble|{sizes}|nz{g0.nz}|F{g0.nfields}|{'fp64' if g0.prec == FP64 else 'fp32'}"


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _timed(fn, reps):
    import torch
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def step_candidates(grid):
    """Per-stage launches for every tile height and column-kernel occupancy, with
    the fused third-stage/column path (8-row tiles only) and without it, and the
    persistent dataflow kernel."""
    rows = (8,) if grid.prec == FP64 else TUNE_STAGE_TILE_ROWS_FP32
    out = [{"step_mode": 0, "stage_tile_rows": r, "col_blocks_per_sm": b, "fused_column": 0}
           for r in rows for b in COL_BLOCKS]
    out += [{"step_mode": 0, "stage_tile_rows": 8, "col_blocks_per_sm": b, "fused_column": 1} for b in COL_BLOCKS]
    out.append({"step_mode": 1, "stage_tile_rows": 8, "col_blocks_per_sm": 3, "fused_column": 0})
    return out


def apply_step(grid, cfg: dict) -> None:
    set_tuning(grid, TUNE_STEP_MODE, cfg.get("step_mode", 0))
    set_tuning(grid, TUNE_STAGE_TILE_ROWS, cfg["stage_tile_rows"])
    set_tuning(grid, TUNE_COL_BLOCKS_PER_SM, cfg["col_blocks_per_sm"])
    set_tuning(grid, TUNE_FUSED_COLUMN, cfg.get("fused_column", 1))


def tune_step(grid, state, dt, *, steps: int = 2, reps: int = 3, save: bool = True) -> dict:
    """Time every candidate on a scratch copy of `state`; apply and cache the fastest."""
    import torch
    results = []
    for cfg in step_candidates(grid):
        apply_step(grid, cfg)
        ws = grid.workspace(device=state.rho.device)
        scratch = state.clone()
        step(grid, scratch, dt, 1, workspace=ws)      # warm-up (and one-time launch set-up)
        ms = _timed(lambda: step(grid, scratch, dt, steps, workspace=ws), reps)
        results.append(dict(cfg, ms_per_step=ms / steps))
        del ws, scratch
        torch.cuda.empty_cache()
    best = min(results, key=lambda r: r["ms_per_step"])
    apply_step(grid, best)
    out = {"best": best, "candidates": results}
    if save:
        d = load_cache()
        d[step_key(_gpu_name(), grid)] = out
        save_cache(d)
    return out


def tune_ensemble(grids, states, dts, *, steps: int = 2, reps: int = 3, save: bool = True) -> dict:
    import torch
    rows = (8,) if grids[0].prec == FP64 else TUNE_ENS_TILE_ROWS_FP32
    results = []
    for r in rows:
        for g in grids:
            set_tuning(g, TUNE_ENSEMBLE_TILE_ROWS, r)
        ws = torch.empty(ensemble_workspace_bytes(grids), dtype=torch.uint8, device=states[0].rho.device)
        scratch = [s.clone() for s in states]
        ensemble_step(grids, scratch, dts, 1, workspace=ws)
        ms = _timed(lambda: ensemble_step(grids, scratch, dts, steps, workspace=ws), reps)
        results.append({"ensemble_tile_rows": r, "ms_per_step": ms / steps})
        del ws, scratch
        torch.cuda.empty_cache()
    best = min(results, key=lambda x: x["ms_per_step"])
    for g in grids:
        set_tuning(g, TUNE_ENSEMBLE_TILE_ROWS, best["ensemble_tile_rows"])
    out = {"best": best, "candidates": results}
    if save:
        d = load_cache()
        d[ensemble_key(_gpu_name(), grids)] = out
        save_cache(d)
    return out


def apply_cached_step(grid) -> bool:
    ent = load_cache().get(step_key(_gpu_name(), grid))
    if not ent:
        return False
    apply_step(grid, ent["best"])
    return True


def apply_cached_ensemble(grids) -> bool:
    ent = load_cache().get(ensemble_key(_gpu_name(), grids))
    if not ent:
        return False
    for g in grids:
        set_tuning(g, TUNE_ENSEMBLE_TILE_ROWS, ent["best"]["ensemble_tile_rows"])
    return True


def current(grid) -> dict:
    return {"step_mode": get_tuning(grid, TUNE_STEP_MODE),
            "fused_column": get_tuning(grid, TUNE_FUSED_COLUMN),
            "stage_tile_rows": get_tuning(grid, TUNE_STAGE_TILE_ROWS),
            "col_blocks_per_sm": get_tuning(grid, TUNE_COL_BLOCKS_PER_SM),
            "ensemble_tile_rows": get_tuning(grid, TUNE_ENSEMBLE_TILE_ROWS)}
