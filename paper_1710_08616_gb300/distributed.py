"""Ensemble members across ranks, one GPU per rank.

Members are independent problems, so a multi-GPU ensemble shards whole
members over the ranks and advances each rank's share with one persistent
launch (asuca_ensemble_step); nothing crosses GPUs inside a step.  The only
collective is the gather of the members' FP64 budgets after the call.

  shard_members(cells, world)       -> member indices per rank (longest first)
  gather_budgets(local, M, nb, group) -> (M, nb) float64 budgets on every rank
  ensemble_step_sharded(...)        -> advance this rank's members, gather budgets

Single domains are not decomposed: every rank of a multi-GPU run advances its
own replica (weak scaling), as the benchmark does.
"""
from __future__ import annotations

import numpy as np


def shard_members(cells, world: int) -> list[list[int]]:
    """Assign members (given their cell counts) to `world` ranks: largest member
    first to the rank with the least work so far, ties to the lower rank and, for
    equal sizes, the lower member index first.  Deterministic: every rank
    computes the same assignment from the same sizes.  Each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cells = [int(c) for c in cells]
    if any(c < 0 for c in cells):
        raise ValueError("cell counts must be non-negative")
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for m in sorted(range(len(cells)), key=lambda m: (-cells[m], m)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(m)
        load[r] += cells[m]
    return [sorted(v) for v in out]


def gather_budgets(local: dict, nmembers: int, nbudget: int, group=None):
    """Every rank contributes the budgets of its own members ({member: vector of
    nbudget doubles}); returns the (nmembers, nbudget) float64 array on every rank.
    Each entry has exactly one contributor and the others add 0.0, so the sum
    all-reduce is exact and the result does not depend on the reduction order."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    buf = torch.zeros((nmembers, nbudget), dtype=torch.float64, device=dev)
    for m, v in local.items():
        t = torch.as_tensor(np.asarray(v, dtype=np.float64)).reshape(-1)
        if t.numel() != nbudget:
            raise ValueError(f"member {m}: {t.numel()} budgets, expected {nbudget}")
        buf[m] = t.to(dev)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf.cpu().numpy()


def ensemble_step_sharded(grids, states, dts, nsteps: int, *, group=None, workspace=None, step=None):
    """Advance this rank's share of the ensemble (members from shard_members over
    all members' cells) with one persistent launch and return every member's
    budgets, gathered over the ranks.  `grids`, `states`, `dts` list all members
    on every rank; only this rank's members are touched.  `workspace`, if given,
    is sized for this rank's members (ensemble_workspace_bytes of that subset).
    `step` replaces asuca_ensemble_step (same arguments and result); it lets the
    host-side sharding and gather run on CPU ranks in tests."""
    import torch.distributed as dist
    if step is None:
        from . import ensemble_step as step

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    cells = [g.nx * g.ny * g.nz for g in grids]
    mine = shard_members(cells, world)[rank]
    nb = grids[0].nfields + 1
    local = {}
    if mine:
        bud = step([grids[m] for m in mine], [states[m] for m in mine], [dts[m] for m in mine],
                   nsteps, workspace=workspace, budgets=True)
        # the copy to the host waits for the step on its stream
        b = bud.cpu().numpy().reshape(len(mine), nb)
        local = {m: b[q] for q, m in enumerate(mine)}
    return gather_budgets(local, len(grids), nb, group)
