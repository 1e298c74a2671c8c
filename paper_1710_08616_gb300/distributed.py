"""Multi-GPU paths: ensemble members across ranks, and one domain decomposed
into horizontal blocks that exchange halos.

Ensemble members are independent problems, so a multi-GPU ensemble shards
whole members over the ranks and advances each rank's share with one
persistent launch (asuca_ensemble_step); nothing crosses GPUs inside a step.
The only collective is the gather of the members' FP64 budgets after the call.

  shard_members(cells, world)       -> member indices per rank (longest first)
  gather_budgets(local, M, nb, group) -> (M, nb) float64 budgets on every rank
  ensemble_step_sharded(...)        -> advance this rank's members, gather budgets

One domain decomposed into px x py horizontal blocks (Sec. 1.1: ASUCA's GPU
version splits the horizontal plane into blocks that communicate halos;
Sec. 2.2: halo updates every time step).  Each block is an open domain of the
library (asuca_open_*): before every RK stage its stage input's two ghost
columns and rows are filled with its neighbours' edge strips (width 2, the
reach of the Koren stencil; the stencil is a cross, so no corners), the
periodic domain's wrap becoming a wrap of the block grid.  The column pass
needs no exchange; the blocks' budgets are summed at the end.

  Decomposition(nx, ny, px, py)     -> block extents and neighbours
  exchange_halos(blocks, decomp, buffer, group)  -> ghosts of every owned block
  step_decomposed(blocks, decomp, dt, nsteps, group) -> advance, summed budgets

A process owns one block per rank in a multi-process run, or several blocks
(exchanged by device copies) when the blocks share a device.
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


# ---------------------------------------------------------------- decomposed domain

W, E, S, N = 0, 1, 2, 3
_OPPOSITE = {W: E, E: W, S: N, N: S}


class Decomposition:
    """px x py blocks of an nx x ny periodic plane; block r sits at
    (r % px, r // px).  Block sizes differ by at most one cell per direction."""

    def __init__(self, nx: int, ny: int, px: int, py: int):
        if px < 1 or py < 1 or px > nx or py > ny:
            raise ValueError("bad block counts")
        self.nx, self.ny, self.px, self.py = nx, ny, px, py
        self.xs = _split(nx, px)
        self.ys = _split(ny, py)

    @property
    def nblocks(self) -> int:
        return self.px * self.py

    def coords(self, r: int):
        return r % self.px, r // self.px

    def rank(self, rx: int, ry: int) -> int:
        return (ry % self.py) * self.px + (rx % self.px)

    def extent(self, r: int):
        """(i0, i1, j0, j1) of block r"""
        rx, ry = self.coords(r)
        return self.xs[rx] + self.ys[ry]

    def neighbour(self, r: int, d: int) -> int:
        rx, ry = self.coords(r)
        dx, dy = {W: (-1, 0), E: (1, 0), S: (0, -1), N: (0, 1)}[d]
        return self.rank(rx + dx, ry + dy)


def _split(n, parts):
    base, extra = divmod(n, parts)
    out, s = [], 0
    for p in range(parts):
        e = s + base + (1 if p < extra else 0)
        out.append((s, e))
        s = e
    return out


def halo_strips(h, nt: int, nz: int, ny: int, nx: int):
    """(W, E, S, N) views of a flat halo-layout tensor of a block of nx x ny x nz
    with nt transported fields: two strips of nt*nz*2*ny values, two of nt*nz*2*nx."""
    sw, ss = nt * nz * 2 * ny, nt * nz * 2 * nx
    return h[:sw], h[sw:2 * sw], h[2 * sw:2 * sw + ss], h[2 * sw + ss:2 * sw + 2 * ss]


def exchange_halos(blocks, decomp: Decomposition, buffer: int, group=None, *, pack=None, unpack=None):
    """Fill the ghosts of stage buffer `buffer` of every block this process owns.

    blocks: {rank: block}; a block has .grid (nx, ny, nz, nfields) and, for the
    default pack/unpack (asuca_halo_pack, asuca_halo_unpack), .workspace.
    Every block sends its packed strip d (W, E, S, N) to its neighbour in
    direction d, which stores it as its received strip opposite(d); one
    direction at a time, so each pair of ranks has at most one message in
    flight per direction.  Blocks of this process exchange by copies;
    others by torch.distributed point-to-point messages (NCCL between GPUs,
    gloo on CPU).  pack(block) -> flat tensor and unpack(block, tensor)
    replace the library calls (host-side tests)."""
    import torch
    if pack is None:
        from . import halo_count, halo_pack

        def pack(b):
            t = torch.empty(halo_count(b.grid), dtype=b.grid.torch_dtype, device=b.workspace.device)
            halo_pack(b.grid, b.workspace, buffer, t)
            return t
    if unpack is None:
        from . import halo_unpack

        def unpack(b, t):
            halo_unpack(b.grid, b.workspace, buffer, t)

    send = {r: pack(b) for r, b in blocks.items()}
    recv = {r: torch.empty_like(t) for r, t in send.items()}
    shape = lambda r: (blocks[r].grid.nfields - 1, blocks[r].grid.nz, blocks[r].grid.ny, blocks[r].grid.nx)
    sstr = {r: halo_strips(t, *shape(r)) for r, t in send.items()}
    rstr = {r: halo_strips(t, *shape(r)) for r, t in recv.items()}
    for d in (W, E, S, N):
        o = _OPPOSITE[d]
        ops = []
        for r in blocks:
            dst = decomp.neighbour(r, d)
            if dst in blocks:
                rstr[dst][o].copy_(sstr[r][d])
            else:
                import torch.distributed as dist
                ops.append(dist.P2POp(dist.isend, sstr[r][d], dst, group))
            src = decomp.neighbour(r, o)
            if src not in blocks:
                import torch.distributed as dist
                ops.append(dist.P2POp(dist.irecv, rstr[r][o], src, group))
        if ops:
            import torch.distributed as dist
            for req in dist.batch_isend_irecv(ops):
                req.wait()
    for r, b in blocks.items():
        unpack(b, recv[r])


class Block:
    """One block of a decomposed domain: its grid, its state (open-domain face
    fluxes), its open-domain workspace and a budgets vector."""

    def __init__(self, grid, state, workspace=None):
        import torch
        from . import open_workspace
        self.grid, self.state = grid, state
        self.workspace = open_workspace(grid, device=state.rho.device) if workspace is None else workspace
        self.budgets = torch.empty(grid.nfields + 1, dtype=torch.float64, device=state.rho.device)


def step_decomposed(blocks, decomp: Decomposition, dt: float, nsteps: int, group=None, *, tendencies=None):
    """Advance every owned block (a {rank: Block} dict) by nsteps RK3 steps with
    a halo exchange before each stage, and return the domain's budgets (the sum
    over all blocks of every rank; an all-reduce when other ranks own blocks)."""
    import torch
    from . import open_prepare, open_stage
    for n in range(nsteps):
        for b in blocks.values():
            open_prepare(b.grid, b.state, b.workspace, first=(n == 0))
        for stage in range(3):
            exchange_halos(blocks, decomp, stage, group)
            for r, b in blocks.items():
                bud = b.budgets if (stage == 2 and n == nsteps - 1) else None
                td = None if tendencies is None else tendencies[r]
                open_stage(b.grid, b.state, dt, stage, b.workspace, tendencies=td, budgets=bud)
    if nsteps == 0:
        return None
    total = torch.zeros_like(next(iter(blocks.values())).budgets)
    for r in sorted(blocks):
        total += blocks[r].budgets
    if len(blocks) < decomp.nblocks:
        import torch.distributed as dist
        dev = total.device if dist.get_backend(group) == "nccl" else torch.device("cpu")
        t = total.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        total = t.to(total.device)
    return total
