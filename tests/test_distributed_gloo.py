"""Multi-rank host logic on CPU (gloo, world size 2): sharding ensemble members
over ranks, the exact FP64 budget gather, ensemble_step_sharded with a
stand-in member step (each rank steps only its own members; every rank ends
with every member's budgets), and the benchmark's max-over-ranks timing.  The
GPU-side step of each rank is the single-GPU path tested elsewhere (and
ensemble_step_sharded itself at world size 1 on the GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_1710_08616_gb300.distributed import shard_members


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_members_covers_each_member_once_and_balances():
    import gen
    sizes = gen.ensemble_sizes()
    cells = [n * n * 58 for n in sizes]
    for world in (1, 2, 3, 4, 8, 40):
        sh = shard_members(cells, world)
        assert len(sh) == world
        flat = sorted(m for r in sh for m in r)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[m] for m in r) for r in sh]
        # greedy largest-first: no rank exceeds the mean load by more than the largest member
        assert max(loads) <= sum(cells) / world + max(cells)
        assert sh == shard_members(cells, world)     # deterministic


def test_shard_members_small_cases():
    assert shard_members([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert shard_members([10, 1, 1, 1], 2) == [[0], [1, 2, 3]]
    assert shard_members([], 3) == [[], [], []]
    assert shard_members([3], 2) == [[0], []]
    with pytest.raises(ValueError):
        shard_members([1], 0)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1710_08616_gb300.distributed import gather_budgets
        import bench
        M, nb = 7, 5
        rng = np.random.default_rng(99)
        full = rng.standard_normal((M, nb)) * 10.0 ** rng.integers(-20, 20, (M, nb))
        sh = shard_members([(m * 37) % 11 + 1 for m in range(M)], world)
        got = gather_budgets({m: full[m] for m in sh[rank]}, M, nb)
        tmax = bench._max_over_ranks(world, 1.5 + rank)
        q.put((rank, got.tobytes() == full.tobytes(), tmax))
    finally:
        dist.destroy_process_group()


def test_gloo_world2_budget_gather_and_max_over_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, exact, tmax in res:
        assert exact, f"rank {rank}: gathered budgets differ"
        assert tmax == 2.5


def _sharded_worker(rank, world, port, q):
    import types
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1710_08616_gb300.distributed import ensemble_step_sharded
        sizes = [64, 97, 40, 71, 33, 120, 58]
        nf = 6
        grids = [types.SimpleNamespace(nx=n, ny=n, nz=12, nfields=nf) for n in sizes]
        states = [{"member": m, "steps": 0} for m in range(len(sizes))]
        dts = [10.0 + m for m in range(len(sizes))]
        seen = []

        def fake_step(gs, sts, ds, nsteps, workspace=None, budgets=False):
            # stand-in for the persistent launch: advance each given member and
            # return its budgets as a deterministic function of the member
            assert budgets
            out = []
            for g, st, dt in zip(gs, sts, ds):
                st["steps"] += nsteps
                seen.append(st["member"])
                m = st["member"]
                out.append([g.nx * g.ny * g.nz * 1e-3 + m, dt * nsteps] + [m * 0.1 + f for f in range(nf - 1)])
            return torch.tensor(out, dtype=torch.float64).reshape(-1)

        got = ensemble_step_sharded(grids, states, dts, 3, step=fake_step)
        q.put((rank, sorted(seen), [st["steps"] for st in states], got.tobytes()))
    finally:
        dist.destroy_process_group()


def test_gloo_world2_ensemble_step_sharded_host_logic():
    import multiprocessing as mp
    from paper_1710_08616_gb300.distributed import shard_members
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [64, 97, 40, 71, 33, 120, 58]
    share = shard_members([n * n * 12 for n in sizes], 2)
    nf = 6
    expect = np.array([[n * n * 12 * 1e-3 + m, (10.0 + m) * 3] + [m * 0.1 + f for f in range(nf - 1)]
                       for m, n in enumerate(sizes)])
    for rank, seen, steps, got in res:
        assert seen == share[rank]                      # this rank stepped exactly its members
        assert steps == [3 if m in share[rank] else 0 for m in range(len(sizes))]
        assert np.frombuffer(got, dtype=np.float64).reshape(expect.shape).tolist() == expect.tolist()


# ---------------------------------------------------------------- decomposed domain: halo exchange

def _np_block(field, decomp, r):
    """A host-side stand-in of a block: its padded buffer [T][nz][ny+4][nx+8]
    (interior at (j+2, i+4)) holding its part of the global field, ghosts NaN."""
    import types
    i0, i1, j0, j1 = decomp.extent(r)
    T, nz = field.shape[0], field.shape[1]
    nx, ny = i1 - i0, j1 - j0
    pad = np.full((T, nz, ny + 4, nx + 8), np.nan)
    pad[:, :, 2:ny + 2, 4:nx + 4] = field[:, :, j0:j1, i0:i1]
    grid = types.SimpleNamespace(nx=nx, ny=ny, nz=nz, nfields=T + 1)
    return types.SimpleNamespace(grid=grid, pad=pad, extent=(i0, i1, j0, j1))


def _np_pack(b):
    """The halo layout's packed strips: W cells i = c, E i = nx-2+c, S j = c, N j = ny-2+c."""
    import torch
    nx, ny, p = b.grid.nx, b.grid.ny, b.pad
    w = np.moveaxis(p[:, :, 2:ny + 2, 4:6], 3, 2)
    e = np.moveaxis(p[:, :, 2:ny + 2, nx + 2:nx + 4], 3, 2)
    s = p[:, :, 2:4, 4:nx + 4]
    n = p[:, :, ny:ny + 2, 4:nx + 4]
    return torch.tensor(np.concatenate([a.reshape(-1) for a in (w, e, s, n)]))


def _np_unpack(b, t):
    """Received strips into the ghosts: W i = c-2, E i = nx+c, S j = c-2, N j = ny+c."""
    from paper_1710_08616_gb300.distributed import halo_strips
    nx, ny, nz, T = b.grid.nx, b.grid.ny, b.grid.nz, b.grid.nfields - 1
    w, e, s, n = (x.numpy() for x in halo_strips(t, T, nz, ny, nx))
    b.pad[:, :, 2:ny + 2, 2:4] = np.moveaxis(w.reshape(T, nz, 2, ny), 2, 3)
    b.pad[:, :, 2:ny + 2, nx + 4:nx + 6] = np.moveaxis(e.reshape(T, nz, 2, ny), 2, 3)
    b.pad[:, :, 0:2, 4:nx + 4] = s.reshape(T, nz, 2, nx)
    b.pad[:, :, ny + 2:ny + 4, 4:nx + 4] = n.reshape(T, nz, 2, nx)


def _check_ghosts(field, b):
    """Every ghost of the cross equals the periodic continuation of the global field."""
    i0, i1, j0, j1 = b.extent
    nx, ny = i1 - i0, j1 - j0
    gx, gy = field.shape[3], field.shape[2]
    cols = [(i0 + i) % gx for i in (-2, -1, nx, nx + 1)]
    for q, i in zip(cols, (2, 3, nx + 4, nx + 5)):
        assert np.array_equal(b.pad[:, :, 2:ny + 2, i], field[:, :, j0:j1, q])
    rows = [(j0 + j) % gy for j in (-2, -1, ny, ny + 1)]
    for q, j in zip(rows, (0, 1, ny + 2, ny + 3)):
        assert np.array_equal(b.pad[:, :, j, 4:nx + 4], field[:, :, q, i0:i1])


def _field():
    return np.random.default_rng(5).standard_normal((3, 4, 11, 13))


def test_halo_exchange_single_process_blocks_continue_the_plane_periodically():
    from paper_1710_08616_gb300.distributed import Decomposition, exchange_halos
    f = _field()
    for px, py in ((1, 1), (2, 1), (1, 2), (3, 2), (2, 3)):
        d = Decomposition(f.shape[3], f.shape[2], px, py)
        blocks = {r: _np_block(f, d, r) for r in range(d.nblocks)}
        exchange_halos(blocks, d, 0, pack=_np_pack, unpack=_np_unpack)
        for b in blocks.values():
            _check_ghosts(f, b)


def _halo_worker(rank, world, port, px, py, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1710_08616_gb300.distributed import Decomposition, exchange_halos
        f = _field()
        d = Decomposition(f.shape[3], f.shape[2], px, py)
        blocks = {rank: _np_block(f, d, rank)}
        exchange_halos(blocks, d, 1, pack=_np_pack, unpack=_np_unpack)
        _check_ghosts(f, blocks[rank])
        q.put((rank, True))
    except AssertionError:
        q.put((rank, False))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
def test_gloo_world2_halo_exchange(px, py):
    """Two ranks, one block each: with two blocks along a direction, a rank's
    west and east neighbour is the same rank, so both directions' messages
    travel between the same pair (one direction at a time)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_halo_worker, args=(r, 2, port, px, py, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True), (1, True)]
