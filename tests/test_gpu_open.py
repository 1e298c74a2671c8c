"""Open lateral boundaries on the GPU (asuca_open_*, asuca_halo_*, asuca_step_open).

* A domain split into px x py blocks on one device, the blocks exchanging
  two-wide halos before every RK stage (pack, copy to the neighbour, unpack),
  advances exactly as the periodic single-domain step: fields bit for bit,
  budgets to rounding (they are summed block by block).  1 x 1 is the
  periodic domain through the open path; ragged and uneven blocks, every
  limiter, with and without forcing, the fused and the separate column pass,
  FP64 and FP32.
* A limited-area domain (ghosts from two boundary datasets interpolated in
  time, outer face fluxes of its own) against the oracle's open step: FP64
  1e-12 (relative L2 and max), FP32 2e-5 (relative L2), budgets included.
* The packed strips are the block's edge cells; bad arguments are rejected.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asuca():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    return a


def _tensor(a, dt):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt).contiguous()


def _blocks(asuca, case, decomp, prec, lim, fused=True):
    from paper_1710_08616_gb300.distributed import Block
    import torch
    dt = torch.float64 if prec == asuca.FP64 else torch.float32
    out = {}
    for r in range(decomp.nblocks):
        rx, ry = decomp.coords(r)
        sd = gen.subdomain(case, decomp.px, decomp.py, rx, ry)
        g = asuca.Grid(sd["nx"], sd["ny"], case.nz, case.ntracers, case.dz, case.dx, case.dy, prec=prec, lim=lim)
        if not fused:
            asuca.set_tuning(g, asuca.TUNE_FUSED_COLUMN, 0)
        Y = sd["Y"]
        st = asuca.State(_tensor(Y[0], dt), _tensor(Y[1], dt), _tensor(Y[2:], dt), _tensor(sd["mu_x"], dt),
                         _tensor(sd["mv_x"], dt), _tensor(sd["mw"], dt))
        out[r] = Block(g, st)
    return out


def _gather(blocks, decomp, case):
    Y = np.zeros((case.nfields, case.nz, case.ny, case.nx))
    for r, b in blocks.items():
        i0, i1, j0, j1 = decomp.extent(r)
        Y[:, :, j0:j1, i0:i1] = b.state.fields().double().cpu().numpy()
    return Y


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,ntr,lim,px,py,fused,forced", [
    ((40, 24, 12), 3, 0, 1, 1, True, False),
    ((40, 24, 12), 3, 0, 2, 1, True, True),
    ((40, 24, 12), 3, 1, 1, 2, True, False),
    ((37, 26, 7), 2, 0, 2, 2, True, False),
    ((37, 26, 7), 2, 2, 3, 2, False, True),
    ((70, 45, 12), 4, 0, 2, 3, True, False),
    ((64, 64, 16), 8, 0, 2, 2, False, False),
])
def test_decomposed_blocks_equal_periodic_step(asuca, prec, shape, ntr, lim, px, py, fused, forced):
    import torch
    from paper_1710_08616_gb300.distributed import Decomposition, step_decomposed
    nx, ny, nz = shape
    case = gen.make_case(nx, ny, nz, ntr, seed=300 + nx + px)
    nsteps = 3
    tend = np.random.default_rng(7).uniform(-1e-6, 1e-6, (1 + ntr, nz, ny, nx)) if forced else None
    g = asuca.Grid.from_case(case, prec=prec, lim=lim)
    if not fused:
        asuca.set_tuning(g, asuca.TUNE_FUSED_COLUMN, 0)
    st = asuca.State.from_case(case, prec=prec)
    td = None if tend is None else _tensor(tend, g.torch_dtype)
    ref_b = asuca.step(g, st, case.dt, nsteps, tendencies=td, budgets=True)
    d = Decomposition(nx, ny, px, py)
    blocks = _blocks(asuca, case, d, prec, lim, fused)
    tds = None
    if tend is not None:
        tds = {}
        for r in blocks:
            i0, i1, j0, j1 = d.extent(r)
            tds[r] = _tensor(tend[:, :, j0:j1, i0:i1], g.torch_dtype)
    got_b = step_decomposed(blocks, d, case.dt, nsteps, tendencies=tds)
    torch.cuda.synchronize()
    for b in blocks.values():
        assert asuca.get_status(b.grid) == asuca.OK
    ref = st.fields().double().cpu().numpy()
    got = _gather(blocks, d, case)
    assert np.array_equal(got, ref)
    rb, gb = ref_b.cpu().numpy(), got_b.cpu().numpy()
    assert np.allclose(gb, rb, rtol=1e-13, atol=0), (gb, rb)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("shape,ntr,lim,dy", [((40, 24, 12), 3, 0, 2000.0), ((37, 26, 7), 2, 1, 2000.0),
                                              ((33, 18, 9), 2, 2, 2000.0), ((70, 45, 16), 4, 0, 2000.0),
                                              ((38, 22, 10), 2, 0, 1600.0)])
def test_limited_area_step_against_oracle(asuca, prec, tol, shape, ntr, lim, dy):
    import torch
    nx, ny, nz = shape
    case = gen.make_case(nx, ny, nz, ntr, seed=500 + nx, dy=dy)
    mu_x, mv_x = gen.extend_fluxes(case.mu, case.mv)
    mu_x = mu_x.copy()
    mv_x = mv_x.copy()
    mu_x[:, :, 0] *= 1.05                     # outer faces of its own: net inflow in the west
    mv_x[:, -1, :] *= 0.9
    b0, b1 = gen.make_open_boundary(case, seed=case.seed + 1)
    tratio, nsteps = 0.3, 4
    ghost = (1.0 - tratio) * b0 + tratio * b1
    tend = np.random.default_rng(3).uniform(-1e-6, 1e-6, (1 + ntr, nz, ny, nx)) if nx == 37 else None
    og = oracle.Grid.from_case(case, lim=lim)
    g = asuca.Grid.from_case(case, prec=prec, lim=lim)
    dt_ = g.torch_dtype
    st = asuca.State(_tensor(case.rho, dt_), _tensor(case.rhotheta, dt_), _tensor(case.rhoq, dt_),
                     _tensor(mu_x, dt_), _tensor(mv_x, dt_), _tensor(case.mw, dt_))
    # the oracle starts from the GPU's (possibly float-rounded) inputs
    cast = lambda a: _tensor(a, dt_).double().cpu().numpy()
    Y0 = np.concatenate([cast(case.rho)[None], cast(case.rhotheta)[None], cast(case.rhoq)])
    ref, rbud = oracle.step_open(og, Y0, cast(mu_x), cast(mv_x), cast(case.mw),
                                 (1.0 - tratio) * cast(b0) + tratio * cast(b1), case.dt, nsteps,
                                 tend=None if tend is None else cast(tend))
    bud = asuca.step_open(g, st, case.dt, nsteps, _tensor(b0, dt_), bnd1=_tensor(b1, dt_), tratio=tratio,
                          tendencies=None if tend is None else _tensor(tend, dt_), budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    got = st.fields().double().cpu().numpy()
    for f in range(ref.shape[0]):
        l2 = np.linalg.norm(got[f] - ref[f]) / np.linalg.norm(ref[f])
        assert l2 <= tol, (f, l2)
        if prec == 0:
            mx = np.abs(got[f] - ref[f]).max() / np.abs(ref[f]).max()
            assert mx <= tol, (f, mx)
    gb = bud.cpu().numpy()
    assert np.all(np.abs(gb - rbud) <= (1e-12 if prec == 0 else 1e-5) * np.abs(rbud).max(axis=0, initial=0) + 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
def test_halo_pack_holds_the_edge_cells(asuca, prec):
    import torch
    case = gen.make_case(21, 14, 5, 2, seed=9)
    g = asuca.Grid.from_case(case, prec=prec)
    dt_ = g.torch_dtype
    mu_x, mv_x = gen.extend_fluxes(case.mu, case.mv)
    st = asuca.State(_tensor(case.rho, dt_), _tensor(case.rhotheta, dt_), _tensor(case.rhoq, dt_),
                     _tensor(mu_x, dt_), _tensor(mv_x, dt_), _tensor(case.mw, dt_))
    ws = asuca.open_workspace(g)
    asuca.open_prepare(g, st, ws)
    send = torch.empty(asuca.halo_count(g), dtype=dt_, device="cuda")
    asuca.halo_pack(g, ws, 0, send)
    torch.cuda.synchronize()
    Y = st.fields()
    phi = (Y[1:] * (1.0 / Y[0])).double().cpu().numpy()
    nx, ny = case.nx, case.ny
    w, e, s, n = gen.halo_strips(send.double().cpu().numpy(), 3, case.nz, ny, nx)
    exp = (np.moveaxis(phi[..., 0:2], 3, 2), np.moveaxis(phi[..., nx - 2:nx], 3, 2), phi[:, :, 0:2, :],
           phi[:, :, ny - 2:ny, :])
    ulp = 4 * np.finfo(np.float64 if prec == 0 else np.float32).eps
    for got, want in zip((w, e, s, n), exp):
        assert np.all(np.abs(got - want) <= ulp * np.abs(want))


def test_open_entry_points_reject_bad_arguments(asuca):
    import torch
    case = gen.make_case(16, 12, 5, 1, seed=2)
    g = asuca.Grid.from_case(case, prec=1)
    dt_ = g.torch_dtype
    mu_x, mv_x = gen.extend_fluxes(case.mu, case.mv)
    st = asuca.State(_tensor(case.rho, dt_), _tensor(case.rhotheta, dt_), _tensor(case.rhoq, dt_),
                     _tensor(mu_x, dt_), _tensor(mv_x, dt_), _tensor(case.mw, dt_))
    ws = asuca.open_workspace(g)
    h = torch.zeros(asuca.halo_count(g), dtype=dt_, device="cuda")
    for stage in (-1, 3):
        with pytest.raises(asuca.AsucaError):
            asuca.open_stage(g, st, case.dt, stage, ws)
    with pytest.raises(asuca.AsucaError):
        asuca.halo_pack(g, ws, 3, h)
    with pytest.raises(asuca.AsucaError):
        asuca.halo_unpack(g, ws, 0, h, tratio=float("nan"))
    small = torch.empty(asuca.open_workspace_bytes(g) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(asuca.AsucaError):
        asuca.open_prepare(g, st, small)
    with pytest.raises(asuca.AsucaError):
        asuca.step_open(g, st, -1.0, 1, h)
    with pytest.raises(ValueError):
        asuca.open_stage(g, asuca.State.from_case(case, prec=1), case.dt, 0, ws)   # periodic face fluxes
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
