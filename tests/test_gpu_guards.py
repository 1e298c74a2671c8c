"""Writes stay inside their buffers: every buffer a call touches is a view into
a larger allocation whose guard bands (4 KiB on each side) hold a fixed bit
pattern, and after the call the bands must be unchanged.  This covers every
kernel of the step (fused and separate column pass, dataflow mode), the
adjoint, the checkpointed forward, the ensemble, the sub-step entry points,
the storage-order stencil, the damping and the acoustic short steps, on ragged and limit sizes."""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

GUARD = 4096   # bytes on each side; keeps 256-byte alignment of the views


@pytest.fixture(scope="module")
def asuca():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    return a


class Guards:
    def __init__(self):
        self.items = []

    def make(self, shape, dtype, data=None):
        import torch
        n = int(np.prod(shape)) if len(shape) else 1
        item = torch.tensor([], dtype=dtype).element_size()
        g = GUARD // item
        big = torch.empty(n + 2 * g, dtype=dtype, device="cuda")
        big.view(torch.uint8).fill_(0xA5)
        view = big[g:g + n].view(shape)
        if data is not None:
            view.copy_(torch.as_tensor(np.array(data, copy=True)).to(device="cuda", dtype=dtype))
        self.items.append((big, g))
        return view

    def check(self):
        import torch
        torch.cuda.synchronize()
        for big, g in self.items:
            raw = big.view(torch.uint8)
            b = g * big.element_size()
            assert bool((raw[:b] == 0xA5).all()) and bool((raw[raw.numel() - b:] == 0xA5).all()), \
                "a kernel wrote outside its buffer"


def _state(asuca, G, case, prec):
    import torch
    dt = torch.float64 if prec == asuca.FP64 else torch.float32
    rhoq = case.rhoq if case.ntracers > 0 else np.zeros((0,) + case.rho.shape)
    return asuca.State(G.make(case.rho.shape, dt, case.rho), G.make(case.rhotheta.shape, dt, case.rhotheta),
                       G.make(rhoq.shape, dt, rhoq), G.make(case.mu.shape, dt, case.mu),
                       G.make(case.mv.shape, dt, case.mv), G.make(case.mw.shape, dt, case.mw))


SHAPES = [((37, 13, 7), 2), ((4, 4, 3), 1), ((70, 9, 5), 0), ((40, 24, 128), 8)]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,ntr", SHAPES)
@pytest.mark.parametrize("mode", ["fused", "separate", "dataflow"])
def test_step_writes_stay_in_bounds(asuca, prec, shape, ntr, mode):
    import torch
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, ntr, seed=31 + nx)
    g = asuca.Grid.from_case(c, prec=prec)
    if mode == "separate":
        asuca.set_tuning(g, asuca.TUNE_FUSED_COLUMN, 0)
    if mode == "dataflow":
        asuca.set_tuning(g, asuca.TUNE_STEP_MODE, 1)
    G = Guards()
    st = _state(asuca, G, c, prec)
    dt_ = g.torch_dtype
    tend = G.make((ntr + 1, nz, ny, nx), dt_, np.random.default_rng(1).standard_normal((ntr + 1, nz, ny, nx)) * 1e-5)
    ws = G.make((g.workspace_bytes(),), torch.uint8)
    bud = G.make((g.nfields + 1,), torch.float64)
    asuca.step(g, st, c.dt, 3, tendencies=tend, workspace=ws, budgets=bud)
    G.check()
    assert asuca.get_status(g) == asuca.OK


@pytest.mark.parametrize("prec", [1, 0])
def test_adjoint_writes_stay_in_bounds(asuca, prec):
    import torch
    c = gen.make_case(37, 13, 9, 3, seed=5)
    g = asuca.Grid.from_case(c, prec=prec)
    G = Guards()
    st = _state(asuca, G, c, prec)
    dt_ = g.torch_dtype
    F = g.nfields
    shp = (F, c.nz, c.ny, c.nx)
    lam = G.make(shp, dt_, np.random.default_rng(2).standard_normal(shp))
    nsteps, K = 5, 2
    ws = G.make((asuca.adjoint_workspace_bytes(g, nsteps, K),), torch.uint8)
    g0, gmu, gmv = G.make(shp, dt_), G.make(c.mu.shape, dt_), G.make(c.mv.shape, dt_)
    gmw = G.make(c.mw.shape, dt_)
    s = st.struct()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = asuca.lib().asuca_adjoint_step(g.handle, ctypes.byref(s), None, float(c.dt), nsteps, K, p(lam), p(g0),
                                        p(gmu), p(gmv), p(gmw), p(ws), ws.numel(),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == asuca.OK
    # the checkpointed forward and the reverse from its checkpoints
    ck = G.make((asuca.checkpoint_bytes(g, nsteps, K),), torch.uint8)
    wst = G.make((g.workspace_bytes(),), torch.uint8)
    asuca.forward_checkpointed(g, st, c.dt, nsteps, checkpoint_every=K, workspace=wst, checkpoints=ck)
    asuca.adjoint_from_checkpoints(g, ck, st, c.dt, nsteps, lam, checkpoint_every=K, workspace=ws)
    G.check()
    assert asuca.get_status(g) == asuca.OK


@pytest.mark.parametrize("prec", [1, 0])
def test_ensemble_writes_stay_in_bounds(asuca, prec):
    import torch
    cases = gen.make_ensemble_cases(sizes=[33, 64, 17], nz=8, ntracers=2)
    grids = [asuca.Grid.from_case(c, prec=prec) for c in cases]
    G = Guards()
    states = [_state(asuca, G, c, prec) for c in cases]
    ws = G.make((asuca.ensemble_workspace_bytes(grids),), torch.uint8)
    bud = G.make((len(cases), grids[0].nfields + 1), torch.float64)
    asuca.ensemble_step(grids, states, [c.dt for c in cases], 3, workspace=ws, budgets=bud)
    G.check()
    assert asuca.get_status(grids[0]) == asuca.OK


@pytest.mark.parametrize("prec", [1, 0])
def test_substep_entry_points_write_in_bounds(asuca, prec):
    import torch
    c = gen.make_case(37, 13, 7, 2, seed=9)
    g = asuca.Grid.from_case(c, prec=prec)
    G = Guards()
    a, b, o = _state(asuca, G, c, prec), _state(asuca, G, c, prec), _state(asuca, G, c, prec)
    asuca.debug_stage(g, a, b, o, c.dt / 3)
    pc = G.make((c.ny, c.nx), torch.float64, np.zeros((c.ny, c.nx)))
    ws = G.make((g.workspace_bytes(),), torch.uint8)
    asuca.debug_column(g, a, c.dt, pc, workspace=ws)
    asuca.column_noalloc(g, b, c.dt, pc)
    dt_ = g.torch_dtype
    f = np.random.default_rng(3).standard_normal((7, 13, 37))
    for layout, shp in ((asuca.LAYOUT_IJK, (7, 13, 37)), (asuca.LAYOUT_KIJ, (13, 37, 7))):
        x = G.make(shp, dt_, f if layout == asuca.LAYOUT_IJK else np.transpose(f, (1, 2, 0)))
        asuca.stencil7(x, G.make(shp, dt_), 0.1, layout)
    Y = c.state()
    ref, b0, b1 = (G.make(Y.shape, dt_, a) for a in gen.make_boundary_data(Y, 5))
    for width, ntop in ((3, 2), (6, 7), (0, 1), (2, 0)):
        asuca.damping(g, o, ref, b0, b1, 0.4, c.dt, width=width, ntop=ntop, nu_lat=1e-2, nu_top=1e-2)
    U, V, W, S, r0c, r0f = gen.make_acoustic_state(c)
    ac = [G.make(a.shape, dt_, a) for a in (U, V, W, S)]
    wsa = G.make((asuca.acoustic_workspace_bytes(g),), torch.uint8)
    asuca.acoustic_steps(g, *ac, r0c, r0f, gen.ACOUSTIC["cs2"], 0.6, 2.0, 3, workspace=wsa)
    G.check()
    assert asuca.get_status(g) == asuca.OK
