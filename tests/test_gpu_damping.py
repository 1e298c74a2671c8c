"""GPU parity of the lateral and upper damping (asuca_damping, Sec. 2.1's
damping kernel) against the FP64 oracle.

Bars: FP64 within 1e-12 relative (per-field L2 and max); FP32 within 2e-5
relative L2 per field; every cell outside the damping zone bit-for-bit
unchanged in both precisions."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


@pytest.fixture(scope="module")
def asuca():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    return a


def _zone(nx, ny, nz, width, ntop):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.minimum(np.minimum(i, nx - 1 - i), np.minimum(j, ny - 1 - j))
    return (d < width) | (k >= nz - ntop)


def _run(asuca, case, prec, tratio, dt, kw, mtratio=None):
    import torch
    dt_ = torch.float64 if prec == asuca.FP64 else torch.float32
    npdt = np.float64 if prec == asuca.FP64 else np.float32
    Y = case.state().astype(npdt)
    ref, b0, b1 = gen.make_boundary_data(Y, case.seed + 17, dtype=npdt)
    g = asuca.Grid.from_case(case, prec=prec)
    st = asuca.State.from_case(case, prec=prec)
    dev = lambda a: torch.as_tensor(np.array(a, copy=True)).to(device="cuda", dtype=dt_)
    asuca.damping(g, st, dev(ref), dev(b0), dev(b1), tratio, dt, mtratio=mtratio, **kw)
    got = st.fields().double().cpu().numpy()
    want = oracle.damping(Y, ref, b0, b1, tratio, dt, mtratio=mtratio, **kw)
    assert asuca.get_status(g) == asuca.OK
    return Y, got, want


def _check(asuca, prec, Y, got, want, zone):
    out = ~zone
    assert np.array_equal(got[:, out], Y[:, out].astype(np.float64)), "a cell outside the zone changed"
    tol = TOL64 if prec == asuca.FP64 else TOL32
    for f in range(want.shape[0]):
        l2 = np.linalg.norm(got[f] - want[f]) / np.linalg.norm(want[f])
        assert l2 <= tol, f"field {f}: rel L2 {l2:.3e}"
        if prec == asuca.FP64:
            assert np.abs(got[f] - want[f]).max() <= tol * np.abs(want[f]).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,ntr,width,ntop", [
    ((37, 13, 7), 2, 3, 2),       # ragged, both zones
    ((4, 4, 3), 1, 2, 3),         # 2 width = nx = ny: the frame is the whole plane; ntop = nz
    ((70, 9, 5), 0, 4, 0),        # lateral zone only, 2 width = 8 of ny = 9
    ((32, 32, 16), 3, 0, 5),      # upper zone only
    ((300, 20, 12), 8, 64, 1),    # the widest zone the library takes, every tracer
    ((33, 41, 10), 2, 7, 10),     # the upper zone covers every level
])
def test_damping_matches_oracle(asuca, prec, shape, ntr, width, ntop):
    nx, ny, nz = shape
    if 2 * width > min(nx, ny):
        width = min(nx, ny) // 2
    c = gen.make_case(nx, ny, nz, ntr, seed=600 + nx)
    kw = dict(width=width, ntop=ntop, nu_lat=1.0 / 300.0, nu_top=1.0 / 600.0)
    Y, got, want = _run(asuca, c, prec, 0.25, c.dt, kw)
    _check(asuca, prec, Y, got, want, _zone(nx, ny, nz, width, ntop))


@pytest.mark.parametrize("prec", [0, 1])
def test_damping_general_weights_and_strong_rates(asuca, prec):
    """mtratio and tratio need not sum to one; very large rates land on the
    target; dt = 0 and nu = 0 leave the state as it is."""
    c = gen.make_case(29, 17, 9, 3, seed=77)
    kw = dict(width=5, ntop=3, nu_lat=1e9, nu_top=1e9)
    Y, got, want = _run(asuca, c, prec, 0.6, c.dt, kw, mtratio=0.7)
    _check(asuca, prec, Y, got, want, _zone(29, 17, 9, 5, 3))
    for dt, nu in ((0.0, 1e-2), (c.dt, 0.0)):
        Y, got, want = _run(asuca, c, prec, 0.3, dt, dict(width=5, ntop=3, nu_lat=nu, nu_top=nu))
        assert np.array_equal(got, Y.astype(np.float64))


def test_empty_zone_launches_nothing(asuca):
    import torch
    c = gen.make_case(16, 16, 4, 1, seed=3)
    g = asuca.Grid.from_case(c)
    st = asuca.State.from_case(c)
    before = st.fields().clone()
    z = torch.zeros((3, 4, 16, 16), dtype=torch.float32, device="cuda")
    asuca.damping(g, st, z, z, z, 0.5, c.dt, width=0, ntop=0, nu_lat=1.0, nu_top=1.0)
    torch.cuda.synchronize()
    assert torch.equal(st.fields(), before)


def test_damping_rejects_bad_arguments(asuca):
    import torch
    c = gen.make_case(16, 12, 5, 1, seed=4)
    g = asuca.Grid.from_case(c)
    st = asuca.State.from_case(c)
    z = torch.zeros((3, 5, 12, 16), dtype=torch.float32, device="cuda")
    good = dict(width=2, ntop=1, nu_lat=1e-2, nu_top=1e-2)
    for bad in (dict(width=-1), dict(width=7), dict(width=65), dict(ntop=-1), dict(ntop=6), dict(nu_lat=-1.0),
                dict(nu_top=float("nan"))):
        with pytest.raises(asuca.AsucaError) as e:
            asuca.damping(g, st, z, z, z, 0.5, c.dt, **{**good, **bad})
        assert e.value.status == asuca.ERR_ARG
    for dt, tr in ((-1.0, 0.5), (float("inf"), 0.5), (1.0, float("nan"))):
        with pytest.raises(asuca.AsucaError):
            asuca.damping(g, st, z, z, z, tr, dt, **good)
    s = st.struct()
    d = asuca.DampingDesc(2, 1, 1e-2, 1e-2)
    p = ctypes.c_void_p(z.data_ptr())
    assert asuca.lib().asuca_damping(g.handle, ctypes.byref(s), None, p, p, 0.5, 0.5, 1.0, ctypes.byref(d),
                                     None) == asuca.ERR_ARG
    assert asuca.lib().asuca_damping(g.handle, ctypes.byref(s), p, p, p, 0.5, 0.5, 1.0, None, None) == asuca.ERR_ARG


def test_damping_full_size_sampled(asuca):
    """1024x1024x58 with 8 tracers, FP32, the zone and rates the benchmark times:
    sampled zone and non-zone cells against the oracle cell by cell."""
    import torch
    c = gen.make_config_case("large_1024x1024x58", dtype=np.float32)
    D = gen.DAMPING
    nx, ny, nz = c.nx, c.ny, c.nz
    Y = c.state()
    ref, b0, b1 = gen.make_boundary_data(Y, c.seed + 17, dtype=np.float32)
    g = asuca.Grid.from_case(c, prec=asuca.FP32_MIXED)
    st = asuca.State.from_case(c, prec=asuca.FP32_MIXED)
    dev = lambda a: torch.from_numpy(a).to("cuda")
    kw = dict(width=D["width"], ntop=D["ntop"], nu_lat=D["nu_lat"], nu_top=D["nu_top"])
    asuca.damping(g, st, dev(ref), dev(b0), dev(b1), D["tratio"], c.dt, **kw)
    got = st.fields()
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    n = 20000
    i = rng.integers(0, nx, n)
    j = np.where(rng.random(n) < 0.5, rng.integers(0, D["width"], n), rng.integers(0, ny, n))
    k = rng.integers(0, nz, n)
    ijk = np.stack([i, j, k], axis=1)
    pick = lambda a: np.ascontiguousarray(a[:, k, j, i], dtype=np.float64)
    want = oracle.damping(pick(Y), pick(ref), pick(b0), pick(b1), D["tratio"], c.dt, ijk=ijk, shape=(nx, ny, nz),
                          **kw)
    gi = torch.as_tensor(k * nx * ny + j * nx + i, device="cuda")
    gv = got.reshape(got.shape[0], -1)[:, gi].double().cpu().numpy()
    zone = _zone_cells(i, j, k, nx, ny, nz, D["width"], D["ntop"])
    assert zone.sum() > 1000 and (~zone).sum() > 1000
    assert np.array_equal(gv[:, ~zone], pick(Y)[:, ~zone])
    for f in range(want.shape[0]):
        w, d = want[f, zone], gv[f, zone] - want[f, zone]
        assert np.linalg.norm(d) <= TOL32 * np.linalg.norm(w), f"field {f}"
        assert np.abs(d).max() <= TOL32 * np.abs(w).max(), f"field {f}"


def _zone_cells(i, j, k, nx, ny, nz, width, ntop):
    d = np.minimum(np.minimum(i, nx - 1 - i), np.minimum(j, ny - 1 - j))
    return (d < width) | (k >= nz - ntop)
