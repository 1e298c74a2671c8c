"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (written here, from the specification): FP64 path within 1e-12
relative, both as per-field ||d||_2/||ref||_2 and max|d|/max|ref|; FP32-mixed
path within 2e-5 relative L2 per field.  Bit-exact where the arithmetic is
exact (Courant-1 upwind shift).
"""
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


def _rel(got, ref):
    l2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    mx = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    return l2, mx


def _assert_fields(got, ref, tol, what, both=True):
    for f in range(ref.shape[0]):
        l2, mx = _rel(got[f], ref[f])
        assert l2 <= tol, f"{what}: field {f} rel L2 {l2:.3e} > {tol}"
        if both:
            assert mx <= tol, f"{what}: field {f} rel max {mx:.3e} > {tol}"


def _grid_pair(asuca, case, prec, **phys):
    kw = dict(tau=oracle.TAU, k0=oracle.K0, kh=oracle.KH, vsed=oracle.VSED, lim=oracle.LIM_KOREN)
    kw.update(phys)
    og = oracle.Grid.from_case(case, tau=kw["tau"], k0=kw["k0"], kh=kw["kh"], vsed=kw["vsed"],
                               lim=kw["lim"])
    g = asuca.Grid.from_case(case, tau_theta=kw["tau"], k0=kw["k0"], k_h=kw["kh"], v_sed=kw["vsed"],
                             lim=kw["lim"], prec=prec)
    return og, g


def _np(st):
    return st.fields().double().cpu().numpy()


# ------------------------------------------------------------------ single stage

@pytest.mark.parametrize("lim", [0, 1, 2])
@pytest.mark.parametrize("shape", [(32, 32, 16), (37, 13, 7), (4, 4, 3), (70, 9, 5)])
def test_stage_fp64(asuca, lim, shape):
    import torch
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, 3, seed=11 + nx)
    og, g = _grid_pair(asuca, c, asuca.FP64, lim=lim)
    rng = np.random.default_rng(5)
    Yin = c.state() * (1 + 0.01 * rng.standard_normal(c.state().shape))
    Ybase = c.state()
    tend = rng.uniform(-1e-4, 1e-4, (4, nz, ny, nx))
    R = oracle.rhs(og, Yin, c.mu, c.mv, c.mw, tend=tend)
    ref = Ybase + (c.dt / 2) * R
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    sin = asuca.State(dev(Yin[0]), dev(Yin[1]), dev(Yin[2:]), dev(c.mu), dev(c.mv), dev(c.mw))
    sbase = asuca.State(dev(Ybase[0]), dev(Ybase[1]), dev(Ybase[2:]), sin.mu, sin.mv, sin.mw)
    sout = sbase.clone()
    asuca.debug_stage(g, sin, sbase, sout, c.dt / 2, tendencies=dev(tend))
    torch.cuda.synchronize()
    _assert_fields(_np(sout), ref, TOL64, f"stage lim={lim} {shape}")


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_courant_one_shift_bit_exact(asuca, axis, sign, prec):
    import torch
    nx, ny, nz = 40, 20, 3
    rng = np.random.default_rng(3)
    Y = np.empty((4, nz, ny, nx))
    Y[0] = 1.0
    Y[1:] = rng.integers(-50, 50, (3, nz, ny, nx))
    mu = np.full((nz, ny, nx), 16.0 * sign if axis == 0 else 0.0)
    mv = np.full((nz, ny, nx), 16.0 * sign if axis == 1 else 0.0)
    mw = np.zeros((nz + 1, ny, nx))
    g = asuca.Grid(nx, ny, nz, 2, np.full(nz, 100.0), 2048.0, 2048.0, tau_theta=0, k0=0, v_sed=0,
                   lim=asuca.LIM_UPWIND1, prec=prec)
    dt_ = torch.float64 if prec == 0 else torch.float32
    dev = lambda a: torch.tensor(a, dtype=dt_, device="cuda")
    s = asuca.State(dev(Y[0]), dev(Y[1]), dev(Y[2:]), dev(mu), dev(mv), dev(mw))
    out = s.clone()
    asuca.debug_stage(g, s, s, out, 128.0)
    torch.cuda.synchronize()
    assert np.array_equal(_np(out), np.roll(Y, sign, axis=3 if axis == 0 else 2))


# ------------------------------------------------------------------ column pass

@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("phys", [dict(), dict(k0=0.0), dict(vsed=0.0, tau=0.0), dict(tau=0.0, k0=0.0)])
def test_column_pass(asuca, prec, tol, phys):
    import torch
    c = gen.make_case(45, 19, 16, 3, seed=99)
    og, g = _grid_pair(asuca, c, prec, **phys)
    ref, pc_ref = oracle.column(og, c.state(), c.dt)
    st = asuca.State.from_case(c, prec=prec)
    pc = torch.zeros((c.ny, c.nx), dtype=torch.float64, device="cuda")
    asuca.debug_column(g, st, c.dt, pc)
    torch.cuda.synchronize()
    _assert_fields(_np(st), ref, tol, f"column {phys}", both=(prec == 0))
    if phys.get("vsed", 1.0) > 0:
        l2, mx = _rel(pc.cpu().numpy(), pc_ref)
        assert l2 <= tol and (prec == 1 or mx <= tol)


# ------------------------------------------------------------------ full steps

def _full_step(asuca, case, prec, nsteps, tend=None, **phys):
    import torch
    og, g = _grid_pair(asuca, case, prec, **phys)
    ref, rbud = oracle.step(og, case.state(), case.mu, case.mv, case.mw, case.dt, nsteps, tend=tend)
    st = asuca.State.from_case(case, prec=prec)
    td = None
    if tend is not None:
        td = torch.tensor(tend, dtype=g.torch_dtype, device="cuda")
    bud = asuca.step(g, st, case.dt, nsteps, tendencies=td, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    return _np(st), ref, bud.cpu().numpy(), rbud


def test_full_step_fp64_32x32x16_20_steps(asuca):
    c = gen.make_config_case("fp64_32x32x16")
    got, ref, bud, rbud = _full_step(asuca, c, asuca.FP64, 20)
    _assert_fields(got, ref, TOL64, "fp64 32x32x16 x20")
    assert np.all(np.abs(bud - rbud) <= TOL64 * np.abs(rbud))


@pytest.mark.parametrize("shape,ntr,nsteps", [((37, 13, 7), 2, 5), ((4, 4, 3), 1, 4), ((70, 9, 5), 0, 3),
                                              ((33, 65, 11), 8, 2)])
def test_full_step_fp64_ragged_with_tendencies(asuca, shape, ntr, nsteps):
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, ntr, seed=1234 + nx)
    rng = np.random.default_rng(nx)
    tend = rng.uniform(-1e-5, 1e-5, (1 + ntr, nz, ny, nx))
    got, ref, bud, rbud = _full_step(asuca, c, asuca.FP64, nsteps, tend=tend)
    _assert_fields(got, ref, TOL64, f"fp64 {shape}")
    nz_b = np.abs(rbud) > 0
    assert np.all(np.abs(bud - rbud)[nz_b] <= TOL64 * np.abs(rbud)[nz_b])


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("mode", ["fused", "separate", "dataflow"])
def test_full_step_with_different_spacings_in_i_and_j(asuca, prec, tol, mode):
    """dx = 2000 m, dy = 1600 m (every other case has dx = dy, where a swapped
    spacing goes unseen): three steps of a ragged grid against the oracle, in
    each arrangement of the column pass."""
    import torch
    c = gen.make_case(37, 26, 9, 2, seed=88, dx=2000.0, dy=1600.0)
    og, g = _grid_pair(asuca, c, prec)
    if mode == "separate":
        asuca.set_tuning(g, asuca.TUNE_FUSED_COLUMN, 0)
    elif mode == "dataflow":
        asuca.set_tuning(g, asuca.TUNE_STEP_MODE, 1)
    ref, rbud = oracle.step(og, c.state(), c.mu, c.mv, c.mw, c.dt, 3)
    st = asuca.State.from_case(c, prec=prec)
    bud = asuca.step(g, st, c.dt, 3, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    _assert_fields(_np(st), ref, tol, f"dx != dy prec={prec} {mode}", both=(prec == 0))
    assert np.all(np.abs(bud.cpu().numpy() - rbud) <= tol * np.abs(rbud))


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("mode", ["fused", "separate", "dataflow"])
@pytest.mark.parametrize("sed", [0, 1, -1])
def test_full_step_with_another_sedimenting_tracer(asuca, prec, tol, mode, sed):
    """Every other case sediments the last tracer, which the column code takes
    as a compile-time index: here the first, a middle one, or none, in each
    arrangement of the column pass, against the oracle (precipitation
    included)."""
    import torch
    c = gen.make_case(29, 21, 10, 3, seed=91)
    og = oracle.Grid.from_case(c, sed=sed)
    g = asuca.Grid.from_case(c, prec=prec, sed_tracer=sed)
    if mode == "separate":
        asuca.set_tuning(g, asuca.TUNE_FUSED_COLUMN, 0)
    elif mode == "dataflow":
        asuca.set_tuning(g, asuca.TUNE_STEP_MODE, 1)
    ref, rbud = oracle.step(og, c.state(), c.mu, c.mv, c.mw, c.dt, 3)
    st = asuca.State.from_case(c, prec=prec)
    bud = asuca.step(g, st, c.dt, 3, budgets=True).cpu().numpy()
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    _assert_fields(_np(st), ref, tol, f"sed={sed} prec={prec} {mode}", both=(prec == 0))
    assert np.all(np.abs(bud - rbud) <= tol * np.abs(rbud))
    assert (rbud[-1] > 0) == (sed >= 0)


@pytest.mark.parametrize("lim", [0, 1, 2])
def test_full_step_fp32_mixed_32x32x16_20_steps(asuca, lim):
    c = gen.make_config_case("fp64_32x32x16")
    got, ref, bud, rbud = _full_step(asuca, c, asuca.FP32_MIXED, 20, lim=lim)
    _assert_fields(got, ref, TOL32, f"fp32 lim={lim}", both=False)
    assert np.all(np.abs(bud - rbud) <= TOL32 * np.abs(rbud))


def test_budgets_only_call(asuca):
    import torch
    c = gen.make_config_case("fp64_32x32x16")
    og, g = _grid_pair(asuca, c, asuca.FP64)
    st = asuca.State.from_case(c, prec=asuca.FP64)
    bud = asuca.step(g, st, c.dt, 0, budgets=True)
    torch.cuda.synchronize()
    rb = oracle.budgets(og, c.state())
    assert np.all(np.abs(bud.cpu().numpy() - rb) <= TOL64 * np.abs(rb) + 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_in_host_input_reports_nonfinite(asuca, prec):
    """Host-side fault injection: a NaN planted in the host copy of one tracer
    reaches the device with the input, the budget reduction flags it, and the
    next status read returns ASUCA_ERR_NONFINITE; the grid is usable after."""
    import torch
    c = gen.make_config_case("fp64_32x32x16")
    c.rhoq = c.rhoq.copy()
    c.rhoq[1, 3, 5, 7] = np.nan
    g = asuca.Grid.from_case(c, prec=prec)
    st = asuca.State.from_case(c, prec=prec)
    asuca.step(g, st, c.dt, 1, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.ERR_NONFINITE
    assert asuca.get_status(g) == asuca.OK          # the word is cleared by the read
    clean = asuca.State.from_case(gen.make_config_case("fp64_32x32x16"), prec=prec)
    asuca.step(g, clean, c.dt, 1, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK


def test_short_or_misaligned_workspace_is_rejected(asuca):
    import torch
    c = gen.make_config_case("fp64_32x32x16")
    g = asuca.Grid.from_case(c, prec=asuca.FP64)
    st = asuca.State.from_case(c, prec=asuca.FP64)
    need = g.workspace_bytes()
    short = torch.empty(need - 256, dtype=torch.uint8, device=st.rho.device)
    with pytest.raises(asuca.AsucaError) as e:
        asuca.step(g, st, c.dt, 1, workspace=short)
    assert e.value.status == asuca.ERR_WORKSPACE
    big = torch.empty(need + 512, dtype=torch.uint8, device=st.rho.device)
    with pytest.raises(asuca.AsucaError) as e:
        asuca.step(g, st, c.dt, 1, workspace=big[8:8 + need])     # not 256-byte aligned
    assert e.value.status == asuca.ERR_WORKSPACE


# ------------------------------------------------------------------ precision workload, full size

@pytest.fixture(scope="module")
def precision_ref():
    """The FP64 oracle after 100 steps of the 256x256x58, 6-tracer workload
    (about two minutes on the host cores)."""
    c = gen.make_config_case("precision_256x256x58")
    og = oracle.Grid.from_case(c)
    ref, rbud = oracle.step(og, c.state(), c.mu, c.mv, c.mw, c.dt, gen.CONFIGS["precision_256x256x58"]["nsteps"])
    return c, ref, rbud


@pytest.mark.slow
@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_precision_256x256x58_100_steps(asuca, precision_ref, prec, tol):
    """The whole 100-step run of the precision workload, every cell of every
    field against the oracle: FP64 within 1e-12 (L2 and max), FP32-mixed within
    2e-5 relative L2 per field; the FP64 budgets (mass, rho theta, tracers,
    precipitation) within the same bars."""
    import torch
    c, ref, rbud = precision_ref
    g = asuca.Grid.from_case(c, prec=prec)
    st = asuca.State.from_case(c, prec=prec)
    bud = asuca.step(g, st, c.dt, gen.CONFIGS["precision_256x256x58"]["nsteps"], budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    _assert_fields(_np(st), ref, tol, f"precision prec={prec}", both=(prec == 0))
    bud = bud.cpu().numpy()
    assert np.all(np.abs(bud - rbud) <= tol * np.abs(rbud))


# ------------------------------------------------------------------ full size, sampled

SAMPLES = [(0, 0), (1023, 1023), (511, 0), (0, 700), (1023, 5)]


@pytest.fixture(scope="module")
def large_case():
    return gen.make_config_case("large_1024x1024x58")


@pytest.mark.parametrize("prec,tol", [(1, TOL32), (0, TOL64)])
def test_large_1024x1024x58_one_step_sampled_columns(asuca, large_case, prec, tol):
    """One step at the full 1024x1024x58, 8-tracer size in the launch
    configuration the benchmark times; sampled 4x4 windows checked against the
    oracle evaluated on their dependency cone."""
    import torch
    c = large_case
    og, g = _grid_pair(asuca, c, prec)
    st = asuca.State.from_case(c, prec=prec)
    asuca.step(g, st, c.dt, 1, budgets=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    picks = SAMPLES + [tuple(int(v) for v in rng.integers(0, 1024, 2)) for _ in range(6)]
    Y0 = c.state()
    for (i0, j0) in picks:
        w = h = 4
        ref = oracle.step_window(og, Y0, c.mu, c.mv, c.mw, c.dt, 1, i0, j0, w, h)
        ii = torch.tensor([(i0 + q) % c.nx for q in range(w)], device="cuda")
        jj = torch.tensor([(j0 + q) % c.ny for q in range(h)], device="cuda")
        got = st.fields()[:, :, jj][:, :, :, ii].double().cpu().numpy()
        _assert_fields(got, ref, tol, f"large prec={prec} window {(i0, j0)}", both=(prec == 0))
    del st


# Conservation bar of the FP32-mixed path over three steps: every stored value
# is rounded to float once per step (2^-24 relative) and the column pass's
# output goes through up to four float roundings (the narrowed unknown and
# its scaling), so the totals can drift by at most 3 * 5 * 2^-24 = 9e-7 of
# their size if every rounding fell the same way.
CONS32 = 2e-6


@pytest.mark.parametrize("prec,tol,cons", [(1, TOL32, CONS32), (0, TOL64, TOL64)])
def test_large_1024x1024x58_three_steps_windows_and_budgets(asuca, large_case, prec, tol, cons):
    """Three steps at the full 1024x1024x58, 8-tracer size in the benchmark's
    launch configuration.  Sampled 4x4 windows (corners, edges, random picks)
    against the oracle on their three-step dependency cone; and the budgets
    against properties that hold at any size: the device's budgets equal the
    oracle's compensated sums over the device's own fields (1e-12 in both
    paths, since floats widen to double exactly); total mass and every
    tracer that does not sediment keep their totals (periodic domain, closed
    lids, conservative advection and diffusion); the sedimenting tracer loses
    exactly the precipitation."""
    import torch
    c = large_case
    nsteps = 3
    og, g = _grid_pair(asuca, c, prec)
    st = asuca.State.from_case(c, prec=prec)
    bud = asuca.step(g, st, c.dt, nsteps, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    bud = bud.cpu().numpy()
    Y0 = c.state()
    rng = np.random.default_rng(29)
    picks = SAMPLES + [tuple(int(v) for v in rng.integers(0, 1024, 2)) for _ in range(3)]
    for (i0, j0) in picks:
        w = h = 4
        ref = oracle.step_window(og, Y0, c.mu, c.mv, c.mw, c.dt, nsteps, i0, j0, w, h)
        ii = torch.tensor([(i0 + q) % c.nx for q in range(w)], device="cuda")
        jj = torch.tensor([(j0 + q) % c.ny for q in range(h)], device="cuda")
        got = st.fields()[:, :, jj][:, :, :, ii].double().cpu().numpy()
        _assert_fields(got, ref, tol, f"large prec={prec} {nsteps} steps window {(i0, j0)}", both=(prec == 0))
    before = oracle.budgets(og, Y0)
    del Y0
    Y1 = _np(st)
    del st
    after = oracle.budgets(og, Y1, precip=float(bud[-1]))
    del Y1
    # the device's sums of its own fields
    d = np.abs(bud - after) / np.abs(after).clip(1e-300)
    assert d.max() <= 1e-12, f"prec={prec}: budgets vs sums of the fields {d}"
    # conservation: mass and the tracers that do not sediment; the sedimenting
    # tracer (the last, the oracle grid's default) loses the precipitation
    F = c.nfields
    sed = F - 1
    assert bud[-1] > 0.0
    for f in [0] + list(range(2, F)):
        loss = bud[-1] if f == sed else 0.0
        drift = abs(before[f] - after[f] - loss) / abs(before[f])
        assert drift <= cons, f"prec={prec}: field {f} total drifts by {drift:.3e} > {cons}"


# ------------------------------------------------------------------ arithmetic helpers

def test_integer_pipe_conversions_match_hardware(asuca):
    """The column solve widens floats and narrows doubles through the IEEE-754
    bit fields; the results must equal CUDA's own conversions bit for bit,
    including ties, the float range limits, zeros, subnormals, inf and NaN."""
    import torch
    rng = np.random.default_rng(8)
    f = rng.standard_normal(200000).astype(np.float32) * (10.0 ** rng.uniform(-30, 30, 200000)).astype(np.float32)
    specials_f = np.array([0.0, -0.0, 1e-45, -1e-40, 1.17549435e-38, 3.4028235e38, np.inf, -np.inf, np.nan],
                          dtype=np.float32)
    f = np.concatenate([f, specials_f])
    d = rng.standard_normal(200000) * 10.0 ** rng.uniform(-50, 50, 200000)
    base = rng.standard_normal(20000).astype(np.float32).astype(np.float64)
    ulp = np.abs(np.spacing(base.astype(np.float32)).astype(np.float64))
    ties = np.concatenate([base + ulp / 2, base - ulp / 2, base + ulp / 2 * (1 + 2 ** -30)])
    specials_d = np.array([0.0, -0.0, 1e-320, 1.1754942e-38, 1.17549435e-38, 3.4028234663852886e38,
                           3.4028235677973366e38, 3.5e38, -3.5e38, 1e300, np.inf, -np.inf, np.nan])
    d = np.concatenate([d, ties, specials_d])
    n = max(len(f), len(d))
    f = np.resize(f, n)
    d = np.resize(d, n)
    tf = torch.tensor(f, device="cuda")
    td = torch.tensor(d, device="cuda")
    w, nr, r = asuca.debug_numerics(tf, td)
    torch.cuda.synchronize()
    hw_w = tf.double()
    hw_n = td.float()
    same_w = (w.view(torch.int64) == hw_w.view(torch.int64)) | (torch.isnan(w) & torch.isnan(hw_w))
    same_n = (nr.view(torch.int32) == hw_n.view(torch.int32)) | (torch.isnan(nr) & torch.isnan(hw_n))
    assert bool(same_w.all()) and bool(same_n.all())
    # Newton reciprocal within 2 ulp of the correctly rounded 1/x on the normal range
    x = torch.tensor(rng.uniform(1e-3, 1e6, 100000) * rng.choice([-1, 1], 100000), device="cuda")
    _, _, r = asuca.debug_numerics(torch.zeros(len(x), dtype=torch.float32, device="cuda"), x)
    exact = 1.0 / x
    ulps = ((r - exact).abs() / torch.abs(exact) / 2.0 ** -52).max().item()
    assert ulps <= 2.0, ulps


# ------------------------------------------------------------------ dataflow step mode

@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,ntr,nsteps", [((70, 45, 12), 3, 20), ((32, 32, 16), 3, 3), ((100, 9, 7), 1, 2),
                                              ((4, 4, 3), 0, 17)])
def test_dataflow_mode_equals_stage_launches(asuca, prec, shape, ntr, nsteps):
    """The persistent dataflow kernel runs the same per-cell arithmetic as the
    per-stage launches, only in another order, so results match bit for bit
    (20 steps span two 16-step launches)."""
    import torch
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, ntr, seed=77 + nx)
    g0 = asuca.Grid.from_case(c, prec=prec)
    g1 = asuca.Grid.from_case(c, prec=prec)
    asuca.set_tuning(g1, asuca.TUNE_STEP_MODE, 1)
    a = asuca.State.from_case(c, prec=prec)
    b = a.clone()
    ba = asuca.step(g0, a, c.dt, nsteps, budgets=True)
    bb = asuca.step(g1, b, c.dt, nsteps, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g1) == asuca.OK
    assert torch.equal(a.fields(), b.fields())
    rel = (ba - bb).abs() / ba.abs().clamp_min(1e-300)
    assert float(rel.max()) <= 1e-13


# ------------------------------------------------------------------ fused third stage + column pass

@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("lim", [0, 1, 2])
@pytest.mark.parametrize("shape,ntr,nsteps,phys", [
    ((70, 45, 12), 3, 4, dict()),
    ((37, 13, 7), 2, 3, dict(tau_theta=0.0)),
    ((4, 4, 3), 1, 5, dict(v_sed=0.0)),
    ((100, 9, 5), 0, 2, dict()),
    ((64, 40, 16), 8, 2, dict()),
])
def test_fused_stage3_column_equals_separate_launches(asuca, prec, lim, shape, ntr, nsteps, phys):
    """The third stage marching downward with the top-down column pass, then
    the bottom-up back substitution, performs every cell's operations exactly as
    the upward stage launch followed by the column kernel, so the fields match
    bit for bit; the density budget is summed in the other direction, so the
    budgets match to rounding."""
    import torch
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, ntr, seed=901 + nx + ntr)
    kw = dict(lim=lim, prec=prec, **phys)
    g0 = asuca.Grid.from_case(c, **kw)
    g1 = asuca.Grid.from_case(c, **kw)
    asuca.set_tuning(g0, asuca.TUNE_FUSED_COLUMN, 0)
    assert asuca.get_tuning(g1, asuca.TUNE_FUSED_COLUMN) == 1
    a = asuca.State.from_case(c, prec=prec)
    b = a.clone()
    tend = None
    if ntr == 2:   # constant forcing too
        rng = np.random.default_rng(5)
        tend = torch.tensor(rng.standard_normal((ntr + 1, nz, ny, nx)) * 1e-4, dtype=g0.torch_dtype,
                            device=a.rho.device).contiguous()
    ba = asuca.step(g0, a, c.dt, nsteps, tendencies=tend, budgets=True)
    bb = asuca.step(g1, b, c.dt, nsteps, tendencies=tend, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g0) == asuca.OK and asuca.get_status(g1) == asuca.OK
    assert torch.equal(a.fields(), b.fields())
    rel = (ba - bb).abs() / ba.abs().clamp_min(1e-300)
    assert float(rel.max()) <= 1e-13


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_full_step_at_the_level_limit(asuca, prec, tol):
    """nz = ASUCA_MAX_NZ levels with the most tracers: every level table of the
    kernels is full; the default (fused) path against the oracle and against the
    separate stage and column launches bit for bit."""
    import torch
    c = gen.make_case(40, 24, asuca.MAX_NZ, asuca.MAX_TRACERS, seed=128)
    og = oracle.Grid.from_case(c)
    ref, rbud = oracle.step(og, c.state(), c.mu, c.mv, c.mw, c.dt, 2)
    g0 = asuca.Grid.from_case(c, prec=prec)
    g1 = asuca.Grid.from_case(c, prec=prec)
    asuca.set_tuning(g1, asuca.TUNE_FUSED_COLUMN, 0)
    a = asuca.State.from_case(c, prec=prec)
    b = a.clone()
    ba = asuca.step(g0, a, c.dt, 2, budgets=True)
    bb = asuca.step(g1, b, c.dt, 2, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g0) == asuca.OK and asuca.get_status(g1) == asuca.OK
    assert torch.equal(a.fields(), b.fields())
    _assert_fields(_np(a), ref, tol, f"nz={asuca.MAX_NZ} prec={prec}", both=prec == 0)
    assert np.all(np.abs(ba.cpu().numpy() - rbud) <= tol * np.abs(rbud) + 1e-300)
