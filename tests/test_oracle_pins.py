"""Pins of the FP64 oracle against what the scheme and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped flux
term, a wrong sign or index, swapped MU/MV, a wrong RK weight, a wrong lid or
ghost rule, a transposed Thomas coefficient) fails at least one of them.
"""
import cmath
import math
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _physics_off(case, **kw):
    return oracle.Grid.from_case(case, tau=0.0, k0=0.0, vsed=0.0, **kw)


# ------------------------------------------------------------------ limiter

def _hand_table():
    rows = []
    with open(os.path.join(GOLDEN, "koren_hand_table.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            d0, d1, L, br = line.split()
            rows.append((float(d0), float(d1), float(L), int(br)))
    return rows


@pytest.mark.parametrize("row", _hand_table())
def test_koren_hand_table(row):
    d0, d1, L, br = row
    v, b = oracle.limiter(d0, d1)
    assert v == L and b == br


def test_koren_matches_psi_of_r_with_division():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        d0 = rng.normal() * 10 ** rng.uniform(-3, 3)
        d1 = rng.normal() * 10 ** rng.uniform(-3, 3)
        r = d1 / d0
        psi = max(0.0, min(2 * r, (1 + 2 * r) / 3, 2.0))
        v, _ = oracle.limiter(d0, d1)
        assert abs(v - psi * d0) <= 4e-16 * max(abs(d0), abs(d1)) * 4


def test_limiter_modes_linear_and_upwind():
    for d0, d1 in [(1.0, 2.0), (-1.0, 3.0), (0.5, -0.25)]:
        v, b = oracle.limiter(d0, d1, oracle.LIM_LINEAR)
        assert v == (d0 + 2 * d1) / 3 and b == 2
        v, b = oracle.limiter(d0, d1, oracle.LIM_UPWIND1)
        assert v == 0.0 and b == 0


def test_face_upwind_side_follows_flux_sign():
    # M >= 0: upwind cell i with neighbours (i-1, i+1); M < 0: mirror around i+1
    v, _ = oracle.face(0.0, 1.0, 2.0, 10.0, 1.0, oracle.LIM_LINEAR)
    assert v == 1.0 + 0.5 * (1.0 + 2.0 * 1.0) / 3.0
    v, _ = oracle.face(10.0, 2.0, 1.0, 0.0, -1.0, oracle.LIM_LINEAR)
    assert v == 1.0 + 0.5 * ((1.0 - 0.0) + 2.0 * (2.0 - 1.0)) / 3.0
    # M = 0 counts as M >= 0
    a, _ = oracle.face(0.0, 1.0, 2.0, 10.0, 0.0, oracle.LIM_LINEAR)
    b, _ = oracle.face(0.0, 1.0, 2.0, 10.0, 1e-300, oracle.LIM_LINEAR)
    assert a == b


# ------------------------------------------------------------------ flux form

def _uniform_case(nx, ny, nz, ntr, u=0.0, v=0.0, w=0.0, dz=None, rng=None, integer=False):
    """rho = 1 and uniform M on a grid; tracers random (integers if asked)."""
    rng = rng or np.random.default_rng(7)
    dz = np.full(nz, 100.0) if dz is None else dz
    F = 2 + ntr
    Y = np.empty((F, nz, ny, nx))
    Y[0] = 1.0
    if integer:
        Y[1:] = rng.integers(-50, 50, (F - 1, nz, ny, nx)).astype(np.float64)
    else:
        Y[1:] = rng.uniform(0.5, 1.5, (F - 1, nz, ny, nx))
    mu = np.full((nz, ny, nx), float(u))
    mv = np.full((nz, ny, nx), float(v))
    mw = np.full((nz + 1, ny, nx), float(w))
    mw[0] = 0.0
    mw[nz] = 0.0
    return Y, mu, mv, mw, dz


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1)])
def test_courant_one_upwind_shift_is_bit_exact(axis, sign):
    """One forward-Euler stage of first-order upwind at Courant 1 moves every
    value exactly one cell downstream (powers of two keep all steps exact).
    The spacing across the flow is half the spacing along it, so a flux
    difference divided by the other direction's spacing moves values two
    cells instead of one."""
    nx, ny, nz = 12, 10, 3
    u = 16.0 * sign if axis == 0 else 0.0
    v = 16.0 * sign if axis == 1 else 0.0
    Y, mu, mv, mw, dz = _uniform_case(nx, ny, nz, 2, u=u, v=v, integer=True)
    dx, dy = (2048.0, 1024.0) if axis == 0 else (1024.0, 2048.0)
    g = oracle.Grid(nx, ny, nz, 2, dz, dx, dy, tau=0, k0=0, vsed=0, lim=oracle.LIM_UPWIND1)
    out = oracle.euler(g, Y, mu, mv, mw, 128.0)
    expect = np.roll(Y, sign, axis=3 if axis == 0 else 2)
    assert np.array_equal(out, expect)


def test_courant_one_vertical_shift_with_lids():
    """Upward Courant-1 upwind stage: interior cells take the value from below,
    the bottom cell empties through its lid-closed lower face, the top cell
    keeps its own value plus the inflow (rigid lids carry no flux)."""
    nx, ny, nz = 4, 4, 6
    Y, mu, mv, mw, dz = _uniform_case(nx, ny, nz, 1, w=16.0, dz=np.full(6, 2048.0),
                                      integer=True)
    g = oracle.Grid(nx, ny, nz, 1, dz, 2000.0, 2000.0, tau=0, k0=0, vsed=0,
                    lim=oracle.LIM_UPWIND1)
    out = oracle.euler(g, Y, mu, mv, mw, 128.0)
    exp = np.empty_like(Y)
    exp[:, 1:nz - 1] = Y[:, 0:nz - 2]
    exp[:, 0] = 0.0
    exp[:, nz - 1] = Y[:, nz - 1] + Y[:, nz - 2]
    assert np.array_equal(out, exp)


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("mode,u", [(1, 20.0), (3, -13.0), (5, 7.5)])
def test_linear_fourier_mode_rk3_closed_form(axis, mode, u):
    """kappa=1/3 upwind-biased fluxes with WS-RK3 on a single Fourier mode:
    the amplitude evolves exactly as P(lambda dt)^n, P(z) = 1 + z + z^2/2 + z^3/6,
    lambda = -(u/dx)(1 - e^{-i th})(5 - e^{-i th} + 2 e^{i th})/6 for u >= 0,
    dx the spacing along the mode (the spacing across it is different)."""
    n, nz, nsteps = 32, 3, 7
    dx = 2000.0
    dt = 0.6 * dx / abs(u)
    th = 2 * math.pi * mode / n
    ph = 0.3
    idx = np.arange(n)
    prof = 1.0 + 0.1 * np.cos(th * idx + ph)
    nx, ny = (n, 4) if axis == 0 else (4, n)
    Y = np.empty((3, nz, ny, nx))
    Y[0] = 1.0
    Y[1] = prof[None, None, :] if axis == 0 else prof[None, :, None]
    Y[2] = 2.0
    mu = np.full((nz, ny, nx), u if axis == 0 else 0.0)
    mv = np.full((nz, ny, nx), u if axis == 1 else 0.0)
    mw = np.zeros((nz + 1, ny, nx))
    g = oracle.Grid(nx, ny, nz, 1, np.full(nz, 50.0), dx if axis == 0 else 1250.0,
                    dx if axis == 1 else 1250.0, tau=0, k0=0, vsed=0, lim=oracle.LIM_LINEAR)
    for _ in range(nsteps):
        Y = oracle.rk3(g, Y, mu, mv, mw, dt)
    s = 1.0 if u >= 0 else -1.0
    e = cmath.exp(-1j * s * th)
    ep = cmath.exp(1j * s * th)
    lam = -(abs(u) / dx) * (1 - e) * (5 - e + 2 * ep) / 6
    z = lam * dt
    amp = (1 + z + z * z / 2 + z ** 3 / 6) ** nsteps
    exact = 1.0 + 0.1 * np.real(amp * np.exp(1j * (th * idx + ph)))
    got = Y[1, 1, 0, :] if axis == 0 else Y[1, 1, :, 0]
    assert np.abs(got - exact).max() < 1e-13
    assert np.abs(Y[2] - 2.0).max() < 1e-14
    assert np.array_equal(Y[0], np.ones_like(Y[0]))


def test_constant_forcing_rk3_is_exact():
    """With M = 0 the RHS is the tendency alone and RK3 adds dt * tendency."""
    nx, ny, nz = 6, 5, 4
    Y, mu, mv, mw, dz = _uniform_case(nx, ny, nz, 2)
    rng = np.random.default_rng(3)
    tend = rng.uniform(-1e-3, 1e-3, (3, nz, ny, nx))
    g = oracle.Grid(nx, ny, nz, 2, dz, tau=0, k0=0, vsed=0)
    out = oracle.rk3(g, Y, mu, mv, mw, 40.0, tend=tend)
    assert np.array_equal(out[0], Y[0])
    assert np.abs(out[1:] - (Y[1:] + 40.0 * tend)).max() < 1e-15


# ------------------------------------------------------------------ invariants

def test_mass_and_tracer_conservation_20_steps():
    c = gen.make_config_case("fp64_32x32x16")
    g = oracle.Grid.from_case(c)                    # all physics on
    Y0 = c.state()
    Y, bud = oracle.step(g, Y0, c.mu, c.mv, c.mw, c.dt, 20)
    b0 = oracle.budgets(g, Y0)
    F = g.F
    assert abs(bud[0] - b0[0]) <= 1e-13 * abs(b0[0])
    for n in range(g.ntr):
        extra = bud[F] if n == g.ntr - 1 else 0.0   # the sedimenting tracer rains out
        assert abs(bud[2 + n] + extra - b0[2 + n]) <= 1e-13 * abs(b0[2 + n])
    assert bud[F] > 0.0


@pytest.mark.parametrize("lim", [oracle.LIM_KOREN, oracle.LIM_LINEAR])
def test_constant_tracer_is_preserved(lim):
    c = gen.make_config_case("fp64_32x32x16")
    g = oracle.Grid.from_case(c, vsed=0.0, lim=lim)  # relaxation + diffusion on
    Y0 = c.state()
    Y0[2] = 0.01 * Y0[0]
    Y, _ = oracle.step(g, Y0, c.mu, c.mv, c.mw, c.dt, 20)
    q = Y[2] / Y[0]
    assert np.abs(q - 0.01).max() <= 1e-13 * 0.01


@pytest.mark.parametrize("dy", [gen.DY, 1600.0])
def test_density_constant_under_nondivergent_flux(dy):
    """The generated mass fluxes satisfy discrete continuity (MW built from
    the horizontal divergence with the grid's own dx and dy), so the density
    stays constant, also with dx != dy."""
    c = gen.make_case(32, 32, 16, 3, seed=gen.SEED_BASE, dy=dy)
    g = _physics_off(c)
    Y = oracle.rk3(g, c.state(), c.mu, c.mv, c.mw, c.dt)
    assert np.abs(Y[0] - c.rho).max() <= 1e-13 * c.rho.max()


def test_overturning_exercises_vertical_flux():
    c = gen.make_config_case("fp64_32x32x16")
    assert np.abs(c.mw[1:-1]).max() > 0.01
    assert np.all(c.mw[0] == 0) and np.all(c.mw[-1] == 0)
    c0 = gen.make_config_case("fp64_32x32x16", overturning=False)
    assert np.all(c0.mw == 0)


# ------------------------------------------------------------------ time order

def test_third_order_temporal_convergence():
    # the 32x32x16 workload's fields on a 16x16 plane (a quarter of the work)
    c = gen.make_config_case("fp64_32x32x16", nx=16, ny=16)
    g = oracle.Grid.from_case(c, tau=0, k0=0, vsed=0, lim=oracle.LIM_LINEAR)
    T = 8 * c.dt
    Y0 = c.state()

    def run(n):
        Y = Y0
        for _ in range(n):
            Y = oracle.rk3(g, Y, c.mu, c.mv, c.mw, T / n)
        return Y

    ref = run(8 * 16)
    errs = [np.sqrt(np.mean((run(8 * m)[2:] - ref[2:]) ** 2)) for m in (1, 2, 4)]
    ratios = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert all(2.8 <= r <= 3.2 for r in ratios), (errs, ratios)


# ------------------------------------------------------------------ column physics

@pytest.mark.parametrize("n", [3, 16, 58])
def test_thomas_matches_dense_solve(n):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(n)
    for _ in range(20):
        a = rng.uniform(-1, 1, n)
        c = rng.uniform(-1, 1, n)
        a[0] = 0.0
        c[-1] = 0.0
        b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 2.0, n)
        d = rng.normal(size=n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        x = oracle.thomas(a, b, c, d)
        ref = scipy_linalg.solve(A, d)
        assert np.abs(x - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def _one_column_grid(nz, **kw):
    dz = gen.make_dz(nz)
    return oracle.Grid(1, 1, nz, 2, dz, **kw), dz


def test_diffusion_conserves_and_matches_dense_system():
    nz = 58
    g, dz = _one_column_grid(nz, tau=0, vsed=0)
    rng = np.random.default_rng(11)
    Y = np.empty((4, nz, 1, 1))
    zf = np.concatenate([[0.0], np.cumsum(dz)])
    zc = zf[:-1] + dz / 2
    Y[0, :, 0, 0] = 1.2 * np.exp(-zc / 8000) * (1 + 0.01 * rng.normal(size=nz))
    Y[1:, :, 0, 0] = Y[0, :, 0, 0] * rng.uniform(0.5, 1.5, (3, nz))
    dt = 80.0
    out, _ = oracle.column(g, Y, dt)
    rho = Y[0, :, 0, 0]
    # dense system built independently from the definition of the implicit diffusion
    A = np.zeros((nz, nz))
    for k in range(nz - 1):
        gk = dt * 0.5 * (rho[k] + rho[k + 1]) * 50.0 * np.exp(-zf[k + 1] / 1000.0) / (zc[k + 1] - zc[k])
        A[k, k] += gk
        A[k + 1, k + 1] += gk
        A[k, k + 1] -= gk
        A[k + 1, k] -= gk
    A += np.diag(rho * dz)
    for f in range(1, 4):
        phi = np.linalg.solve(A, dz * Y[f, :, 0, 0])
        assert np.abs(out[f, :, 0, 0] - rho * phi).max() <= 1e-13 * np.abs(rho * phi).max()
        s0 = np.sum(Y[f, :, 0, 0] * dz)
        assert abs(np.sum(out[f, :, 0, 0] * dz) - s0) <= 1e-14 * abs(s0)
    assert np.array_equal(out[0], Y[0])
    # a constant mixing ratio does not diffuse
    Yc = Y.copy()
    Yc[1:] = 0.37 * Y[0]
    outc, _ = oracle.column(g, Yc, dt)
    assert np.abs(outc[1:] / outc[0] - 0.37).max() < 1e-14


def test_sedimentation_single_cell_and_column_closure():
    g1 = oracle.Grid(1, 1, 1, 1, np.array([100.0]), tau=0, k0=0, vsed=2.0)
    Y = np.array([1.0, 300.0, 0.015]).reshape(3, 1, 1, 1)
    out, pc = oracle.column(g1, Y, 40.0)
    assert out[2, 0, 0, 0] == 0.015 * 100.0 / (100.0 + 40.0 * 2.0)
    assert abs(pc[0, 0] - 40.0 * 2.0 * out[2, 0, 0, 0] * 2000.0 * 2000.0) < 1e-12
    # two levels by hand: the top level feeds the bottom one
    g2 = oracle.Grid(1, 1, 2, 1, np.array([100.0, 200.0]), tau=0, k0=0, vsed=2.0)
    Y2 = np.array([[1.0, 1.0], [300.0, 300.0], [0.01, 0.02]]).reshape(3, 2, 1, 1)
    out2, pc2 = oracle.column(g2, Y2, 40.0)
    top = 0.02 * 200.0 / (200.0 + 80.0)
    bot = (0.01 * 100.0 + 40.0 * 2.0 * top) / (100.0 + 80.0)
    assert out2[2, 1, 0, 0] == top and out2[2, 0, 0, 0] == bot
    # column budget closure on a real column: sum(rho q dz) + precip / (dx dy) is unchanged
    c = gen.make_config_case("fp64_32x32x16")
    g = oracle.Grid.from_case(c, tau=0, k0=0)
    Y0 = c.state()
    out, pc = oracle.column(g, Y0, c.dt)
    s0 = (Y0[-1] * c.dz[:, None, None]).sum(axis=0)
    s1 = (out[-1] * c.dz[:, None, None]).sum(axis=0) + pc / (c.dx * c.dy)
    assert np.abs(s1 - s0).max() <= 1e-14 * np.abs(s0).max()
    assert np.array_equal(out[:-1], Y0[:-1])


def test_relaxation_closed_form_and_fixed_point():
    nz = 16
    g, dz = _one_column_grid(nz, k0=0, vsed=0, tau=3600.0)
    zf = np.concatenate([[0.0], np.cumsum(dz)])
    zc = zf[:-1] + dz / 2
    thref = 300.0 + 0.004 * zc
    Y = np.empty((4, nz, 1, 1))
    Y[0, :, 0, 0] = 1.1
    Y[1, :, 0, 0] = 1.1 * thref
    Y[2:] = 0.0
    out, _ = oracle.column(g, Y, 90.0)
    assert np.abs(out[1, :, 0, 0] / 1.1 - thref).max() < 1e-12
    Y[1, :, 0, 0] = 1.1 * (thref + 2.0)
    out, _ = oracle.column(g, Y, 90.0)
    r = 90.0 / 3600.0
    assert np.abs(out[1, :, 0, 0] / 1.1 - (thref + 2.0 / (1 + r))).max() < 1e-12


# ------------------------------------------------------------------ windows

@pytest.mark.parametrize("forced", [False, True])
def test_window_step_equals_full_domain_step(forced):
    c = gen.make_config_case("fp64_32x32x16")
    g = oracle.Grid.from_case(c)
    Y0 = c.state()
    tend = np.random.default_rng(4).uniform(-1e-6, 1e-6, (g.F - 1,) + Y0.shape[1:]) if forced else None
    Yf, _ = oracle.step(g, Y0, c.mu, c.mv, c.mw, c.dt, 2, tend=tend)
    for (i0, j0, w, h) in [(30, 5, 4, 3), (0, 0, 1, 1), (31, 31, 2, 2)]:
        win = oracle.step_window(g, Y0, c.mu, c.mv, c.mw, c.dt, 2, i0, j0, w, h, tend=tend)
        ii = [(i0 + q) % c.nx for q in range(w)]
        jj = [(j0 + q) % c.ny for q in range(h)]
        ref = Yf[:, :, jj][:, :, :, ii]
        assert np.array_equal(win, ref)


def test_thread_count_does_not_change_results():
    c = gen.make_config_case("fp64_32x32x16")
    g = oracle.Grid.from_case(c)
    n0 = oracle.get_threads()
    try:
        oracle.set_threads(1)
        a, ba = oracle.step(g, c.state(), c.mu, c.mv, c.mw, c.dt, 2)
        oracle.set_threads(max(2, n0))
        b, bb = oracle.step(g, c.state(), c.mu, c.mv, c.mw, c.dt, 2)
    finally:
        oracle.set_threads(n0)
    assert np.array_equal(a, b) and np.array_equal(ba, bb)


def test_budgets_are_the_correctly_rounded_sum():
    """Budgets are sums over every cell of f dV (dV = dz_k dx dy).  Against
    Python's math.fsum of the same products (correctly rounded, Shewchuk's
    algorithm), on a field with cancellation and a wide range of magnitudes,
    the oracle's sum agrees to a few ulp of the sum of |terms|; a plain running
    sum over this many terms is off by far more."""
    rng = np.random.default_rng(5)
    nx, ny, nz = 96, 80, 12
    dz = np.geomspace(40.0, 1000.0, nz)
    g = oracle.Grid(nx, ny, nz, 0, dz, 2000.0, 2000.0)
    Y = rng.standard_normal((2, nz, ny, nx)) * 10.0 ** rng.uniform(-3, 6, (2, nz, ny, nx))
    Y[0] += 1e7          # a large common offset, as a mass budget has
    out = oracle.budgets(g, Y, precip=0.25)
    for f in range(2):
        terms = ((Y[f] * dz[:, None, None]) * 2000.0) * 2000.0
        exact = math.fsum(terms.ravel().tolist())
        scale = math.fsum(np.abs(terms).ravel().tolist())
        assert abs(out[f] - exact) <= 4 * np.finfo(float).eps * scale, (f, out[f], exact)
        if f == 1:   # the cancelling field: correct to a few ulp of the result itself
            assert abs(out[f] - exact) <= 4 * np.finfo(float).eps * abs(exact) + 1e-300
        # the bound is tight enough to tell: a plain running sum in the same order misses it
        plain = np.cumsum(terms.transpose(1, 2, 0).ravel())[-1]
        assert abs(plain - exact) > 4 * np.finfo(float).eps * scale
    assert out[2] == 0.25


@pytest.mark.parametrize("w", [1.0, -1.0])
def test_vertical_kappa_third_exact_for_quadratics_and_ghosts(w):
    """The kappa=1/3 face value is exact for cell averages of z^2: with
    phi_k = k^2 + 1/12 (average of z^2 over [k-1/2, k+1/2]) every face whose
    stencil is interior gets (k+1/2)^2.  Next to a lid the ghost copies the
    boundary cell, so d0 = 0 there and the face is phi_up + (phi_down - phi_up)/3."""
    from fractions import Fraction as Fr
    nz = 9
    phi = [Fr(k * k) + Fr(1, 12) for k in range(nz)]
    face = {}
    for k in range(nz - 1):                       # face k+1/2
        if w > 0 and k == 0:
            face[k] = phi[0] + (phi[1] - phi[0]) / 3
        elif w < 0 and k == nz - 2:
            face[k] = phi[nz - 1] + (phi[nz - 2] - phi[nz - 1]) / 3
        else:
            face[k] = (Fr(2 * k + 1, 2)) ** 2
    Zp = lambda k: Fr(0) if k < 0 or k >= nz - 1 else Fr(int(w)) * face[k]
    expect = [-(Zp(k) - Zp(k - 1)) for k in range(nz)]
    Y = np.empty((3, nz, 4, 4))
    Y[0] = 1.0
    Y[1] = np.array([float(p) for p in phi])[:, None, None]
    Y[2] = 1.0
    mu = np.zeros((nz, 4, 4))
    mv = np.zeros((nz, 4, 4))
    mw = np.full((nz + 1, 4, 4), w)
    mw[0] = mw[nz] = 0.0
    g = oracle.Grid(4, 4, nz, 1, np.ones(nz), tau=0, k0=0, vsed=0, lim=oracle.LIM_LINEAR)
    R = oracle.rhs(g, Y, mu, mv, mw)
    got = R[1, :, 2, 1]
    assert np.abs(got - np.array([float(e) for e in expect])).max() < 1e-12


# ------------------------------------------------------------------ 7-point diffusion stencil (Sec. 4)

def test_stencil7_constant_and_conservation():
    """A constant field is a fixed point; periodic sides and zero-flux lids
    conserve the total (every interior difference enters two cells with opposite
    signs), to rounding."""
    c = 0.12
    const = np.full((6, 9, 11), 3.25)
    assert np.array_equal(oracle.stencil7(const, c), const)
    f = np.random.default_rng(3).standard_normal((7, 10, 13))
    out = oracle.stencil7(f, c)
    assert abs(out.sum() - f.sum()) <= 1e-13 * np.abs(f).sum()


@pytest.mark.parametrize("axis", [0, 1])
def test_stencil7_fourier_mode_closed_form(axis):
    """A level-uniform periodic Fourier mode cos(2 pi m x / n) along i (or j) is an
    eigenvector with eigenvalue 1 + c (2 cos(2 pi m / n) - 2)."""
    nz, ny, nx, m, c = 4, 12, 16, 3, 0.09
    n = nx if axis == 0 else ny
    x = np.arange(n)
    mode = np.cos(2 * np.pi * m * x / n + 0.4)
    f = np.broadcast_to(mode[None, None, :] if axis == 0 else mode[None, :, None], (nz, ny, nx)).copy()
    lam = 1.0 + c * (2.0 * np.cos(2 * np.pi * m / n) - 2.0)
    assert np.max(np.abs(oracle.stencil7(f, c) - lam * f)) <= 1e-13


def test_stencil7_linear_in_k_with_zero_flux_lids():
    """f = k: the interior Laplacian of a linear profile is zero; at the bottom the
    ghost copies level 0, so out = 0 + c (1 - 0), at the top out = (nz-1) - c."""
    nz, ny, nx, c = 9, 5, 6, 0.2
    f = np.broadcast_to(np.arange(nz, dtype=float)[:, None, None], (nz, ny, nx)).copy()
    out = oracle.stencil7(f, c)
    assert np.array_equal(out[1:-1], f[1:-1])
    assert np.allclose(out[0], c, rtol=0, atol=1e-15)
    assert np.allclose(out[-1], (nz - 1) - c, rtol=0, atol=1e-14)


# ------------------------------------------------------------------ lateral and upper damping (Sec. 2.1)

def _damp_fields(F, nz, ny, nx, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((F, nz, ny, nx)) for _ in range(4)]


def test_damping_touches_exactly_the_zone():
    """Only cells fewer than `width` cells from an i or j edge, or on the top
    ntop levels, change; their number is the closed-form zone size
    ntop nx ny + (nz - ntop) (nx ny - (nx - 2 width)(ny - 2 width))."""
    F, nz, ny, nx, W, ntop = 3, 7, 11, 17, 3, 2
    Y, R, B0, B1 = _damp_fields(F, nz, ny, nx, 1)
    out = oracle.damping(Y, R, B0, B1, 0.3, 40.0, width=W, ntop=ntop, nu_lat=1e-2, nu_top=5e-3)
    changed = np.any(out != Y, axis=0)
    assert changed.sum() == ntop * nx * ny + (nz - ntop) * (nx * ny - (nx - 2 * W) * (ny - 2 * W))
    kk, jj, ii = np.nonzero(changed)
    d = np.minimum(np.minimum(ii, nx - 1 - ii), np.minimum(jj, ny - 1 - jj))
    assert np.all((d < W) | (kk >= nz - ntop))


def test_damping_zero_rate_is_the_identity():
    Y, R, B0, B1 = _damp_fields(2, 5, 9, 10, 2)
    out = oracle.damping(Y, R, B0, B1, 0.7, 30.0, width=4, ntop=5, nu_lat=0.0, nu_top=0.0)
    assert np.array_equal(out, Y)


@pytest.mark.parametrize("tratio", [0.0, 0.3, 1.0])
def test_damping_strong_limit_is_the_interpolated_boundary_state(tratio):
    """With a very large rate the implicit relaxation lands on its target, and
    with mtratio = 1 - tratio the reference terms of the paper's target cancel:
    target = ref + (1 - tratio) bnd0 + tratio bnd1."""
    F, nz, ny, nx = 2, 4, 8, 9
    Y, R, B0, B1 = _damp_fields(F, nz, ny, nx, 3)
    out = oracle.damping(Y, R, B0, B1, tratio, 1.0, width=1, ntop=1, nu_lat=1e15, nu_top=1e15)
    want = R + (1.0 - tratio) * B0 + tratio * B1
    edge = np.zeros((nz, ny, nx), bool)
    edge[:, 0, :] = edge[:, -1, :] = edge[:, :, 0] = edge[:, :, -1] = True
    edge[-1] = True
    assert np.max(np.abs(out[:, edge] - want[:, edge])) <= 1e-12
    assert np.array_equal(out[:, ~edge], Y[:, ~edge])


def test_damping_strong_limit_with_independent_weights():
    """The target weights the two boundary datasets by mtratio and tratio
    independently (Sec. 2.1's damping kernel; they need not add to one): with
    a very large rate the edge cells land on mtratio (ref + bnd0) +
    tratio (ref + bnd1)."""
    F, nz, ny, nx = 2, 4, 8, 9
    Y, R, B0, B1 = _damp_fields(F, nz, ny, nx, 5)
    out = oracle.damping(Y, R, B0, B1, 0.3, 1.0, width=1, ntop=0, nu_lat=1e15, nu_top=0.0, mtratio=0.55)
    want = 0.55 * (R + B0) + 0.3 * (R + B1)
    edge = np.zeros((nz, ny, nx), bool)
    edge[:, 0, :] = edge[:, -1, :] = edge[:, :, 0] = edge[:, :, -1] = True
    assert np.max(np.abs(out[:, edge] - want[:, edge])) <= 1e-12 * np.abs(want).max()
    assert np.array_equal(out[:, ~edge], Y[:, ~edge])


def test_damping_is_backward_euler_of_the_relaxation_ode():
    """Repeated calls with a fixed target integrate dy/dt = -nu (y - target):
    the result stays between y0 and the target for any step (unconditionally
    stable, monotone), and converges at first order to the exact
    target + (y0 - target) exp(-nu t)."""
    nu, t, y0, T = 1.0 / 300.0, 900.0, 2.0, -1.0
    shape = (1, 1, 2, 2)                   # every cell is an edge cell (d = 0, full rate)
    R = np.full(shape, T)
    Z = np.zeros(shape)
    exact = T + (y0 - T) * math.exp(-nu * t)
    errs = []
    for n in (8, 16, 32, 64):
        y = np.full(shape, y0)
        for _ in range(n):
            y = oracle.damping(y, R, Z, Z, 0.5, t / n, width=1, ntop=0, nu_lat=nu, nu_top=0.0)
            assert np.all((y > T) & (y < y0))
        errs.append(abs(y[0, 0, 0, 0] - exact))
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2
    y = oracle.damping(np.full(shape, y0), R, Z, Z, 0.5, 1e9, width=1, ntop=0, nu_lat=nu, nu_top=0.0)
    assert T < y[0, 0, 0, 0] < T + 1e-6


def test_damping_mirror_symmetry_and_profile_shape():
    """The zone is symmetric under i -> nx-1-i and j -> ny-1-j, and the rate
    falls off from the edges: with y = 1, target = 0 the damped value rises
    strictly from the outermost cell inward (and from the top level down)
    and reaches 1 outside the zone."""
    F, nz, ny, nx, W, ntop = 2, 6, 12, 14, 4, 3
    Y, R, B0, B1 = _damp_fields(F, nz, ny, nx, 4)
    kw = dict(width=W, ntop=ntop, nu_lat=2e-2, nu_top=1e-2)
    out = oracle.damping(Y, R, B0, B1, 0.4, 25.0, **kw)
    flip = lambda a: a[:, :, ::-1, ::-1]
    assert np.array_equal(flip(oracle.damping(flip(Y), flip(R), flip(B0), flip(B1), 0.4, 25.0, **kw)), out)
    one, zero = np.ones((1, nz, ny, nx)), np.zeros((1, nz, ny, nx))
    p = oracle.damping(one, zero, zero, zero, 0.5, 25.0, **kw)[0]
    row = p[0, ny // 2, :nx // 2]          # bottom level, middle row, from the left edge inward
    assert np.all(np.diff(row[:W + 1]) > 0) and np.all(row[W:] == 1.0)
    col = p[nz - ntop - 1:, ny // 2, nx // 2]    # centre column, from below the top zone upward
    assert col[0] == 1.0 and np.all(np.diff(col) < 0)


def test_damping_rate_profile_is_quadratic():
    """The rate one call applies, recovered from y = 1, target = 0 as
    nu = (1 / y' - 1) / dt: the full lateral rate on the edge cells, its square
    root falling by equal amounts per cell to zero at `width` cells from the
    edge; likewise from the top level down over ntop levels; the larger rate
    where the zones overlap."""
    nz, ny, nx, W, ntop, dt = 9, 20, 22, 5, 4, 30.0
    nu_lat, nu_top = 2e-2, 8e-3
    one, zero = np.ones((1, nz, ny, nx)), np.zeros((1, nz, ny, nx))
    p = oracle.damping(one, zero, zero, zero, 0.5, dt, width=W, ntop=ntop, nu_lat=nu_lat, nu_top=nu_top)[0]
    nu = (1.0 / p - 1.0) / dt
    lat = nu[0, ny // 2, :W + 2]                     # bottom level, middle row, from the left edge
    assert abs(lat[0] - nu_lat) <= 1e-12 * nu_lat
    r = np.sqrt(lat[:W + 1] / nu_lat)
    assert np.allclose(np.diff(r), -1.0 / W, rtol=0, atol=1e-9) and lat[W] == 0.0 and lat[W + 1] == 0.0
    top = nu[::-1, ny // 2, nx // 2][:ntop + 1]      # centre column, from the top level down
    assert abs(top[0] - nu_top) <= 1e-12 * nu_top
    r = np.sqrt(top / nu_top)
    assert np.allclose(np.diff(r), -1.0 / ntop, rtol=0, atol=1e-9) and top[ntop] == 0.0
    corner = nu[nz - 1, 0, W - 2]                    # top level, edge row: lateral rate is the larger
    assert abs(corner - nu_lat) <= 1e-12 * nu_lat


def test_damping_sampled_cells_equal_the_whole_domain():
    """The sampled-cell form (explicit (i, j, k) list, [F][n] arrays) gives the
    whole-domain result at those cells."""
    F, nz, ny, nx = 3, 5, 9, 11
    Y, R, B0, B1 = _damp_fields(F, nz, ny, nx, 5)
    kw = dict(width=3, ntop=2, nu_lat=1e-2, nu_top=3e-3)
    full = oracle.damping(Y, R, B0, B1, 0.6, 20.0, **kw)
    rng = np.random.default_rng(6)
    ijk = np.stack([rng.integers(0, nx, 40), rng.integers(0, ny, 40), rng.integers(0, nz, 40)], axis=1)
    g = lambda a: a[:, ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    part = oracle.damping(g(Y), g(R), g(B0), g(B1), 0.6, 20.0, ijk=ijk, shape=(nx, ny, nz), **kw)
    assert np.array_equal(part, g(full))


# ------------------------------------------------------------------ HEVI acoustic short steps (Sec. 1.1)

CS2 = 340.0 ** 2


def _acoustic_base(nz, dz=None, gravity=True):
    dz = np.linspace(60.0, 500.0, nz) if dz is None else np.asarray(dz, float)
    zf = np.concatenate([[0.0], np.cumsum(dz)])
    zc = zf[:-1] + 0.5 * dz
    if not gravity:
        return dz, np.full(nz, 1.2), np.full(nz + 1, 1.2)
    return dz, 1.2 * np.exp(-9.81 * zc / CS2), 1.2 * np.exp(-9.81 * zf / CS2)


def _acoustic_random(nz, ny, nx, seed, uniform=False):
    rng = np.random.default_rng(seed)
    shape = (nz, 1, 1) if uniform else (nz, ny, nx)
    S = np.broadcast_to(rng.standard_normal(shape) * 1e-3, (nz, ny, nx)).copy()
    W = np.broadcast_to(rng.standard_normal((nz + 1,) + shape[1:]) * 0.5, (nz + 1, ny, nx)).copy()
    W[0] = W[-1] = 0.0
    if uniform:
        return np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)), W, S
    return rng.standard_normal((nz, ny, nx)), rng.standard_normal((nz, ny, nx)), W, S


def _acoustic_energy(W, S, dz, r0c, r0f):
    dzc = 0.5 * (dz[:-1] + dz[1:])
    ew = 0.5 * np.sum(W[1:-1] ** 2 * (dzc / (CS2 * r0f[1:-1]))[:, None, None])
    es = 0.5 * np.sum(S ** 2 * (r0c * dz)[:, None, None])
    return ew + es


def test_acoustic_rest_state_and_mass():
    """The resting state stays at rest, and the flux form with periodic sides and
    rigid lids conserves the perturbation mass sum rho0 s dz (to rounding)."""
    nz, ny, nx = 7, 6, 9
    dz, r0c, r0f = _acoustic_base(nz)
    z = [np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)), np.zeros((nz + 1, ny, nx)), np.zeros((nz, ny, nx))]
    out = oracle.acoustic(*z, dz, r0c, r0f, CS2, 0.6, 2.0, 3)
    assert all(np.array_equal(a, b) for a, b in zip(out, z))
    U, V, W, S = _acoustic_random(nz, ny, nx, 1)
    mass = lambda s: np.sum(s * (r0c * dz)[:, None, None])
    scale = np.sum(np.abs(S) * (r0c * dz)[:, None, None])
    out = oracle.acoustic(U, V, W, S, dz, r0c, r0f, CS2, 0.6, 2.0, 5)
    assert abs(mass(out[3]) - mass(S)) <= 1e-13 * scale


def test_acoustic_vertical_mode_is_crank_nicolson_exact():
    """Horizontally uniform, constant rho0 and dz, beta = 1/2: the lid-bounded
    mode s_k = cos(theta (k + 1/2)), theta = pi m / nz, is an eigenvector of the
    vertical operator with frequency omega = 2 c sin(theta / 2) / dz, and the
    trapezoidal (Crank-Nicolson) step turns it by exactly 2 atan(omega h / 2)."""
    nz, ny, nx, m, h, n = 12, 3, 4, 3, 5.0, 9
    dz, r0c, r0f = _acoustic_base(nz, dz=np.full(nz, 250.0), gravity=False)
    th = math.pi * m / nz
    mode = np.cos(th * (np.arange(nz) + 0.5))
    S = np.broadcast_to(mode[:, None, None], (nz, ny, nx)).copy() * 1e-3
    zeros = np.zeros((nz, ny, nx))
    out = oracle.acoustic(zeros, zeros, np.zeros((nz + 1, ny, nx)), S, dz, r0c, r0f, CS2, 0.5, h, n)
    omega = 2.0 * math.sqrt(CS2) * math.sin(th / 2) / 250.0
    phi = 2.0 * math.atan(omega * h / 2)
    assert np.max(np.abs(out[3] - math.cos(n * phi) * S)) <= 1e-15
    # W carries the quadrature part: b_n = sin(n phi) c rho0 a_0 in energy-normalised units
    wmode = np.sin(th * np.arange(nz + 1))
    want_w = math.sin(n * phi) * math.sqrt(CS2) * 1.2 * 1e-3 * wmode
    assert np.max(np.abs(out[2][:, 0, 0] - want_w)) <= 1e-12
    assert np.array_equal(out[0], zeros) and np.array_equal(out[1], zeros)


@pytest.mark.parametrize("beta", [0.5, 0.7])
def test_acoustic_vertical_energy(beta):
    """Horizontally uniform states (gravity base state, stretched levels): the
    discrete acoustic energy sum W^2 dzc / (2 c^2 rho0f) + rho0 dz s^2 / 2 is
    conserved by the centred implicit step and decays for beta > 1/2."""
    nz, ny, nx = 20, 2, 3
    dz, r0c, r0f = _acoustic_base(nz)
    U, V, W, S = _acoustic_random(nz, ny, nx, 2, uniform=True)
    e = [_acoustic_energy(W, S, dz, r0c, r0f)]
    for _ in range(30):
        U, V, W, S = oracle.acoustic(U, V, W, S, dz, r0c, r0f, CS2, beta, 4.0, 1)
        e.append(_acoustic_energy(W, S, dz, r0c, r0f))
    e = np.array(e)
    if beta == 0.5:
        assert np.max(np.abs(e / e[0] - 1.0)) <= 1e-12
    else:
        assert np.all(np.diff(e) < 0) and e[-1] < 0.9 * e[0]


def test_acoustic_off_centring_changes_the_step_at_second_order():
    """beta only shares each implicit vertical term between the new and the
    old state, so every beta gives the same tendency: a short step with
    beta = 0.8 differs from the centred one (beta = 1/2) by O(h^2), while the
    step itself changes W and s by O(h).  Their ratio therefore halves with
    h.  (Weights that do not add to one change the vertical force itself,
    and the ratio then stays of order one.)"""
    nz, ny, nx = 8, 4, 5
    dz, r0c, r0f = _acoustic_base(nz)
    U, V, W, S = _acoustic_random(nz, ny, nx, 4)
    rel = []
    for h in (0.02, 0.01, 0.005, 0.0025):
        a = oracle.acoustic(U, V, W, S, dz, r0c, r0f, CS2, 0.5, h, 1)
        b = oracle.acoustic(U, V, W, S, dz, r0c, r0f, CS2, 0.8, h, 1)
        rel.append(max(np.abs(b[q] - a[q]).max() / np.abs(a[q] - x0).max() for q, x0 in ((2, W), (3, S))))
    for p, q in zip(rel, rel[1:]):
        assert 1.8 < p / q < 2.3, rel
    assert rel[-1] < 0.02


@pytest.mark.parametrize("axis", [0, 1])
def test_acoustic_horizontal_mode_converges_at_second_order(axis):
    """A horizontal acoustic mode s = cos(2 pi m i / n) along i or j (constant
    rho0) has the centred-difference frequency omega = 2 c sin(pi m / n) / d,
    d the spacing along the mode (the other spacing differs); the two-stage
    short step converges to cos(omega t) s at second order in the step, and
    the momentum across the mode stays zero."""
    nz, n, m, T = 3, 16, 2, 10.0                     # omega T = 1.3 / 1.7, away from an extremum of cos
    dx, dy = (2000.0, 1500.0) if axis == 0 else (1500.0, 2000.0)
    nx, ny = (n, 2) if axis == 0 else (2, n)
    dz, r0c, r0f = _acoustic_base(nz, gravity=False)
    mode = np.cos(2 * math.pi * m * np.arange(n) / n)
    shape = (1, 1, n) if axis == 0 else (1, n, 1)
    S0 = np.broadcast_to(mode.reshape(shape), (nz, ny, nx)).copy() * 1e-3
    omega = 2.0 * math.sqrt(CS2) * math.sin(math.pi * m / n) / (dx if axis == 0 else dy)
    errs = []
    for ns in (8, 16, 32, 64):
        z = np.zeros((nz, ny, nx))
        out = oracle.acoustic(z, z, np.zeros((nz + 1, ny, nx)), S0, dz, r0c, r0f, CS2, 0.6, T / ns, ns,
                              dx=dx, dy=dy)
        errs.append(np.max(np.abs(out[3] - math.cos(omega * T) * S0)))
        assert np.max(np.abs(out[2])) <= 1e-15      # no vertical motion from a k-uniform mode
        assert np.array_equal(out[1 - axis], z)     # none across the mode
    for a, b in zip(errs, errs[1:]):
        assert 3.9 < a / b < 4.1


def test_acoustic_i_j_transposition_symmetry():
    """With dx = dy, transposing i and j (and swapping U and V) transposes the
    result bit for bit; the lids of W are left as they are."""
    nz, n = 5, 8
    dz, r0c, r0f = _acoustic_base(nz)
    U, V, W, S = _acoustic_random(nz, n, n, 3)
    W[0], W[-1] = 5.0, -3.0
    t = lambda a: np.ascontiguousarray(np.swapaxes(a, 1, 2))
    a = oracle.acoustic(U, V, W, S, dz, r0c, r0f, CS2, 0.6, 2.0, 2)
    b = oracle.acoustic(t(V), t(U), t(W), t(S), dz, r0c, r0f, CS2, 0.6, 2.0, 2)
    assert np.array_equal(t(b[1]), a[0]) and np.array_equal(t(b[0]), a[1])
    assert np.array_equal(t(b[2]), a[2]) and np.array_equal(t(b[3]), a[3])
    assert np.all(a[2][0] == 5.0) and np.all(a[2][-1] == -3.0)
    W0 = W.copy()
    W0[0] = W0[-1] = 0.0
    c = oracle.acoustic(U, V, W0, S, dz, r0c, r0f, CS2, 0.6, 2.0, 2)
    assert np.array_equal(c[3], a[3]) and np.array_equal(c[2][1:-1], a[2][1:-1])
