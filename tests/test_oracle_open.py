"""Pins of the oracle's open (non-periodic) lateral boundaries (orc_rhs_open,
orc_step_open), CPU only.

* With the periodic continuation as ghosts and the periodic face fluxes
  extended by the last face, the open right-hand side equals the periodic one
  bit for bit (every limiter, with forcing).
* With no lateral mass flux the ghosts do not matter, and two open steps
  (forcing, column physics) equal two periodic steps bit for bit, budgets
  and precipitation included.
* A constant mixing ratio, with the same constant in the ghosts, stays
  constant under non-divergent fluxes (3 steps, 1e-13).
* Inflow: first-order upwind at Courant number 1 (u = 16, dt = 128,
  dx = 2048, rho = 1, integer values) shifts every column by one cell in one
  forward-Euler stage, bit for bit, the inflow column taking the ghost next
  to it; in +-i and +-j.
* Outflow: with first-order upwind, no downstream ghost enters the result;
  with the Koren limiter only the ghost next to the outflow face does.
* Mass: the domain's mass changes by exactly the mass that crossed the outer
  faces (dt times the net outer face flux per step, 1e-13 relative).
"""
import numpy as np
import pytest

import gen
import oracle


def _phi(Y):
    return Y[1:] / Y[0][None]


@pytest.mark.parametrize("lim", [0, 1, 2])
def test_open_rhs_with_periodic_ghosts_equals_periodic_rhs(lim):
    c = gen.make_case(20, 16, 10, 3, seed=5)
    g = oracle.Grid.from_case(c, lim=lim)
    Y = c.state()
    tend = np.random.default_rng(1).uniform(-1e-6, 1e-6, (g.F - 1,) + Y.shape[1:])
    mu_x, mv_x = gen.extend_fluxes(c.mu, c.mv)
    ghost = gen.halo_periodic(_phi(Y))
    a = oracle.rhs_open(g, Y, mu_x, mv_x, c.mw, ghost, tend=tend)
    b = oracle.rhs(g, Y, c.mu, c.mv, c.mw, tend=tend)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("lim", [0, 1])
def test_open_step_without_lateral_flow_equals_periodic_step(lim):
    """With no mass crossing any lateral face (MU = MV = 0 everywhere, the outer
    faces included) the ghosts enter only multiplied by a zero flux, so two
    open steps with forcing and the column physics equal two periodic steps
    bit for bit, budgets and precipitation included: the stage weights, the
    column pass and the budget sums of the open step are the periodic one's."""
    c = gen.make_case(18, 14, 10, 3, seed=8)
    g = oracle.Grid.from_case(c, lim=lim)
    Y = c.state()
    tend = np.random.default_rng(2).uniform(-1e-6, 1e-6, (g.F - 1,) + Y.shape[1:])
    zu, zv = np.zeros_like(c.mu), np.zeros_like(c.mv)
    mu_x, mv_x = gen.extend_fluxes(zu, zv)
    ghost = gen.halo_periodic(_phi(Y))
    a, ba = oracle.step_open(g, Y, mu_x, mv_x, c.mw, ghost, c.dt, 2, tend=tend)
    b, bb = oracle.step(g, Y, zu, zv, c.mw, c.dt, 2, tend=tend)
    assert np.array_equal(a, b)
    assert np.array_equal(ba, bb) and ba[-1] > 0.0


def test_open_step_preserves_constant_mixing_ratio():
    c = gen.make_case(24, 20, 12, 2, seed=6)
    g = oracle.Grid.from_case(c, tau=0.0, k0=0.0, vsed=0.0)
    consts = np.array([301.5, 0.011, 0.004])
    Y = c.state().copy()
    Y[1:] = consts[:, None, None, None] * Y[0][None]
    mu_x, mv_x = gen.extend_fluxes(c.mu, c.mv)
    ghost = gen.halo_periodic(np.broadcast_to(consts[:, None, None, None], Y[1:].shape))
    out, _ = oracle.step_open(g, Y, mu_x, mv_x, c.mw, ghost, c.dt, 3)
    phi = _phi(out)
    for f in range(3):
        assert np.abs(phi[f] - consts[f]).max() <= 1e-13 * consts[f]


def _shift_case(nx, ny, nz, axis, sign):
    """rho = 1, uniform flux of 16 along one axis, integer phi and ghosts."""
    rng = np.random.default_rng(11)
    F = 3
    Y = np.ones((F, nz, ny, nx))
    Y[1:] = rng.integers(-50, 50, (F - 1, nz, ny, nx)).astype(np.float64)
    mu_x = np.zeros((nz, ny, nx + 1))
    mv_x = np.zeros((nz, ny + 1, nx))
    (mu_x if axis == 0 else mv_x)[...] = 16.0 * sign
    mw = np.zeros((nz + 1, ny, nx))
    T = F - 1
    ghost = rng.integers(-50, 50, 2 * (2 * ny + 2 * nx) * nz * T).astype(np.float64)
    g = oracle.Grid(nx, ny, nz, F - 2, np.full(nz, 100.0), dx=2048.0, dy=2048.0, lim=oracle.LIM_UPWIND1,
                    tau=0.0, k0=0.0, vsed=0.0)
    return g, Y, mu_x, mv_x, mw, ghost


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1)])
def test_open_inflow_courant_one_shift_is_exact(axis, sign):
    nx, ny, nz = 9, 7, 3
    g, Y, mu_x, mv_x, mw, ghost = _shift_case(nx, ny, nz, axis, sign)
    out = Y + 128.0 * oracle.rhs_open(g, Y, mu_x, mv_x, mw, ghost)
    W, E, S, N = gen.halo_strips(ghost, 2, nz, ny, nx)
    phi = Y[1:]
    ax = 3 if axis == 0 else 2
    expect = np.roll(phi, sign, axis=ax)
    if axis == 0 and sign > 0:
        expect[..., :, 0] = W[:, :, 1, :]           # ghost i = -1
    elif axis == 0:
        expect[..., :, nx - 1] = E[:, :, 0, :]      # ghost i = nx
    elif sign > 0:
        expect[..., 0, :] = S[:, :, 1, :]           # ghost j = -1
    else:
        expect[..., ny - 1, :] = N[:, :, 0, :]      # ghost j = ny
    assert np.array_equal(out[1:], expect)
    assert np.array_equal(out[0], Y[0])


def _perturb_strip(ghost, which, c_sel, T, nz, ny, nx, rng):
    g2 = ghost.copy()
    strips = gen.halo_strips(g2, T, nz, ny, nx)
    for c in c_sel:
        strips[which][:, :, c, :] += rng.standard_normal(strips[which][:, :, c, :].shape)
    return g2


def test_open_outflow_reads_no_ghost_upwind_and_only_the_adjacent_one_koren():
    nx, ny, nz = 12, 9, 4
    c = gen.make_case(nx, ny, nz, 2, seed=9)
    Y = c.state()
    mu_x = np.full((nz, ny, nx + 1), 5.0)           # eastward everywhere: E is the outflow side
    mv_x = np.zeros((nz, ny + 1, nx))
    mw = np.zeros((nz + 1, ny, nx))
    T = 3
    rng = np.random.default_rng(4)
    ghost = gen.halo_periodic(_phi(Y))
    for lim, untouched in ((oracle.LIM_UPWIND1, (0, 1)), (oracle.LIM_KOREN, (1,))):
        g = oracle.Grid.from_case(c, lim=lim)
        a = oracle.rhs_open(g, Y, mu_x, mv_x, mw, ghost)
        b = oracle.rhs_open(g, Y, mu_x, mv_x, mw, _perturb_strip(ghost, 1, untouched, T, nz, ny, nx, rng))
        assert np.array_equal(a, b)
    # with Koren the ghost next to the outflow face is the downwind cell of that face
    g = oracle.Grid.from_case(c, lim=oracle.LIM_KOREN)
    a = oracle.rhs_open(g, Y, mu_x, mv_x, mw, ghost)
    b = oracle.rhs_open(g, Y, mu_x, mv_x, mw, _perturb_strip(ghost, 1, (0,), T, nz, ny, nx, rng))
    assert not np.array_equal(a, b)


def test_open_step_mass_changes_by_outer_face_flux():
    c = gen.make_case(20, 18, 10, 2, seed=12)
    g = oracle.Grid.from_case(c)
    mu_x, mv_x = gen.extend_fluxes(c.mu, c.mv)
    mu_x = mu_x.copy()
    mv_x = mv_x.copy()
    mu_x[:, :, 0] *= 1.1                              # net inflow through the west faces
    mv_x[:, -1, :] *= 0.8                             # and a changed outflow in the north
    Y = c.state()
    ghost, _ = gen.make_open_boundary(c, seed=3)
    nsteps = 3
    out, bud = oracle.step_open(g, Y, mu_x, mv_x, c.mw, ghost, c.dt, nsteps)
    dz = c.dz[:, None]
    outer = (np.sum((mu_x[:, :, -1] - mu_x[:, :, 0]) * dz) * c.dy +
             np.sum((mv_x[:, -1, :] - mv_x[:, 0, :]) * dz) * c.dx)
    m0 = np.sum(Y[0] * c.dz[:, None, None]) * c.dx * c.dy
    m1 = np.sum(out[0] * c.dz[:, None, None]) * c.dx * c.dy
    assert abs((m1 - m0) - (-nsteps * c.dt * outer)) <= 1e-13 * m0
    assert abs(bud[0] - m1) <= 1e-13 * m0
