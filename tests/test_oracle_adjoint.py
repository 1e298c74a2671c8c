"""Pins of the oracle's tangent-linear and adjoint (FP64, CPU).

* dot-product tests <TL dx, dy> = <dx, AD dy> for the RHS, the column pass
  and whole steps (branches frozen; exact up to rounding);
* the TL against central differences of the nonlinear oracle (also with
  dx != dy);
* the adjoint gradient of J = 1/2 sum (q - q_target)^2 against central
  differences (eps = 1e-6) on seeded directions scaled by each field's RMS,
  redrawing any direction whose perturbed trajectories change a limiter
  branch or the sign of a mass flux.
"""
import numpy as np
import pytest

import gen
import oracle


def _case(nx=12, ny=10, nz=8, ntr=2, seed=5, dy=gen.DY):
    c = gen.make_case(nx, ny, nz, ntr, seed=seed, dy=dy)
    return c, oracle.Grid.from_case(c)


def _dirs(rng, c):
    Y = c.state()
    dY = rng.standard_normal(Y.shape) * np.sqrt(np.mean(Y ** 2, axis=(1, 2, 3)))[:, None, None, None]
    dmu = rng.standard_normal(c.mu.shape) * np.sqrt(np.mean(c.mu ** 2))
    dmv = rng.standard_normal(c.mv.shape) * np.sqrt(np.mean(c.mv ** 2))
    dmw = rng.standard_normal(c.mw.shape) * np.sqrt(np.mean(c.mw ** 2))
    dmw[0] = dmw[-1] = 0.0
    return dY, dmu, dmv, dmw


def _dot(*pairs):
    return sum(float(np.sum(a * b)) for a, b in pairs)


@pytest.mark.parametrize("lim", [0, 1, 2])
def test_rhs_dot_product(lim):
    c, _ = _case()
    g = oracle.Grid.from_case(c, lim=lim)
    rng = np.random.default_rng(1)
    Y = c.state() * (1 + 0.01 * rng.standard_normal(c.state().shape))
    dY, dmu, dmv, dmw = _dirs(rng, c)
    lam = rng.standard_normal(Y.shape)
    dR = oracle.rhs_tl(g, Y, c.mu, c.mv, c.mw, dY, dmu, dmv, dmw)
    lY, gmu, gmv, gmw = oracle.rhs_adj(g, Y, c.mu, c.mv, c.mw, lam)
    lhs = _dot((dR, lam))
    rhs = _dot((dY, lY), (dmu, gmu), (dmv, gmv), (dmw, gmw))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("dy", [gen.DY, 1500.0])
def test_rhs_tl_matches_central_differences(dy):
    c, g = _case(dy=dy)
    rng = np.random.default_rng(2)
    Y = c.state()
    dY, dmu, dmv, dmw = _dirs(rng, c)
    eps = 1e-6
    Rp, bp = oracle.rhs(g, Y + eps * dY, c.mu + eps * dmu, c.mv + eps * dmv, c.mw + eps * dmw, branches=True)
    Rm, bm = oracle.rhs(g, Y - eps * dY, c.mu - eps * dmu, c.mv - eps * dmv, c.mw - eps * dmw, branches=True)
    _, b0 = oracle.rhs(g, Y, c.mu, c.mv, c.mw, branches=True)
    tl = oracle.rhs_tl(g, Y, c.mu, c.mv, c.mw, dY, dmu, dmv, dmw)
    fd = (Rp - Rm) / (2 * eps)
    face_same = (bp == b0) & (bm == b0)          # each cell's own +1/2 faces, per field
    # a cell's R reads its own three +1/2 faces and the +1/2 faces of its
    # i-1, j-1 and k-1 neighbours: compare only cells all six kept their branch
    same = face_same & np.roll(face_same, 1, axis=3) & np.roll(face_same, 1, axis=2)
    same[:, 1:] &= face_same[:, :-1]
    assert same.mean() > 0.3
    err = np.abs(fd - tl)[same]
    assert err.max() <= 1e-6 * np.abs(tl).max()


@pytest.mark.parametrize("phys", [dict(), dict(k0=0.0), dict(vsed=0.0, tau=0.0)])
def test_column_dot_product_and_fd(phys):
    c, _ = _case(nz=16)
    g = oracle.Grid.from_case(c, **phys)
    rng = np.random.default_rng(3)
    Y3 = c.state() * (1 + 0.01 * rng.standard_normal(c.state().shape))
    dY, _, _, _ = _dirs(rng, c)
    lam = rng.standard_normal(Y3.shape)
    tl = oracle.column_tl(g, Y3, dY, c.dt)
    ad = oracle.column_adj(g, Y3, lam, c.dt)
    lhs, rhs = _dot((tl, lam)), _dot((dY, ad))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
    eps = 1e-6
    fp, _ = oracle.column(g, Y3 + eps * dY, c.dt)
    fm, _ = oracle.column(g, Y3 - eps * dY, c.dt)
    fd = (fp - fm) / (2 * eps)
    assert np.abs(fd - tl).max() <= 1e-7 * np.abs(tl).max()


def test_step_dot_product_five_steps():
    c, g = _case()
    rng = np.random.default_rng(4)
    dY, dmu, dmv, dmw = _dirs(rng, c)
    lam = rng.standard_normal(c.state().shape)
    n = 5
    tl = oracle.step_tl(g, c.state(), c.mu, c.mv, c.mw, c.dt, n, dY, dmu, dmv, dmw)
    l0, gmu, gmv, gmw = oracle.step_adj(g, c.state(), c.mu, c.mv, c.mw, c.dt, n, lam)
    lhs = _dot((tl, lam))
    rhs = _dot((dY, l0), (dmu, gmu), (dmv, gmv), (dmw, gmw))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
    assert np.all(gmw[0] == 0) and np.all(gmw[-1] == 0)


def _away_from_kinks(g, c, Y0, dY, dm, eps, n):
    """Tracer-field branches and every flux sign unchanged at x +- eps d (theta
    never feeds back into the tracers or rho, so its branches cannot move J)."""
    b0 = oracle.trajectory_branches(g, Y0, c.mu, c.mv, c.mw, c.dt, n)[:, :, 2:]
    for s in (1, -1):
        Y = Y0 + s * eps * dY
        mu, mv, mw = (c.mu + s * eps * dm[0], c.mv + s * eps * dm[1], c.mw + s * eps * dm[2])
        for M, M0 in ((mu, c.mu), (mv, c.mv), (mw, c.mw)):
            if np.any(np.signbit(M) != np.signbit(M0)):
                return False
        b = oracle.trajectory_branches(g, Y, mu, mv, mw, c.dt, n)[:, :, 2:]
        if not np.array_equal(b, b0):
            return False
    return True


def test_gradient_of_tracer_cost_matches_central_differences():
    """20 seeded directions, eps = 1e-6, relative tolerance 1e-6."""
    c = gen.make_case(10, 8, 6, 2, seed=7, smooth_tracers=True)
    g = oracle.Grid.from_case(c)
    n = 3
    rng = np.random.default_rng(11)
    Y0 = c.state()
    q_t = np.clip(Y0[2:] / Y0[0] + 0.002 * rng.standard_normal(Y0[2:].shape), 0, None)

    def J(Y, mu, mv, mw):
        Yn, _ = oracle.step(g, Y, mu, mv, mw, c.dt, n)
        return oracle.tracer_cost(g, Yn, q_t)[0]

    Yn, _ = oracle.step(g, Y0, c.mu, c.mv, c.mw, c.dt, n)
    _, lam = oracle.tracer_cost(g, Yn, q_t)
    l0, gmu, gmv, gmw = oracle.step_adj(g, Y0, c.mu, c.mv, c.mw, c.dt, n, lam)
    eps = 1e-6
    checked = 0
    draws = 0
    while checked < 20 and draws < 80:
        draws += 1
        dY, dmu, dmv, dmw = _dirs(rng, c)
        dY[:2] = 0.0          # the gradient asked for: initial tracers and the three mass fluxes
        if not _away_from_kinks(g, c, Y0, dY, (dmu, dmv, dmw), eps, n):
            continue
        fd = (J(Y0 + eps * dY, c.mu + eps * dmu, c.mv + eps * dmv, c.mw + eps * dmw) -
              J(Y0 - eps * dY, c.mu - eps * dmu, c.mv - eps * dmv, c.mw - eps * dmw)) / (2 * eps)
        ad = _dot((dY, l0), (dmu, gmu), (dmv, gmv), (dmw, gmw))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
        checked += 1
    assert checked >= 10, f"only {checked} directions away from kinks in {draws} draws"


def test_adjoint_of_linear_scheme_is_exact_transpose():
    """With the unlimited kappa=1/3 scheme and rho = 1 the step is linear in the
    tracers: the adjoint applied to unit vectors reproduces columns of the
    Jacobian computed by the tangent-linear model."""
    c, _ = _case(nx=5, ny=4, nz=4, ntr=1, seed=3)
    g = oracle.Grid.from_case(c, lim=oracle.LIM_LINEAR, tau=0.0, vsed=0.0)
    Y0 = c.state()
    rng = np.random.default_rng(9)
    for _ in range(3):
        a = tuple(int(rng.integers(0, s)) for s in Y0.shape[1:])
        b = tuple(int(rng.integers(0, s)) for s in Y0.shape[1:])
        e_in = np.zeros(Y0.shape)
        e_in[2][a] = 1.0
        e_out = np.zeros(Y0.shape)
        e_out[2][b] = 1.0
        tl = oracle.step_tl(g, Y0, c.mu, c.mv, c.mw, c.dt, 2, e_in)
        l0, *_ = oracle.step_adj(g, Y0, c.mu, c.mv, c.mw, c.dt, 2, e_out)
        assert abs(tl[2][b] - l0[2][a]) <= 1e-14 + 1e-12 * abs(tl[2][b])
