"""Pins of the oracle's long step with nested acoustic short steps
(orc_step_hevi), CPU only.

* With the acoustic terms off (c^2 = 0: no pressure gradient), one short step
  per stage and beta = 1/2, the momenta never change and the mean effective
  mass fluxes are the momenta themselves exactly: the step equals the plain
  step (orc_step) with M = (U, V, W) bit for bit.
* Mass consistency: the advected density after a step equals rho0 (1 + s) of
  the acoustic integration (1e-13), which holds only if every stage advects
  with exactly the fluxes the acoustic density equation applies, weighted and
  summed over the right short steps.
* The same holds for the density of the first two RK stages, each against
  an acoustic integration over its own weight times dt (1e-13).
* The new momenta are the third stage's integration: orc_acoustic over n_3
  short steps of dt / n_3 from (U, V, W)^n and s^n = rho^n / rho0 - 1, bit
  for bit.
* The short-step counts per stage are round(ns / 3), round(ns / 2), ns, each
  the integer nearest to c_q ns (halves up), at least one, for ns = 1 .. 24.
"""
import numpy as np
import pytest

import gen
import oracle


def _setup(nx=20, ny=16, nz=10, ntr=2, seed=3):
    c = gen.make_case(nx, ny, nz, ntr, seed=seed)
    Y, U, V, W, r0c, r0f, dt, ns = gen.make_hevi_state(c)
    return c, Y, U, V, W, r0c, r0f, dt, ns


def test_short_step_counts():
    assert [oracle.hevi_short_steps(6, q) for q in range(3)] == [2, 3, 6]
    assert [oracle.hevi_short_steps(1, q) for q in range(3)] == [1, 1, 1]
    assert [oracle.hevi_short_steps(12, q) for q in range(3)] == [4, 6, 12]
    # every count is the integer nearest to c_q ns (halves go up), at least one
    for ns in range(1, 25):
        for q, cq in enumerate((1 / 3, 1 / 2, 1.0)):
            n = oracle.hevi_short_steps(ns, q)
            x = cq * ns
            assert n >= 1
            if x >= 0.5:
                assert abs(n - x) < 0.5 + 1e-12 and not (abs(n - x + 0.5) < 1e-12), (ns, q, n)


@pytest.mark.parametrize("lim", [0, 1])
def test_acoustic_off_reduces_to_the_plain_step(lim):
    c, Y, U, V, W, r0c, r0f, dt, _ = _setup()
    g = oracle.Grid.from_case(c, lim=lim)
    got, U1, V1, W1, _, bud = oracle.step_hevi(g, Y, U, V, W, r0c, r0f, 0.0, 0.5, 1, dt, 2)
    ref, rbud = oracle.step(g, Y, U, V, W, dt, 2)
    assert np.array_equal(got, ref)
    assert np.array_equal(bud, rbud)
    for a, b in ((U1, U), (V1, V), (W1, W)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("nsteps,ns,beta", [(1, 6, 0.6), (2, 6, 0.6), (1, 4, 0.5), (1, 12, 1.0)])
def test_advected_density_equals_acoustic_density(nsteps, ns, beta):
    c, Y, U, V, W, r0c, r0f, dt, _ = _setup()
    g = oracle.Grid.from_case(c)
    cs2 = gen.ACOUSTIC["cs2"]
    out, _, _, _, s_fin, _ = oracle.step_hevi(g, Y, U, V, W, r0c, r0f, cs2, beta, ns, dt, nsteps)
    rho_ac = r0c[:, None, None] * (1.0 + s_fin)
    assert np.abs(out[0] - rho_ac).max() <= 1e-13 * np.abs(out[0]).max()
    # and the density did move: the acoustic fluxes are not divergence free
    assert np.abs(out[0] - Y[0]).max() > 1e-9 * np.abs(Y[0]).max()


@pytest.mark.parametrize("ns,beta", [(6, 0.6), (7, 0.5), (11, 1.0)])
def test_every_stage_density_equals_its_acoustic_density(ns, beta):
    """The same consistency inside the step: the density of RK stage q (q = 1,
    2) equals rho0 (1 + s) after an acoustic integration over the stage's
    weight times dt (1/3 dt, 1/2 dt) in its own short steps, from the
    momenta and s at t^n (1e-13).  A stage integrated over the wrong length
    or from the wrong start fails this."""
    c, Y, U, V, W, r0c, r0f, dt, _ = _setup()
    g = oracle.Grid.from_case(c)
    cs2 = gen.ACOUSTIC["cs2"]
    *_, srho = oracle.step_hevi(g, Y, U, V, W, r0c, r0f, cs2, beta, ns, dt, 1, stage_rho=True)
    S0 = Y[0] / r0c[:, None, None] - 1.0
    for q, cq in ((0, 1.0 / 3.0), (1, 0.5)):
        nq = oracle.hevi_short_steps(ns, q)
        Sq = oracle.acoustic(U, V, W, S0, c.dz, r0c, r0f, cs2, beta, cq * dt / nq, nq)[3]
        rho_ac = r0c[:, None, None] * (1.0 + Sq)
        assert np.abs(srho[q] - rho_ac).max() <= 1e-13 * np.abs(rho_ac).max(), q
        assert np.abs(srho[q] - Y[0]).max() > 1e-9 * np.abs(Y[0]).max()


def test_new_momenta_are_the_third_stage_integration():
    c, Y, U, V, W, r0c, r0f, dt, ns = _setup()
    g = oracle.Grid.from_case(c)
    A = gen.ACOUSTIC
    _, U1, V1, W1, s_fin, _ = oracle.step_hevi(g, Y, U, V, W, r0c, r0f, A["cs2"], A["beta"], ns, dt, 1)
    n3 = oracle.hevi_short_steps(ns, 2)
    S0 = Y[0] / r0c[:, None, None] - 1.0
    Ua, Va, Wa, Sa = oracle.acoustic(U, V, W, S0, c.dz, r0c, r0f, A["cs2"], A["beta"], dt / n3, n3)
    for a, b in ((U1, Ua), (V1, Va), (W1, Wa), (s_fin, Sa)):
        assert np.array_equal(a, b)
