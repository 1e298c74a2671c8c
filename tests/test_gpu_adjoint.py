"""GPU adjoint (asuca_adjoint_step) against the oracle and against the forward map.

* FP64 adjoint vs the oracle's FP64 adjoint, element by element (1e-12
  relative, the FP64 parity bar), with the oracle linearised along its own
  forward pass's limiter branches.  The GPU's forward pass may take another
  branch only at a face whose limiter decision is a rounding tie: the two
  competing limiter terms (or, for the zero branch, d0 or d1 themselves) lie
  within TIE_ULP units in the last place of the field's scale in the oracle's
  own trajectory.  Only at those faces is the GPU's branch substituted; a
  differing branch anywhere else fails the test, and the mismatch fraction is
  printed;
* results independent of the checkpoint interval (bit for bit);
* dot-product test between the oracle's tangent-linear model and the GPU
  adjoint, along the oracle's branches with the same tie substitution;
* central differences of J = 1/2 sum (q - q_target)^2 through the GPU forward
  (eps = 1e-6, 20 seeded directions scaled by field RMS, relative 1e-6), with
  the Koren limiter on a grid where kink-free directions exist (checked with the
  recorded branches), and on the 128x128x58, 4-tracer, 50-step adjoint workload
  with the unlimited kappa=1/3 scheme, which has no limiter kinks;
* torch.autograd.gradcheck through AdjointFn on an 8x8x6 grid in FP64;
* the FP32 adjoint against the FP64 adjoint.
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


def _rel(got, ref):
    return (np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300),
            np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _gpu_branches(asuca, case, nsteps, lim=0, tend=None, prec=0, **gkw):
    """GPU-recorded branch bytes in the oracle's layout [nsteps][3][F][nz][ny][nx]."""
    import torch
    g = asuca.Grid.from_case(case, prec=prec, lim=lim, **gkw)
    st = asuca.State.from_case(case, prec=prec)
    td = None if tend is None else torch.tensor(tend, dtype=g.torch_dtype, device="cuda")
    b = asuca.record_branches(g, st, case.dt, nsteps, tendencies=td).cpu().numpy()
    out = np.zeros((nsteps, 3, case.nfields) + b.shape[3:], dtype=np.uint8)
    out[:, :, 1:] = b
    return out


# A branch differing between the GPU and the oracle is accepted only where the
# limiter's decision is a rounding tie in the oracle's own trajectory: the
# competing terms within TIE_ULP ulp of the field's scale (max |phi| of the
# field at that stage).  The two FP64 trajectories differ by a few ulp per
# operation (different but exact-to-rounding evaluation orders); a stage's
# flux differences, divided by the spacing and scaled by the stage weight,
# carry that to several ulp of a field's scale per step.  Measured on the
# parity cases below: at most 2.6e-4 of the faces differ; with the column
# physics on every differing face lies within 3.6 ulp, and with a tracer
# only advected (no vertical diffusion) one face after one step lies at
# 6.61 ulp.  A wrongly recorded branch at a face that is not a tie has a
# margin of order the field's own differences, many orders above this bar.
TIE_ULP = 16
EPS64 = np.finfo(np.float64).eps


def _oracle_stage_inputs(og, c, nsteps, tend=None):
    """The oracle's stage inputs (Y^n, Y*, Y**) of every step, in its own
    arithmetic: Y^(s) = Y^n + c_s R(Y^(s-1)) in double, then the column pass."""
    Y = c.state().astype(np.float64)
    cs = (c.dt / 3.0, c.dt / 2.0, c.dt)
    out = []
    for _ in range(nsteps):
        st = [Y]
        S = Y
        for q in range(3):
            S = Y + cs[q] * oracle.rhs(og, S, c.mu, c.mv, c.mw, tend=tend)
            if q < 2:
                st.append(S)
        out.append(st)
        Y, _ = oracle.column(og, S, c.dt)
    return out


def _face_margins(Y, mu, mv, mw):
    """Per direction (i, j, k), the limiter arguments' distances from the branch
    boundaries at every face i+1/2, j+1/2, k+1/2 of fields 1..F-1:
    (zero-branch margin min(|d0|, |d1|), |t1 - t2|, |t2 - t3|, |t1 - t3|) with
    t1 = 2|d1|, t2 = (|d0| + 2|d1|)/3, t3 = 2|d0| and the upwind side by sign(M)."""
    phi = Y[1:] / Y[0]
    nz = phi.shape[1]
    out = []
    for d in range(3):
        if d < 2:
            ax = 3 - d
            pm1, p1, p2 = (np.roll(phi, s, axis=ax) for s in (1, -1, -2))
            m = (mu if d == 0 else mv)[None]
        else:
            up = lambda s: phi[:, np.clip(np.arange(nz) + s, 0, nz - 1)]
            pm1, p1, p2 = up(-1), up(1), up(2)
            m = np.concatenate([mw[1:nz], np.zeros_like(mw[:1])])[None]
        pos = m >= 0
        d0 = np.where(pos, phi - pm1, p1 - p2)
        d1 = np.where(pos, p1 - phi, phi - p1)
        a0, a1 = np.abs(d0), np.abs(d1)
        t1, t2, t3 = 2 * a1, (a0 + 2 * a1) / 3, 2 * a0
        out.append((np.minimum(a0, a1), np.abs(t1 - t2), np.abs(t2 - t3), np.abs(t1 - t3)))
    return out


def _tie_substituted_branches(og, c, nsteps, gpu_br, own_br, tend=None):
    """own_br with the GPU's branch at tie faces; asserts that every face where
    the two differ is a tie.  Returns (branches, mismatch fraction, worst margin
    of a mismatch in ulp of the field's scale)."""
    states = _oracle_stage_inputs(og, c, nsteps, tend)
    out = own_br.copy()
    nmis, worst = 0, 0.0
    for s in range(nsteps):
        for q in range(3):
            Y = states[s][q]
            scale = np.abs(Y[1:] / Y[0]).reshape(Y.shape[0] - 1, -1).max(axis=1)[:, None, None, None]
            margins = _face_margins(Y, c.mu, c.mv, c.mw)
            bg, bo = gpu_br[s, q, 1:], own_br[s, q, 1:]
            for d in range(3):
                xg, xo = (bg >> (2 * d)) & 3, (bo >> (2 * d)) & 3
                mis = xg != xo
                if not mis.any():
                    continue
                zero, m12, m23, m13 = margins[d]
                lo, hi = np.minimum(xg, xo), np.maximum(xg, xo)
                marg = np.where(lo == 0, zero, np.where((lo == 1) & (hi == 2), m12,
                                                        np.where((lo == 2) & (hi == 3), m23, m13)))
                ulp = marg / (EPS64 * scale)
                bad = mis & (ulp > TIE_ULP)
                assert not bad.any(), (
                    f"step {s} stage {q} dir {d}: {int(bad.sum())} faces differ outside a rounding tie "
                    f"(worst {float(ulp[bad].max()):.3g} ulp of the field's scale)")
                worst = max(worst, float(ulp[mis].max()))
                nmis += int(mis.sum())
                sub = out[s, q, 1:]
                sub[mis] = (sub[mis] & ~np.uint8(3 << (2 * d))) | (xg[mis] << (2 * d)).astype(np.uint8)
    frac = nmis / float(3 * own_br[:, :, 1:].size)
    return out, frac, worst


def _gpu_adjoint(asuca, case, lam, nsteps, K, prec=0, lim=0, tend=None, tile_rows=None, **gkw):
    import torch
    g = asuca.Grid.from_case(case, prec=prec, lim=lim, **gkw)
    if tile_rows is not None:
        asuca.set_tuning(g, asuca.TUNE_STAGE_TILE_ROWS, tile_rows)
    st = asuca.State.from_case(case, prec=prec)
    dt_ = g.torch_dtype
    td = None if tend is None else torch.tensor(tend, dtype=dt_, device="cuda")
    l = torch.tensor(lam, dtype=dt_, device="cuda")
    g0, gmu, gmv, gmw = asuca.adjoint_step(g, st, case.dt, nsteps, l, checkpoint_every=K, tendencies=td)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    f = lambda t: t.double().cpu().numpy()
    return f(g0), f(gmu), f(gmv), f(gmw)


@pytest.mark.parametrize("lim", [0, 1, 2])
@pytest.mark.parametrize("shape,ntr,nsteps,dy", [((20, 16, 10), 3, 5, 2000.0), ((37, 13, 7), 2, 4, 2000.0),
                                                 ((32, 32, 16), 3, 3, 2000.0), ((26, 22, 9), 2, 3, 1600.0)])
def test_adjoint_fp64_matches_oracle(asuca, lim, shape, ntr, nsteps, dy):
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, ntr, seed=100 + nx, dy=dy)
    rng = np.random.default_rng(nx)
    lam = rng.standard_normal(c.state().shape)
    tend = rng.uniform(-1e-6, 1e-6, (1 + ntr, nz, ny, nx)) if nx == 37 else None
    og = oracle.Grid.from_case(c, lim=lim)
    br = _gpu_branches(asuca, c, nsteps, lim=lim, tend=tend)
    own = oracle.trajectory_branches(og, c.state(), c.mu, c.mv, c.mw, c.dt, nsteps, tend=tend)
    traj, frac, worst = _tie_substituted_branches(og, c, nsteps, br, own, tend=tend)
    print(f"lim {lim} {shape}: branch mismatch fraction {frac:.3e} (all rounding ties, "
          f"worst {worst:.3g} ulp of the field's scale)")
    ref = oracle.step_adj(og, c.state(), c.mu, c.mv, c.mw, c.dt, nsteps, lam, tend=tend, traj_br=traj)
    got = _gpu_adjoint(asuca, c, lam, nsteps, nsteps, lim=lim, tend=tend)
    for name, a, b in zip(("lam0", "gmu", "gmv", "gmw"), got, ref):
        l2, mx = _rel(a, b)
        print(f"  {name}: rel L2 {l2:.3e}, rel max {mx:.3e}")
        assert l2 <= 1e-12 and mx <= 1e-12, (name, l2, mx)


@pytest.mark.parametrize("sed", [0, -1])
def test_adjoint_fp64_with_another_sedimenting_tracer(asuca, sed):
    """The first tracer sedimenting, or none (every other case sediments the
    last one): the FP64 adjoint against the oracle's at 1e-12."""
    c = gen.make_case(24, 18, 9, 3, seed=131)
    nsteps = 3
    lam = np.random.default_rng(17).standard_normal(c.state().shape)
    og = oracle.Grid.from_case(c, sed=sed)
    br = _gpu_branches(asuca, c, nsteps, sed_tracer=sed)
    own = oracle.trajectory_branches(og, c.state(), c.mu, c.mv, c.mw, c.dt, nsteps)
    traj, _, _ = _tie_substituted_branches(og, c, nsteps, br, own)
    ref = oracle.step_adj(og, c.state(), c.mu, c.mv, c.mw, c.dt, nsteps, lam, traj_br=traj)
    got = _gpu_adjoint(asuca, c, lam, nsteps, 2, sed_tracer=sed)
    for name, a, b in zip(("lam0", "gmu", "gmv", "gmw"), got, ref):
        l2, mx = _rel(a, b)
        assert l2 <= 1e-12 and mx <= 1e-12, (name, l2, mx)


@pytest.mark.parametrize("gkw,okw", [(dict(k0=0.0), dict(k0=0.0)),
                                     (dict(tau_theta=0.0, v_sed=0.0), dict(tau=0.0, vsed=0.0)),
                                     (dict(tau_theta=0.0, k0=0.0, v_sed=0.0), dict(tau=0.0, k0=0.0, vsed=0.0))])
def test_adjoint_fp64_with_column_physics_switched_off(asuca, gkw, okw):
    """No vertical diffusion, no relaxation and sedimentation, or no column
    physics at all (every other case runs all three): the FP64 adjoint against
    the oracle's at 1e-12."""
    c = gen.make_case(22, 17, 9, 2, seed=141)
    nsteps = 3
    lam = np.random.default_rng(19).standard_normal(c.state().shape)
    og = oracle.Grid.from_case(c, **okw)
    br = _gpu_branches(asuca, c, nsteps, **gkw)
    own = oracle.trajectory_branches(og, c.state(), c.mu, c.mv, c.mw, c.dt, nsteps)
    traj, _, _ = _tie_substituted_branches(og, c, nsteps, br, own)
    ref = oracle.step_adj(og, c.state(), c.mu, c.mv, c.mw, c.dt, nsteps, lam, traj_br=traj)
    got = _gpu_adjoint(asuca, c, lam, nsteps, 2, **gkw)
    for name, a, b in zip(("lam0", "gmu", "gmv", "gmw"), got, ref):
        l2, mx = _rel(a, b)
        assert l2 <= 1e-12 and mx <= 1e-12, (name, l2, mx)


def test_adjoint_independent_of_checkpoint_interval(asuca):
    c = gen.make_case(24, 20, 12, 2, seed=3)
    lam = np.random.default_rng(1).standard_normal(c.state().shape)
    a = _gpu_adjoint(asuca, c, lam, 7, 1)
    for K in (3, 10):
        b = _gpu_adjoint(asuca, c, lam, 7, K)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_adjoint_independent_of_recording_tile_rows(asuca):
    """The recomputation records branches with the grid's tile height; 4- and
    8-row tiles give the same trajectory, hence the same gradients bit for bit."""
    c = gen.make_case(70, 21, 9, 3, seed=12)
    lam = np.random.default_rng(2).standard_normal(c.state().shape)
    a = _gpu_adjoint(asuca, c, lam, 4, 2, prec=1, tile_rows=8)
    b = _gpu_adjoint(asuca, c, lam, 4, 2, prec=1, tile_rows=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nsteps,K", [(7, 3), (6, 3), (1, 10), (0, 4)])
def test_checkpointed_forward_and_adjoint_from_checkpoints(asuca, prec, nsteps, K):
    """asuca_forward_checkpointed advances the state bit for bit as asuca_step
    (budgets included), and asuca_adjoint_from_checkpoints on its checkpoints
    returns asuca_adjoint_step's gradients bit for bit."""
    import torch
    c = gen.make_case(40, 24, 10, 3, seed=11)
    g = asuca.Grid.from_case(c, prec=prec)
    st_a = asuca.State.from_case(c, prec=prec)
    st_b = st_a.clone()
    st_0 = st_a.clone()
    ba = asuca.step(g, st_a, c.dt, nsteps, budgets=True)
    bb = torch.empty_like(ba)
    ck = asuca.forward_checkpointed(g, st_b, c.dt, nsteps, checkpoint_every=K, budgets=bb)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    for x, y in zip(st_a.fields(), st_b.fields()):
        assert torch.equal(x, y)
    assert torch.equal(ba, bb)
    lam = torch.tensor(np.random.default_rng(2).standard_normal(c.state().shape), dtype=g.torch_dtype,
                       device="cuda")
    ref = asuca.adjoint_step(g, st_0, c.dt, nsteps, lam, checkpoint_every=K)
    got = asuca.adjoint_from_checkpoints(g, ck, st_0, c.dt, nsteps, lam, checkpoint_every=K)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    for x, y in zip(ref, got):
        assert torch.equal(x, y)


def test_dot_product_oracle_tangent_linear_vs_gpu_adjoint(asuca):
    c = gen.make_case(20, 16, 10, 3, seed=21)
    og = oracle.Grid.from_case(c)
    rng = np.random.default_rng(5)
    Y = c.state()
    dY = rng.standard_normal(Y.shape) * np.sqrt(np.mean(Y ** 2, axis=(1, 2, 3)))[:, None, None, None]
    dmu = rng.standard_normal(c.mu.shape) * 20
    dmv = rng.standard_normal(c.mv.shape) * 20
    dmw = rng.standard_normal(c.mw.shape) * 0.1
    dmw[0] = dmw[-1] = 0
    lam = rng.standard_normal(Y.shape)
    n = 4
    br = _gpu_branches(asuca, c, n)
    own = oracle.trajectory_branches(og, Y, c.mu, c.mv, c.mw, c.dt, n)
    traj, _, _ = _tie_substituted_branches(og, c, n, br, own)
    tl = oracle.step_tl(og, Y, c.mu, c.mv, c.mw, c.dt, n, dY, dmu, dmv, dmw, traj_br=traj)
    g0, gmu, gmv, gmw = _gpu_adjoint(asuca, c, lam, n, n)
    lhs = float(np.sum(tl * lam))
    rhs = float(np.sum(dY * g0) + np.sum(dmu * gmu) + np.sum(dmv * gmv) + np.sum(dmw * gmw))
    print(f"dot product: lhs {lhs:.17g}, rhs {rhs:.17g}, rel {abs(lhs - rhs) / max(abs(lhs), abs(rhs)):.3e}")
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def _fd_check(asuca, case, nsteps, lim, K, ndir=20, check_kinks=True, max_draws=60):
    import torch
    g = asuca.Grid.from_case(case, prec=asuca.FP64, lim=lim)
    st0 = asuca.State.from_case(case, prec=asuca.FP64)
    rng = np.random.default_rng(2024)
    q_t = torch.tensor(np.clip(case.rhoq / case.rho + 0.002 * rng.standard_normal(case.rhoq.shape), 0, None),
                       device="cuda")

    def run(dq, dmu, dmv, dmw, eps):
        st = asuca.State(st0.rho.clone(), st0.rhotheta.clone(), (st0.rhoq + eps * dq).contiguous(),
                         (st0.mu + eps * dmu).contiguous(), (st0.mv + eps * dmv).contiguous(),
                         (st0.mw + eps * dmw).contiguous())
        return st

    def J(st):
        s2 = st.clone()
        asuca.step(g, s2, case.dt, nsteps)
        r = s2.rhoq / s2.rho - q_t
        return 0.5 * float(torch.sum(r * r)), s2

    J0, sN = J(st0)
    r = sN.rhoq / sN.rho - q_t
    lam = torch.zeros((g.nfields,) + tuple(st0.rho.shape), dtype=torch.float64, device="cuda")
    lam[2:] = r / sN.rho
    lam[0] = -torch.sum(r * sN.rhoq / sN.rho, 0) / sN.rho
    g0, gmu, gmv, gmw = asuca.adjoint_step(g, st0, case.dt, nsteps, lam.contiguous(), checkpoint_every=K)
    b0 = asuca.record_branches(g, st0, case.dt, nsteps)[:, :, 1:] if check_kinks else None
    rms = lambda t: float(torch.sqrt(torch.mean(t * t)))
    eps = 1e-6
    ok = draws = 0
    while ok < ndir and draws < max_draws:
        draws += 1
        dq = torch.randn(st0.rhoq.shape, generator=None, dtype=torch.float64, device="cuda") * rms(st0.rhoq)
        dmu = torch.randn(st0.mu.shape, dtype=torch.float64, device="cuda") * rms(st0.mu)
        dmv = torch.randn(st0.mv.shape, dtype=torch.float64, device="cuda") * rms(st0.mv)
        dmw = torch.randn(st0.mw.shape, dtype=torch.float64, device="cuda") * rms(st0.mw)
        dmw[0] = 0
        dmw[-1] = 0
        sp, sm = run(dq, dmu, dmv, dmw, eps), run(dq, dmu, dmv, dmw, -eps)
        kinked = False
        for M in ("mu", "mv", "mw"):
            if bool((torch.signbit(getattr(sp, M)) != torch.signbit(getattr(st0, M))).any()) or \
                    bool((torch.signbit(getattr(sm, M)) != torch.signbit(getattr(st0, M))).any()):
                kinked = True
        if check_kinks and not kinked:
            for s_ in (sp, sm):
                if not torch.equal(asuca.record_branches(g, s_, case.dt, nsteps)[:, :, 1:], b0):
                    kinked = True
                    break
        if kinked:
            continue
        fd = (J(sp)[0] - J(sm)[0]) / (2 * eps)
        ad = float(torch.sum(dq * g0[2:]) + torch.sum(dmu * gmu) + torch.sum(dmv * gmv) + torch.sum(dmw * gmw))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
        ok += 1
    return ok, draws


def test_fd_gradient_koren_kink_free_directions(asuca):
    import torch
    torch.manual_seed(7)
    # white-noise directions meet a limiter kink somewhere once the grid and the
    # step count grow (about one near-kink face per 5e4 face evaluations here),
    # so the Koren check runs on a grid where most directions stay kink-free
    c = gen.make_case(12, 10, 8, 2, seed=8, smooth_tracers=True)
    ok, draws = _fd_check(asuca, c, 3, asuca.LIM_KOREN, 2, max_draws=100)
    assert ok >= 10, f"{ok} kink-free directions in {draws}"


def test_fd_gradient_adjoint_workload_128x128x58_50_steps_linear(asuca):
    import torch
    torch.manual_seed(11)
    c = gen.make_config_case("adjoint_128x128x58")
    # about 70% of white-noise directions flip the sign of some of the 2.8M
    # face mass fluxes (a kink of the upwind choice); those are redrawn
    ok, draws = _fd_check(asuca, c, 50, asuca.LIM_LINEAR, 10, check_kinks=False, max_draws=150)
    assert ok == 20, f"{ok} of 20 directions usable in {draws}"


def test_gradcheck_through_autograd_function(asuca):
    import torch
    c = gen.make_case(8, 8, 6, 2, seed=31, smooth_tracers=True)
    g = asuca.Grid.from_case(c, prec=asuca.FP64, lim=asuca.LIM_LINEAR)
    st = asuca.State.from_case(c, prec=asuca.FP64)
    q0 = st.rhoq.clone().requires_grad_(True)
    mu = st.mu.clone().requires_grad_(True)
    Fn = asuca.AdjointFn

    def f(q, m):
        _, _, qn = Fn.apply(st.rho, st.rhotheta, q, m, st.mv, st.mw, g, c.dt, 2, 1)
        return qn

    assert torch.autograd.gradcheck(f, (q0, mu), eps=1e-6, atol=1e-9, rtol=1e-6)


@pytest.mark.parametrize("gkw,okw", [(dict(), dict()), (dict(k0=0.0), dict(k0=0.0)),
                                     (dict(tau_theta=0.0, k0=0.0, v_sed=0.0), dict(tau=0.0, k0=0.0, vsed=0.0))])
def test_fp32_adjoint_against_oracle_along_its_branches(asuca, gkw, okw):
    """The FP32 adjoint linearises the FP32 forward pass, whose branches differ
    from the FP64 pass at faces whose limiter arguments are rounding noise; it is
    compared with the FP64 oracle adjoint taken along the FP32 pass's branches
    (with the column physics on, without vertical diffusion, and with none)."""
    c = gen.make_case(32, 24, 16, 3, seed=41)
    lam = np.random.default_rng(2).standard_normal(c.state().shape)
    n = 5
    br = _gpu_branches(asuca, c, n, prec=1, **gkw)
    og = oracle.Grid.from_case(c, **okw)
    ref = oracle.step_adj(og, c.state(), c.mu, c.mv, c.mw, c.dt, n, lam, traj_br=br)
    a32 = _gpu_adjoint(asuca, c, lam, n, n, prec=1, **gkw)
    for name, x, y in zip(("lam0", "gmu", "gmv", "gmw"), a32, ref):
        l2, _ = _rel(x, y)
        assert l2 <= 1e-4, (name, l2)
