"""Acoustic short steps nested in the RK3 long step on the GPU (asuca_step_hevi).

* Against the oracle's coupled step (orc_step_hevi): the scalar fields, the
  momenta U, V, W and the final acoustic density perturbation, FP64 within
  1e-12 (relative L2 and max, every component), FP32 within 2e-5 (relative
  L2 per scalar field; the momentum as one vector field (U, V, W)); ragged
  sizes, two limiters, forcing, several short-step counts and implicit
  weights.
* Mass consistency on the GPU: the advected density equals rho0 (1 + s) of
  the acoustic integration (FP64 1e-13, FP32 1e-6).
* Bad arguments are rejected.
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
    return torch.as_tensor(np.array(a, copy=True)).to(device="cuda", dtype=dt).contiguous()


def _run(asuca, case, prec, lim, ns, beta, nsteps, tend=None):
    import torch
    Y, U, V, W, r0c, r0f, dt, _ = gen.make_hevi_state(case)
    cs2 = gen.ACOUSTIC["cs2"]
    g = asuca.Grid.from_case(case, prec=prec, lim=lim)
    dt_ = g.torch_dtype
    st = asuca.State(_tensor(Y[0], dt_), _tensor(Y[1], dt_), _tensor(Y[2:], dt_), _tensor(U, dt_), _tensor(V, dt_),
                     _tensor(W, dt_))
    sfin = torch.zeros((case.nz, case.ny, case.nx), dtype=dt_, device="cuda")
    td = None if tend is None else _tensor(tend, dt_)
    bud = asuca.step_hevi(g, st, dt, nsteps, r0c, r0f, cs2, beta, ns, tendencies=td, s_final=sfin, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    cast = lambda a: _tensor(a, dt_).double().cpu().numpy()
    og = oracle.Grid.from_case(case, lim=lim)
    ref = oracle.step_hevi(og, cast(Y), cast(U), cast(V), cast(W), r0c, r0f, cs2, beta, ns, dt, nsteps,
                           tend=None if tend is None else cast(tend))
    got = (st.fields().double().cpu().numpy(), st.mu.double().cpu().numpy(), st.mv.double().cpu().numpy(),
           st.mw.double().cpu().numpy(), sfin.double().cpu().numpy(), bud.cpu().numpy())
    return got, ref, r0c


def _rel(a, b):
    return (np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300),
            np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("shape,ntr,lim,ns,beta,nsteps,forced,dy", [
    ((20, 16, 10), 2, 0, 6, 0.6, 2, False, 2000.0),
    ((37, 13, 7), 2, 0, 6, 0.6, 2, True, 2000.0),
    ((32, 32, 16), 3, 1, 4, 0.5, 1, False, 2000.0),
    ((45, 19, 12), 1, 0, 9, 1.0, 2, False, 2000.0),
    ((64, 48, 58), 4, 0, 6, 0.6, 1, False, 2000.0),
    ((30, 22, 9), 2, 0, 6, 0.6, 2, False, 1600.0),     # dx != dy
])
def test_hevi_step_against_oracle(asuca, prec, tol, shape, ntr, lim, ns, beta, nsteps, forced, dy):
    nx, ny, nz = shape
    case = gen.make_case(nx, ny, nz, ntr, seed=700 + nx, dy=dy)
    tend = np.random.default_rng(4).uniform(-1e-6, 1e-6, (1 + ntr, nz, ny, nx)) if forced else None
    got, ref, _ = _run(asuca, case, prec, lim, ns, beta, nsteps, tend)
    Yg, Ug, Vg, Wg, Sg, Bg = got
    Yr, Ur, Vr, Wr, Sr, Br = ref
    for f in range(Yr.shape[0]):
        l2, mx = _rel(Yg[f], Yr[f])
        assert l2 <= tol and (prec == 1 or mx <= tol), ("field", f, l2, mx)
    if prec == 0:
        for name, a, b in (("U", Ug, Ur), ("V", Vg, Vr), ("W", Wg[1:-1], Wr[1:-1])):
            l2, mx = _rel(a, b)
            assert l2 <= tol and mx <= tol, (name, l2, mx)
    else:
        # FP32: the momentum is one vector field; W is two orders of magnitude
        # smaller than U and V and is the difference of large implicit-solve
        # terms, so its own-norm error is not a measure of the field's error
        l2, _ = _rel(np.concatenate([Ug.ravel(), Vg.ravel(), Wg.ravel()]),
                     np.concatenate([Ur.ravel(), Vr.ravel(), Wr.ravel()]))
        assert l2 <= tol, ("momentum", l2)
    # s is a small perturbation (|s| ~ 1e-3): compare it on the scale of 1 + s, the density it stands for
    assert np.abs(Sg - Sr).max() <= tol * 1.0, np.abs(Sg - Sr).max()
    assert np.all(np.abs(Bg - Br) <= (1e-12 if prec == 0 else 1e-5) * np.abs(Br) + 1e-300)


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6)])
def test_advected_density_equals_acoustic_density(asuca, prec, tol):
    case = gen.make_case(40, 24, 12, 2, seed=77)
    got, _, r0c = _run(asuca, case, prec, 0, 6, 0.6, 2)
    Y, S = got[0], got[4]
    rho_ac = r0c[:, None, None] * (1.0 + S)
    assert np.abs(Y[0] - rho_ac).max() <= tol * np.abs(Y[0]).max()


def test_hevi_rejects_bad_arguments(asuca):
    import torch
    case = gen.make_case(16, 12, 6, 1, seed=5)
    Y, U, V, W, r0c, r0f, dt, ns = gen.make_hevi_state(case)
    g = asuca.Grid.from_case(case, prec=1)
    d = g.torch_dtype
    st = asuca.State(_tensor(Y[0], d), _tensor(Y[1], d), _tensor(Y[2:], d), _tensor(U, d), _tensor(V, d),
                     _tensor(W, d))
    cs2 = gen.ACOUSTIC["cs2"]
    for kw in (dict(nshort=0), dict(beta=0.4), dict(beta=1.2), dict(cs2=0.0), dict(cs2=-1.0)):
        a = dict(cs2=cs2, beta=0.6, nshort=ns)
        a.update(kw)
        with pytest.raises(asuca.AsucaError):
            asuca.step_hevi(g, st, dt, 1, r0c, r0f, a["cs2"], a["beta"], a["nshort"])
    with pytest.raises(asuca.AsucaError):
        asuca.step_hevi(g, st, dt, 1, -r0c, r0f, cs2, 0.6, ns)
    small = torch.empty(asuca.hevi_workspace_bytes(g) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(asuca.AsucaError):
        asuca.step_hevi(g, st, dt, 1, r0c, r0f, cs2, 0.6, ns, workspace=small)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
