"""GPU parity of the HEVI acoustic short steps (asuca_acoustic_steps, Sec. 1.1)
against the FP64 oracle, which solves each column's implicit W-s system in its
interleaved form (the CUDA path eliminates s and uses a factorisation computed
once per stage on the host).

Bars: FP64 within 1e-12 relative (per-field L2 and max); FP32 within 2e-5
relative L2 per field; the lids of W never touched."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
A = gen.ACOUSTIC


@pytest.fixture(scope="module")
def asuca():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    return a


def _run(asuca, case, prec, nshort, beta=A["beta"], dtau=A["dtau"], lids=(7.0, -5.0)):
    import torch
    npdt = np.float64 if prec == asuca.FP64 else np.float32
    U, V, W, S, r0c, r0f = gen.make_acoustic_state(case, dtype=npdt)
    W = W.copy()
    W[0], W[-1] = lids                     # sentinels: the lids are never read or written
    g = asuca.Grid.from_case(case, prec=prec)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to("cuda") for a in (U, V, W, S)]
    asuca.acoustic_steps(g, *dev, r0c, r0f, A["cs2"], beta, dtau, nshort)
    got = [t.double().cpu().numpy() for t in dev]
    want = oracle.acoustic(U, V, W, S, case.dz, r0c, r0f, A["cs2"], beta, dtau, nshort, dx=case.dx, dy=case.dy)
    assert asuca.get_status(g) == asuca.OK
    return got, want, lids


def _check(asuca, prec, got, want, lids):
    tol = TOL64 if prec == asuca.FP64 else TOL32
    assert np.all(got[2][0] == lids[0]) and np.all(got[2][-1] == lids[1])
    for name, g, w in zip("UVWS", got, want):
        if name == "W":
            g, w = g[1:-1], w[1:-1]
        if not np.any(w):
            assert not np.any(g)
            continue
        l2 = np.linalg.norm(g - w) / np.linalg.norm(w)
        assert l2 <= tol, f"{name}: rel L2 {l2:.3e}"
        if prec == asuca.FP64:
            assert np.abs(g - w).max() <= tol * np.abs(w).max(), name


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,nshort", [((37, 13, 7), 3), ((4, 4, 3), 2), ((70, 9, 5), 4), ((32, 32, 16), 6),
                                          ((40, 24, 128), 2)])
def test_acoustic_matches_oracle(asuca, prec, shape, nshort):
    nx, ny, nz = shape
    c = gen.make_case(nx, ny, nz, 1, seed=900 + nx)
    got, want, lids = _run(asuca, c, prec, nshort)
    _check(asuca, prec, got, want, lids)


@pytest.mark.parametrize("prec", [0, 1])
def test_acoustic_with_different_spacings_in_i_and_j(asuca, prec):
    """dx = 2000 m, dy = 1600 m: the gradients and the divergence each take
    their own direction's spacing."""
    c = gen.make_case(37, 26, 9, 1, seed=901, dy=1600.0)
    got, want, lids = _run(asuca, c, prec, 3)
    _check(asuca, prec, got, want, lids)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("beta,dtau", [(0.5, 2.0), (1.0, 2.0), (0.6, 0.0), (0.55, 5.5)])
def test_acoustic_weights_and_step_lengths(asuca, prec, beta, dtau):
    c = gen.make_case(29, 17, 9, 1, seed=71)
    got, want, lids = _run(asuca, c, prec, 3, beta=beta, dtau=dtau)
    _check(asuca, prec, got, want, lids)


def test_acoustic_zero_steps_and_bad_arguments(asuca):
    import torch
    c = gen.make_case(16, 12, 5, 1, seed=4)
    g = asuca.Grid.from_case(c)
    U, V, W, S, r0c, r0f = gen.make_acoustic_state(c, dtype=np.float32)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to("cuda") for a in (U, V, W, S)]
    before = [t.clone() for t in dev]
    asuca.acoustic_steps(g, *dev, r0c, r0f, A["cs2"], 0.6, 2.0, 0)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(dev, before))
    bad_r0c = r0c.copy()
    bad_r0c[2] = 0.0
    for kw in (dict(beta=0.4), dict(beta=1.5), dict(cs2=0.0), dict(dtau=-1.0), dict(nshort=-1),
               dict(rho0c=bad_r0c), dict(dtau=float("nan"))):
        args = dict(rho0c=r0c, rho0f=r0f, cs2=A["cs2"], beta=0.6, dtau=2.0, nshort=1)
        args.update(kw)
        with pytest.raises(asuca.AsucaError) as e:
            asuca.acoustic_steps(g, *dev, **args)
        assert e.value.status == asuca.ERR_ARG
    need = asuca.acoustic_workspace_bytes(g)
    big = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    for ws in (big[:need - 256], big[8:8 + need]):
        with pytest.raises(asuca.AsucaError) as e:
            asuca.acoustic_steps(g, *dev, r0c, r0f, A["cs2"], 0.6, 2.0, 1, workspace=ws)
        assert e.value.status == asuca.ERR_WORKSPACE
    dp = ctypes.POINTER(ctypes.c_double)
    d = asuca.AcousticDesc(r0c.ctypes.data_as(dp), None, A["cs2"], 0.6)
    p = [ctypes.c_void_p(t.data_ptr()) for t in dev]
    assert asuca.lib().asuca_acoustic_steps(g.handle, *p, ctypes.byref(d), 2.0, 1, ctypes.c_void_p(big.data_ptr()),
                                            need, None) == asuca.ERR_ARG


def test_acoustic_full_size_fp32(asuca):
    """1024x1024x58, FP32, the short steps the benchmark times: every value
    against the oracle."""
    c = gen.make_config_case("large_1024x1024x58", ntracers=1)
    got, want, lids = _run(asuca, c, asuca.FP32_MIXED, 2)
    _check(asuca, asuca.FP32_MIXED, got, want, lids)
