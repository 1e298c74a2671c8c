"""The bounds-check build of the library (compiled with ASUCA_BOUNDS_CHECK,
libasuca_bc.so): the step's kernels test each global-memory index, and each
offset into the stage's shared-memory ring, against its buffer's extent and
record ASUCA_ERR_BOUNDS instead of accessing outside the buffer.

Small cases of every checked path run with that build in a child process (the
library is chosen per process through ASUCA_LIBRARY): the periodic step in
both precisions with the column pass split over stages 2 and 3, with the whole
top-down half in stage 3 (the nested acoustic step's arrangement, reached
through the limited-area step) and as separate launches, ragged sizes, forcing,
the 4x4x3 minimum and the 128-level, 8-tracer limit; the adjoint (branch-
recording stages, the column pass with its record); the ensemble's persistent
kernel, with and without vertical diffusion.  Every call must leave the status word at ASUCA_OK, and every result
must equal the normal build's bit for bit (the checks add integer work only).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:   # run as the child script
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

pytestmark = pytest.mark.gpu


def _cases(asuca):
    """Run every case with the loaded library; returns {name: array}."""
    import torch
    out = {}

    def ok(g, what):
        torch.cuda.synchronize()
        st = asuca.get_status(g)
        assert st == asuca.OK, f"{what}: status {st}"

    shapes = [((37, 13, 7), 2, True), ((4, 4, 3), 1, False), ((70, 45, 12), 3, False),
              ((40, 24, asuca.MAX_NZ), asuca.MAX_TRACERS, False)]
    for prec in (asuca.FP64, asuca.FP32_MIXED):
        for (nx, ny, nz), ntr, with_tend in shapes:
            c = gen.make_case(nx, ny, nz, ntr, seed=300 + nx + ntr)
            for fused in (1, 0):
                g = asuca.Grid.from_case(c, prec=prec)
                asuca.set_tuning(g, asuca.TUNE_FUSED_COLUMN, fused)
                st = asuca.State.from_case(c, prec=prec)
                tend = None
                if with_tend:
                    rng = np.random.default_rng(7)
                    tend = torch.tensor(rng.standard_normal((ntr + 1, nz, ny, nx)) * 1e-4, dtype=g.torch_dtype,
                                        device=st.rho.device).contiguous()
                bud = asuca.step(g, st, c.dt, 2, tendencies=tend, budgets=True)
                name = f"step_p{prec}_{nx}x{ny}x{nz}_f{fused}"
                ok(g, name)
                out[name] = st.fields().cpu().numpy()
                out[name + "_budgets"] = bud.cpu().numpy()
            # the whole top-down half of the column pass in stage 3, and the
            # open-boundary face fluxes: the limited-area step
            if nx >= 8:
                mu_x, mv_x = gen.extend_fluxes(c.mu, c.mv)
                b0, b1 = gen.make_open_boundary(c, seed=c.seed + 1)
                g = asuca.Grid.from_case(c, prec=prec)
                tt = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=g.torch_dtype)
                st = asuca.State(tt(c.rho), tt(c.rhotheta), tt(c.rhoq), tt(mu_x), tt(mv_x), tt(c.mw))
                bud = asuca.step_open(g, st, c.dt, 2, tt(b0), bnd1=tt(b1), tratio=0.3, budgets=True)
                name = f"open_p{prec}_{nx}x{ny}x{nz}"
                ok(g, name)
                out[name] = st.fields().cpu().numpy()
                out[name + "_budgets"] = bud.cpu().numpy()
    # adjoint: recording stages, the column pass with its record, the transposes
    c = gen.make_case(24, 20, 10, 2, seed=41)
    for prec in (asuca.FP64, asuca.FP32_MIXED):
        g = asuca.Grid.from_case(c, prec=prec)
        st = asuca.State.from_case(c, prec=prec)
        rng = np.random.default_rng(3)
        lam = torch.tensor(rng.standard_normal((c.nfields, c.nz, c.ny, c.nx)), dtype=g.torch_dtype,
                           device=st.rho.device).contiguous()
        res = asuca.adjoint_step(g, st, c.dt, 4, lam, checkpoint_every=2)
        ok(g, f"adjoint_p{prec}")
        for k, r in zip(("l0", "gmu", "gmv", "gmw"), res):
            out[f"adjoint_p{prec}_{k}"] = r.cpu().numpy()
    # ensemble: the persistent kernel, with and without vertical diffusion
    cases = gen.make_ensemble_cases(sizes=[36, 50, 29], nz=9, ntracers=2)
    for prec in (asuca.FP64, asuca.FP32_MIXED):
        for k0 in (50.0, 0.0):
            grids = [asuca.Grid.from_case(cc, prec=prec, k0=k0) for cc in cases]
            states = [asuca.State.from_case(cc, prec=prec) for cc in cases]
            asuca.ensemble_step(grids, states, [cc.dt for cc in cases], 2)
            ok(grids[0], f"ensemble_p{prec}_k{k0:g}")
            for m, s in enumerate(states):
                out[f"ensemble_p{prec}_k{k0:g}_m{m}"] = s.fields().cpu().numpy()
    return out


@pytest.fixture(scope="module")
def asuca():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    return a


def test_bounds_check_build_records_nothing_and_matches_the_normal_build(asuca, tmp_path):
    from paper_1710_08616_gb300 import build as b
    lib_bc = b.build(bounds_check=True)
    assert not asuca.bounds_checked()
    ref = _cases(asuca)
    out = tmp_path / "bc.npz"
    env = dict(os.environ, ASUCA_LIBRARY=lib_bc)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    got = np.load(out)
    assert sorted(got.files) == sorted(ref)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


if __name__ == "__main__":
    # child: the bounds-check build, selected by ASUCA_LIBRARY
    import torch
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    assert a.bounds_checked(), a.library_path()
    np.savez(sys.argv[1], **_cases(a))
