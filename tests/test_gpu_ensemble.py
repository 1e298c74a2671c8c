"""Ensemble path (asuca_ensemble_step): uneven members in one persistent launch.

* every member equals asuca_step on that member alone, bit for bit (members
  never share a tile; the same tile and column code runs in both);
* a second call replays the cached CUDA graph and still matches;
* an FP64 member against the oracle (1e-12);
* the device-wide barrier gives up (test hook: it waits for one CTA more than
  the grid has) and the call reports ASUCA_ERR_TIMEOUT without faulting; the
  next call succeeds.
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


def _members(sizes, ntr=4, nz=14):
    return gen.make_ensemble_cases(sizes=sizes, nz=nz, ntracers=ntr)


@pytest.mark.parametrize("prec", [1, 0])
def test_members_equal_single_member_steps(asuca, prec):
    import torch
    cases = _members([64, 71, 40, 97, 33])
    grids = [asuca.Grid.from_case(c, prec=prec) for c in cases]
    ens = [asuca.State.from_case(c, prec=prec) for c in cases]
    one = [s.clone() for s in ens]
    n = 3
    bud = asuca.ensemble_step(grids, ens, [c.dt for c in cases], n, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(grids[0]) == asuca.OK
    for m, (g, c) in enumerate(zip(grids, cases)):
        b1 = asuca.step(g, one[m], c.dt, n, budgets=True)
        torch.cuda.synchronize()
        assert torch.equal(ens[m].fields(), one[m].fields()), f"member {m}"
        rel = (bud[m] - b1).abs() / b1.abs().clamp_min(1e-300)
        assert float(rel.max()) <= 1e-13


@pytest.mark.parametrize("prec", [1, 0])
def test_members_with_their_own_spacings_against_the_oracle(asuca, prec):
    """Members whose horizontal spacings differ from each other and between i
    and j (2000 x 1600 m, 1500 x 2000 m, 2000 x 2000 m): each member against
    the oracle's step on its own grid."""
    import torch
    spacings = [(2000.0, 1600.0), (1500.0, 2000.0), (2000.0, 2000.0)]
    cases = [gen.make_case(n, n - 5, 10, 2, seed=610 + q, dx=dx, dy=dy)
             for q, (n, (dx, dy)) in enumerate(zip([36, 44, 29], spacings))]
    grids = [asuca.Grid.from_case(c, prec=prec) for c in cases]
    states = [asuca.State.from_case(c, prec=prec) for c in cases]
    asuca.ensemble_step(grids, states, [c.dt for c in cases], 2)
    torch.cuda.synchronize()
    assert asuca.get_status(grids[0]) == asuca.OK
    tol = 1e-12 if prec == 0 else 2e-5
    for m, c in enumerate(cases):
        ref, _ = oracle.step(oracle.Grid.from_case(c), c.state(), c.mu, c.mv, c.mw, c.dt, 2)
        got = states[m].fields().double().cpu().numpy()
        for f in range(ref.shape[0]):
            l2 = np.linalg.norm(got[f] - ref[f]) / np.linalg.norm(ref[f])
            assert l2 <= tol, (m, f, l2)
            if prec == 0:
                assert np.abs(got[f] - ref[f]).max() <= tol * np.abs(ref[f]).max(), (m, f)


@pytest.mark.parametrize("sed", [0, -1])
def test_members_with_another_sedimenting_tracer_equal_single_member_steps(asuca, sed):
    """The first tracer sedimenting, or none: members equal their own
    asuca_step runs bit for bit (those are checked against the oracle for
    the same settings)."""
    import torch
    cases = _members([40, 57, 33], ntr=3, nz=10)
    grids = [asuca.Grid.from_case(c, prec=asuca.FP32_MIXED, sed_tracer=sed) for c in cases]
    ens = [asuca.State.from_case(c, prec=asuca.FP32_MIXED) for c in cases]
    one = [s.clone() for s in ens]
    asuca.ensemble_step(grids, ens, [c.dt for c in cases], 2)
    torch.cuda.synchronize()
    assert asuca.get_status(grids[0]) == asuca.OK
    for m, (g, c) in enumerate(zip(grids, cases)):
        asuca.step(g, one[m], c.dt, 2)
        torch.cuda.synchronize()
        assert torch.equal(ens[m].fields(), one[m].fields()), f"member {m}"


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("ntr,gkw", [(3, dict(lim=1)), (3, dict(lim=2)), (2, dict(tau_theta=0.0, k0=0.0, v_sed=0.0)),
                                     (2, dict(k0=0.0)), (0, dict())])
def test_members_equal_single_member_steps_across_settings(asuca, prec, ntr, gkw):
    """The other limiters, the column physics switched off in part or whole,
    and no tracers: members equal their own asuca_step runs bit for bit."""
    import torch
    cases = _members([44, 29, 61], ntr=ntr, nz=9)
    grids = [asuca.Grid.from_case(c, prec=prec, **gkw) for c in cases]
    ens = [asuca.State.from_case(c, prec=prec) for c in cases]
    one = [s.clone() for s in ens]
    bud = asuca.ensemble_step(grids, ens, [c.dt for c in cases], 2, budgets=True)
    torch.cuda.synchronize()
    assert asuca.get_status(grids[0]) == asuca.OK
    for m, (g, c) in enumerate(zip(grids, cases)):
        b1 = asuca.step(g, one[m], c.dt, 2, budgets=True)
        torch.cuda.synchronize()
        assert torch.equal(ens[m].fields(), one[m].fields()), f"member {m}"
        rel = (bud[m] - b1).abs() / b1.abs().clamp_min(1e-300)
        assert float(rel.max()) <= 1e-13


def test_graph_replay_matches(asuca):
    import torch
    cases = _members([50, 81, 64])
    grids = [asuca.Grid.from_case(c) for c in cases]
    ens = [asuca.State.from_case(c) for c in cases]
    one = [s.clone() for s in ens]
    ws = torch.empty(asuca.ensemble_workspace_bytes(grids), dtype=torch.uint8, device="cuda")
    dts = [c.dt for c in cases]
    for _ in range(3):      # the first call captures, the next ones replay
        asuca.ensemble_step(grids, ens, dts, 2, workspace=ws)
    for m, (g, c) in enumerate(zip(grids, cases)):
        for _ in range(3):
            asuca.step(g, one[m], c.dt, 2)
    torch.cuda.synchronize()
    for m in range(len(cases)):
        assert torch.equal(ens[m].fields(), one[m].fields())


def test_fp64_member_against_oracle(asuca):
    import torch
    cases = _members([40, 36], ntr=2, nz=10)
    grids = [asuca.Grid.from_case(c, prec=0) for c in cases]
    ens = [asuca.State.from_case(c, prec=0) for c in cases]
    asuca.ensemble_step(grids, ens, [c.dt for c in cases], 4)
    torch.cuda.synchronize()
    for m, c in enumerate(cases):
        ref, _ = oracle.step(oracle.Grid.from_case(c), c.state(), c.mu, c.mv, c.mw, c.dt, 4)
        got = ens[m].fields().cpu().numpy()
        for f in range(ref.shape[0]):
            assert np.linalg.norm(got[f] - ref[f]) <= 1e-12 * np.linalg.norm(ref[f])
            assert np.abs(got[f] - ref[f]).max() <= 1e-12 * np.abs(ref[f]).max()


def test_barrier_timeout_reports_status(asuca):
    import time
    import torch
    cases = _members([48, 40], nz=8)
    grids = [asuca.Grid.from_case(c) for c in cases]
    ens = [asuca.State.from_case(c) for c in cases]
    asuca.set_tuning(grids[0], asuca.TUNE_BARRIER_EXTRA, 1)
    t0 = time.time()
    asuca.ensemble_step(grids, ens, [c.dt for c in cases], 1)
    assert asuca.get_status(grids[0]) == asuca.ERR_TIMEOUT
    assert time.time() - t0 < 30
    asuca.set_tuning(grids[0], asuca.TUNE_BARRIER_EXTRA, 0)
    fresh = [asuca.State.from_case(c) for c in cases]
    asuca.ensemble_step(grids, fresh, [c.dt for c in cases], 1)
    torch.cuda.synchronize()
    assert asuca.get_status(grids[0]) == asuca.OK


def test_tile_shapes_give_identical_results_and_autotuner_picks_one(asuca, tmp_path, monkeypatch):
    import torch
    from paper_1710_08616_gb300 import autotune
    monkeypatch.setenv("ASUCA_TUNE_CACHE", str(tmp_path / "tuning.json"))
    c = gen.make_case(70, 45, 12, 3, seed=5)
    g = asuca.Grid.from_case(c)
    ref = None
    for rows in (4, 8, 16):
        for blocks in (1, 3):
            asuca.set_tuning(g, asuca.TUNE_STAGE_TILE_ROWS, rows)
            asuca.set_tuning(g, asuca.TUNE_COL_BLOCKS_PER_SM, blocks)
            st = asuca.State.from_case(c)
            asuca.step(g, st, c.dt, 3)
            torch.cuda.synchronize()
            if ref is None:
                ref = st.fields()
            assert torch.equal(st.fields(), ref), (rows, blocks)
    out = autotune.tune_step(g, asuca.State.from_case(c), c.dt, steps=1, reps=1)
    assert out["best"]["stage_tile_rows"] in (4, 8, 16)
    assert autotune.apply_cached_step(g)
    cases = _members([64, 40, 71], nz=10)
    grids = [asuca.Grid.from_case(m) for m in cases]
    outs = []
    for rows in (4, 8):
        for gg in grids:
            asuca.set_tuning(gg, asuca.TUNE_ENSEMBLE_TILE_ROWS, rows)
        sts = [asuca.State.from_case(m) for m in cases]
        asuca.ensemble_step(grids, sts, [m.dt for m in cases], 2)
        torch.cuda.synchronize()
        outs.append([s.fields() for s in sts])
    assert all(torch.equal(a, b) for a, b in zip(*outs))
    e = autotune.tune_ensemble(grids, [asuca.State.from_case(m) for m in cases], [m.dt for m in cases], steps=1, reps=1)
    assert e["best"]["ensemble_tile_rows"] in (4, 8)


def test_ensemble_step_sharded_world_size_1_equals_ensemble_step(asuca, tmp_path):
    """ensemble_step_sharded on a one-rank group (gloo, budgets gathered on the
    host) advances every member as ensemble_step does, bit for bit, and returns
    the same budgets."""
    import torch
    import torch.distributed as dist
    from paper_1710_08616_gb300.distributed import ensemble_step_sharded
    cases = _members([64, 40, 71], ntr=3, nz=10)
    grids = [asuca.Grid.from_case(c, prec=1) for c in cases]
    a = [asuca.State.from_case(c, prec=1) for c in cases]
    b = [s.clone() for s in a]
    dts = [c.dt for c in cases]
    ref = asuca.ensemble_step(grids, a, dts, 3, budgets=True).cpu().numpy().reshape(len(cases), -1)
    dist.init_process_group("gloo", init_method=f"file://{tmp_path / 'pg'}", rank=0, world_size=1)
    try:
        got = ensemble_step_sharded(grids, b, dts, 3)
    finally:
        dist.destroy_process_group()
    torch.cuda.synchronize()
    assert asuca.get_status(grids[0]) == asuca.OK
    for x, y in zip(a, b):
        assert torch.equal(x.fields(), y.fields())
    assert np.array_equal(got, ref)
