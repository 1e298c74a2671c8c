"""The workspace-free column pass against the workspace one.

asuca_column_noalloc serves callers that cannot allocate device memory (a
host model with a pool fixed at start-up, or code that is capturing a
stream); its scratch is an array compiled into the library instead of a
caller workspace.  Here it is called through the C ABI twice in a row on one
state, and asuca_debug_column twice in a row on a copy of it; the states and
the accumulated precipitation must agree within the parity tolerance of the
other GPU tests.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}


@pytest.mark.parametrize("prec", [0, 1])
def test_column_noalloc_matches_workspace_column_on_two_calls(prec):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as asuca
    torch.cuda.set_device(0)
    case = gen.make_case(45, 19, 16, 3, seed=2024)
    g = asuca.Grid.from_case(case, prec=prec)
    ref = asuca.State.from_case(case, prec=prec)
    got = ref.clone()
    pc_ref = torch.zeros((case.ny, case.nx), dtype=torch.float64, device="cuda")
    pc_got = torch.zeros_like(pc_ref)
    ws = g.workspace()
    for call in range(2):
        asuca.debug_column(g, ref, case.dt, pc_ref, workspace=ws)
        asuca.column_noalloc(g, got, case.dt, pc_got)
        torch.cuda.synchronize()
        a = got.fields().double().cpu().numpy()
        b = ref.fields().double().cpu().numpy()
        for f in range(a.shape[0]):
            err = np.linalg.norm(a[f] - b[f]) / np.linalg.norm(b[f])
            assert err <= TOL[prec], f"call {call} field {f}: rel L2 {err:.3e}"
        pa, pb = pc_got.cpu().numpy(), pc_ref.cpu().numpy()
        assert np.linalg.norm(pa - pb) <= TOL[prec] * np.linalg.norm(pb)
        assert np.abs(pb).max() > 0.0
    assert asuca.get_status(g) == asuca.OK


@pytest.mark.parametrize("prec", [0, 1])
def test_column_noalloc_at_compiled_limits_reuses_scratch_slots(prec):
    """128 levels and 8 tracers (the compiled limits) on 64 x 64 columns: a
    128-column block needs 1.44 MB of scratch, so 11 blocks fit in the array
    while the columns need 32.  Each thread then carries its scratch slot from
    column to column (the grid-stride reuse), over two calls in a row."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as asuca
    torch.cuda.set_device(0)
    case = gen.make_case(64, 64, 128, 8, seed=77)
    g = asuca.Grid.from_case(case, prec=prec)
    ref = asuca.State.from_case(case, prec=prec)
    got = ref.clone()
    pc_ref = torch.zeros((case.ny, case.nx), dtype=torch.float64, device="cuda")
    pc_got = torch.zeros_like(pc_ref)
    ws = g.workspace()
    for call in range(2):
        asuca.debug_column(g, ref, case.dt, pc_ref, workspace=ws)
        asuca.column_noalloc(g, got, case.dt, pc_got)
        torch.cuda.synchronize()
        a = got.fields().double().cpu().numpy()
        b = ref.fields().double().cpu().numpy()
        for f in range(a.shape[0]):
            err = np.linalg.norm(a[f] - b[f]) / np.linalg.norm(b[f])
            mx = np.abs(a[f] - b[f]).max() / np.abs(b[f]).max()
            assert err <= TOL[prec] and mx <= TOL[prec], f"call {call} field {f}: rel L2 {err:.3e}, max {mx:.3e}"
        pa, pb = pc_got.cpu().numpy(), pc_ref.cpu().numpy()
        assert np.linalg.norm(pa - pb) <= TOL[prec] * np.linalg.norm(pb)
    assert asuca.get_status(g) == asuca.OK


@pytest.mark.parametrize("prec", [0, 1])
def test_column_noalloc_256x256x58_8_tracers_against_oracle(prec):
    """65,536 columns with 8 tracers: 25 blocks fit in the array, so most
    scratch slots serve about 20 columns each; the result is compared with the
    oracle's FP64 column pass on the same state."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1710_08616_gb300 as asuca
    torch.cuda.set_device(0)
    case = gen.make_case(256, 256, 58, 8, seed=58)
    g = asuca.Grid.from_case(case, prec=prec)
    st = asuca.State.from_case(case, prec=prec)
    pc = torch.zeros((case.ny, case.nx), dtype=torch.float64, device="cuda")
    asuca.column_noalloc(g, st, case.dt, pc)
    torch.cuda.synchronize()
    assert asuca.get_status(g) == asuca.OK
    # the oracle starts from the state the GPU started from (rounded to float for FP32)
    y0 = asuca.State.from_case(case, prec=prec).fields().double().cpu().numpy()
    ref, pref = oracle.column(oracle.Grid.from_case(case), y0, case.dt)
    got = st.fields().double().cpu().numpy()
    for f in range(ref.shape[0]):
        err = np.linalg.norm(got[f] - ref[f]) / np.linalg.norm(ref[f])
        assert err <= TOL[prec], f"field {f}: rel L2 {err:.3e}"
        if prec == 0:
            mx = np.abs(got[f] - ref[f]).max() / np.abs(ref[f]).max()
            assert mx <= TOL[prec], f"field {f}: rel max {mx:.3e}"
    assert np.linalg.norm(pc.cpu().numpy() - pref) <= TOL[prec] * np.linalg.norm(pref)
