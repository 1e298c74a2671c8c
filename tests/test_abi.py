"""The C-ABI library builds, loads and exports every symbol include/asuca.h declares;
host-side argument checks (no GPU compute)."""
import ctypes
import os
import re

import pytest

import paper_1710_08616_gb300 as asuca
from paper_1710_08616_gb300 import build as asuca_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(asuca_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    asuca_build.build()
    return asuca.lib()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"asuca_init_grid", "asuca_step", "asuca_free_grid"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(asuca.SIGNATURES) == declared


def test_status_strings(lib):
    for s in range(7):
        assert lib.asuca_status_string(s)


def test_oracle_is_not_linked_into_the_product():
    # the product library must not reference the oracle's symbols
    import subprocess
    out = subprocess.run(["nm", "-D", asuca.library_path()], capture_output=True, text=True).stdout
    assert "orc_" not in out


def _desc(**kw):
    import numpy as np
    dz = np.full(kw.pop("nz", 8), 100.0)
    d = dict(nx=16, ny=12, nz=len(dz), ntracers=2, dx=2000.0, dy=2000.0, tau_theta=3600.0,
             k0=50.0, k_h=1000.0, v_sed=2.0, sed_tracer=1, lim=0, prec=1)
    d.update(kw)
    d["nz"] = len(dz)
    desc = asuca.GridDesc(d["nx"], d["ny"], d["nz"], d["ntracers"], d["dx"], d["dy"],
                          dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), d["tau_theta"], d["k0"],
                          d["k_h"], d["v_sed"], d["sed_tracer"], d["lim"], d["prec"])
    return desc, dz


@pytest.mark.parametrize("bad,status", [
    (dict(nx=3), asuca.ERR_ARG), (dict(ny=0), asuca.ERR_ARG), (dict(ntracers=9), asuca.ERR_UNSUPPORTED),
    (dict(dx=0.0), asuca.ERR_ARG), (dict(dx=float("nan")), asuca.ERR_ARG), (dict(k0=-1.0), asuca.ERR_ARG),
    (dict(sed_tracer=2), asuca.ERR_ARG), (dict(lim=7), asuca.ERR_ARG), (dict(prec=5), asuca.ERR_ARG),
])
def test_init_grid_rejects_bad_descriptions(lib, bad, status):
    desc, dz = _desc(**bad)
    h = ctypes.c_void_p()
    assert lib.asuca_init_grid(ctypes.byref(desc), ctypes.byref(h)) == status


def test_init_grid_rejects_too_many_levels(lib):
    import numpy as np
    dz = np.full(129, 100.0)
    desc = asuca.GridDesc(16, 16, 129, 1, 2000.0, 2000.0,
                          dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 0, 1, 0, -1, 0, 0)
    h = ctypes.c_void_p()
    assert lib.asuca_init_grid(ctypes.byref(desc), ctypes.byref(h)) == asuca.ERR_UNSUPPORTED


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.asuca_init_grid(None, ctypes.byref(h)) == asuca.ERR_ARG
    assert lib.asuca_free_grid(None) == asuca.ERR_ARG
    assert lib.asuca_workspace_bytes(None, 0, 0) == 0
    assert lib.asuca_step(None, None, None, 1.0, 1, None, 0, None, None) == asuca.ERR_ARG
    assert lib.asuca_stencil7(None, None, 8, 8, 4, 0, 0, 0.1, None) == asuca.ERR_ARG
    assert lib.asuca_damping(None, None, None, None, None, 0.5, 0.5, 1.0, None, None) == asuca.ERR_ARG
    assert lib.asuca_acoustic_workspace_bytes(None) == 0
    assert lib.asuca_acoustic_steps(None, None, None, None, None, None, 1.0, 1, None, 0, None) == asuca.ERR_ARG


@pytest.mark.parametrize("Q,R", [(4, 1), (4, 2), (8, 3), (64, 5), (64, 128), (12, 129)])
def test_dataflow_task_order_is_topological(lib, Q, R):
    """Host logic of the dataflow kernel: every (phase, row) task appears once
    and after the tasks it reads (phase - 1 on rows r - 1, r, r + 1, periodic)."""
    import numpy as np
    out = np.zeros(Q * R, dtype=np.uint32)
    assert lib.asuca_debug_dataflow_order(Q, R, out.ctypes.data_as(ctypes.c_void_p)) == asuca.OK
    tasks = [(int(v) >> 12, int(v) & 0xFFF) for v in out]
    assert len(set(tasks)) == Q * R
    pos = {t: k for k, t in enumerate(tasks)}
    for (q, r), k in pos.items():
        for dr in (-1, 0, 1):
            if q > 0:
                assert pos[(q - 1, (r + dr) % R)] < k
    assert lib.asuca_debug_dataflow_order(65, 4, out.ctypes.data_as(ctypes.c_void_p)) == asuca.ERR_ARG
