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
    """Every status the header declares has its own message; other values
    read as unknown."""
    src = open(os.path.join(ROOT, "include", "asuca.h")).read()
    codes = {int(v) for v in re.findall(r"\bASUCA_(?:OK|ERR_[A-Z]+)\s*=\s*(\d+)", src)}
    assert codes == set(range(len(codes))) and len(codes) >= 8
    msgs = [lib.asuca_status_string(c) for c in sorted(codes)]
    assert all(msgs) and len(set(msgs)) == len(msgs)
    unknown = lib.asuca_status_string(max(codes) + 1)
    assert unknown not in msgs and lib.asuca_status_string(-1) == unknown


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


@pytest.mark.parametrize("nx,ny,nz,width,ntop", [(17, 11, 7, 3, 2), (4, 4, 3, 2, 3), (70, 9, 5, 4, 0),
                                                 (32, 32, 16, 0, 5), (300, 130, 12, 64, 1), (512, 256, 20, 16, 8),
                                                 (5, 7, 4, 0, 0)])
def test_damping_zone_enumeration(lib, nx, ny, nz, width, ntop):
    """Host logic of the damping kernel: its flat index visits every cell of
    the zone (fewer than `width` cells from an i or j edge, or on the top ntop
    levels) exactly once and nothing else, consecutive indices mostly on
    consecutive i (coalesced)."""
    import numpy as np
    n = lib.asuca_damping_zone_cells(nx, ny, nz, width, ntop)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.minimum(np.minimum(i, nx - 1 - i), np.minimum(j, ny - 1 - j))
    zone = (d < width) | (k >= nz - ntop)
    assert n == int(zone.sum())
    if n == 0:
        return
    out = np.zeros(3 * n, dtype=np.uint32)
    assert lib.asuca_debug_damping_cells(nx, ny, nz, width, ntop, out.ctypes.data_as(ctypes.c_void_p), n) == asuca.OK
    ijk = out.reshape(n, 3).astype(np.int64)
    assert ijk[:, 0].max() < nx and ijk[:, 1].max() < ny and ijk[:, 2].max() < nz
    flat = (ijk[:, 2] * ny + ijk[:, 1]) * nx + ijk[:, 0]
    assert len(np.unique(flat)) == n
    assert zone.reshape(-1)[flat].all()
    steps = np.diff(flat)
    assert np.mean(steps == 1) > 0.5


def test_damping_zone_arguments(lib):
    import numpy as np
    assert lib.asuca_damping_zone_cells(16, 12, 5, 7, 1) == 0        # 2 width > ny
    assert lib.asuca_damping_zone_cells(16, 12, 5, 2, 6) == 0        # ntop > nz
    assert lib.asuca_damping_zone_cells(200, 200, 5, 65, 1) == 0     # wider than the library takes
    n = lib.asuca_damping_zone_cells(16, 12, 5, 2, 1)
    out = np.zeros(3 * n, dtype=np.uint32)
    assert lib.asuca_debug_damping_cells(16, 12, 5, 2, 1, out.ctypes.data_as(ctypes.c_void_p), n - 1) == asuca.ERR_ARG
    assert lib.asuca_debug_damping_cells(16, 12, 5, 2, 1, None, n) == asuca.ERR_ARG


def test_binding_matches_the_header_layouts_and_constants(tmp_path):
    """A small C program compiled against include/asuca.h prints the size and
    every member's offset and size of the structures the binding mirrors, and
    the value of every ASUCA_ constant; the ctypes structures and the module's
    constants of the same names must agree."""
    import subprocess
    structs = {"asuca_grid_desc": asuca.GridDesc, "asuca_state": asuca.StateStruct,
               "asuca_damping_desc": asuca.DampingDesc, "asuca_acoustic_desc": asuca.AcousticDesc}
    src = open(os.path.join(ROOT, "include", "asuca.h")).read()
    names = sorted(set(re.findall(r"\bASUCA_([A-Z][A-Z0-9_]*)\b", src)) - {"H", "BOUNDS_CHECK"})
    names = [n for n in names if hasattr(asuca, n)]
    assert {"OK", "ERR_BOUNDS", "FP64", "FP32_MIXED", "LIM_KOREN", "MAX_NZ", "MAX_TRACERS",
            "KERNEL_STAGE_FACTOR", "TUNE_FUSED_COLUMN", "OP_STEP"} <= set(names)
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "asuca.h"', "int main(void) {"]
    for cname, py in structs.items():
        prog.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            prog.append(f'printf("{cname}.{fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                        f'sizeof((({cname} *)0)->{fname}));')
    for n in names:
        prog.append(f'printf("ASUCA_{n} %lld\\n", (long long)(ASUCA_{n}));')
    prog.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["cc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        key, *vals = line.split()
        vals = [int(v) for v in vals]
        if key.startswith("ASUCA_"):
            assert getattr(asuca, key[len("ASUCA_"):]) == vals[0], key
        elif "." in key:
            cname, fname = key.split(".")
            fld = getattr(structs[cname], fname)
            assert (fld.offset, fld.size) == tuple(vals), key
        else:
            assert ctypes.sizeof(structs[key]) == vals[0], key
        seen += 1
    assert seen == len(names) + sum(1 + len(py._fields_) for py in structs.values())


def _prototypes():
    """{name: (return type, [parameter declarations])} from include/*.h"""
    protos = {}
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
        src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
        for ret, name, params in re.findall(r"([A-Za-z_][\w \t\*]*?)\s*\b(asuca_[a-z0-9_]+)\s*\(([^;{}]*?)\)\s*;",
                                            src, flags=re.S):
            ps = [p.strip() for p in params.split(",")]
            protos[name] = (" ".join(ret.split()), [] if ps == ["void"] or ps == [""] else ps)
    return protos


def test_binding_signatures_match_the_header_prototypes():
    """Every ctypes signature has the header prototype's parameter count, a
    pointer type where the prototype takes a pointer, and the scalar type it
    declares (double, size_t, long long; int for int and the enums); the
    return types agree likewise."""
    protos = _prototypes()
    assert set(protos) == set(asuca.SIGNATURES)

    def is_ptr(t):
        return t in (ctypes.c_void_p, ctypes.c_char_p) or isinstance(t, type) and issubclass(t, ctypes._Pointer)

    def scalar(decl):
        words = decl.replace("const", " ").split()[:-1]          # drop the parameter name
        base = " ".join(words) if words else decl.split()[0]
        return {"double": ctypes.c_double, "size_t": ctypes.c_size_t, "long long": ctypes.c_longlong,
                "int": ctypes.c_int}.get(base, ctypes.c_int if base.startswith("asuca_") else None)

    for name, (ret, params) in protos.items():
        want_ret, args = asuca.SIGNATURES[name]
        assert len(args) == len(params), f"{name}: {len(args)} ctypes arguments, header has {len(params)}"
        for q, (decl, t) in enumerate(zip(params, args)):
            if "*" in decl:
                assert is_ptr(t), f"{name} argument {q} ({decl}) is a pointer, binding has {t}"
            else:
                assert t is scalar(decl), f"{name} argument {q} ({decl}): binding has {t}"
        if "*" in ret:
            assert want_ret is ctypes.c_char_p and "char" in ret, name
        else:
            assert want_ret is scalar(ret + " x"), f"{name} returns {ret}, binding has {want_ret}"
