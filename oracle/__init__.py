"""FP64 CPU oracle of the ASUCA-style step -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It compiles asuca_oracle.c (plain C, FP64, no fast-math, no FP
contraction) into liborc.so next to the source and calls it through ctypes
(ORACLE_LIBRARY, if set, names another build of the same source to load).
It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asuca_oracle.c")
_HDR = os.path.join(_HERE, "asuca_oracle.h")
_SO = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

LIM_KOREN, LIM_LINEAR, LIM_UPWIND1 = 0, 1, 2
# default physics constants (relaxation time, diffusivity scale, decay height, fall speed)
TAU, K0, KH, VSED = 3600.0, 50.0, 1000.0, 2.0


def compile_library(src: str, out: str) -> str:
    """Compile an oracle source file (including asuca_oracle.h from this
    directory) into the shared library `out`, with the oracle's flags."""
    cc = os.environ.get("CC", "cc")
    cmd = [cc, "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-std=c11",
           "-shared", "-fPIC", "-I", _HERE, "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
            return _SO
        tmp = _SO + f".tmp{os.getpid()}"
        compile_library(_SRC, tmp)
        os.replace(tmp, _SO)
        return _SO


class OrcGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ntr", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.POINTER(ctypes.c_double)), ("tau", ctypes.c_double),
                ("k0", ctypes.c_double), ("kh", ctypes.c_double), ("vsed", ctypes.c_double),
                ("sed", ctypes.c_int), ("lim", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


def lib():
    """The loaded oracle library: liborc.so built from the source beside this
    file, or the library named by ORACLE_LIBRARY (the mutation test loads
    copies of the oracle with one planted slip each through it)."""
    global _lib
    if _lib is None:
        so = os.environ.get("ORACLE_LIBRARY")
        if not so:
            build()
            so = _SO
        L = ctypes.CDLL(so)
        G = ctypes.POINTER(OrcGrid)
        L.orc_limiter.restype = ctypes.c_double
        L.orc_limiter.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int)]
        L.orc_face.restype = ctypes.c_double
        L.orc_face.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_rhs.argtypes = [G, _D, _D, _D, _D, _D, _D, _U8]
        L.orc_euler.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, _D]
        L.orc_rk3.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double]
        L.orc_column.argtypes = [G, _D, ctypes.c_double, _D]
        L.orc_thomas.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_budgets.argtypes = [G, _D, ctypes.c_double, _D]
        L.orc_step.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D]
        L.orc_step_window.restype = ctypes.c_int
        L.orc_step_window.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.orc_stencil7.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_acoustic.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_D, _D, _D] + \
            [ctypes.c_double] * 3 + [ctypes.c_int, _D, _D, _D, _D]
        L.orc_damping.argtypes = [ctypes.c_int] * 6 + [ctypes.c_double] * 5 + [ctypes.c_longlong,
                                  ctypes.POINTER(ctypes.c_int), _D, _D, _D, _D]
        L.orc_rhs_open.argtypes = [G, _D, _D, _D, _D, _D, _D, _D]
        L.orc_step_open.argtypes = [G, _D, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D]
        L.orc_hevi_short_steps.restype = ctypes.c_int
        L.orc_hevi_short_steps.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_step_hevi.argtypes = [G, _D, _D, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, _D, _D, _D]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Grid:
    """Grid + physics constants.  Defaults follow the scheme's readings."""

    def __init__(self, nx, ny, nz, ntr, dz, dx=2000.0, dy=2000.0, *, tau=TAU, k0=K0, kh=KH,
                 vsed=VSED, sed=None, lim=LIM_KOREN):
        self.dz = np.ascontiguousarray(dz, dtype=np.float64)
        assert self.dz.shape == (nz,)
        if sed is None:
            sed = ntr - 1
        self.s = OrcGrid(nx, ny, nz, ntr, dx, dy, _p(self.dz), tau, k0, kh, vsed, sed, lim)
        self.nx, self.ny, self.nz, self.ntr = nx, ny, nz, ntr

    @classmethod
    def from_case(cls, case, **kw):
        return cls(case.nx, case.ny, case.nz, case.ntracers, case.dz, case.dx, case.dy, **kw)

    @property
    def F(self):
        return 2 + self.ntr

    @property
    def shape(self):
        return (self.F, self.nz, self.ny, self.nx)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def limiter(d0, d1, lim=LIM_KOREN):
    b = ctypes.c_int(-1)
    v = lib().orc_limiter(float(d0), float(d1), lim, ctypes.byref(b))
    return v, b.value


def face(pm1, p0, p1, p2, m, lim=LIM_KOREN):
    b = ctypes.c_int(-1)
    v = lib().orc_face(float(pm1), float(p0), float(p1), float(p2), float(m), lim, ctypes.byref(b))
    return v, b.value


def rhs(g: Grid, Y, mu, mv, mw, tend=None, branches=False):
    Y, mu, mv, mw = _f64(Y), _f64(mu), _f64(mv), _f64(mw)
    tend = None if tend is None else _f64(tend)
    R = np.empty(g.shape)
    br = np.zeros(g.shape, dtype=np.uint8) if branches else None
    lib().orc_rhs(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(tend), _p(R),
                  None if br is None else br.ctypes.data_as(_U8))
    return (R, br) if branches else R


def euler(g: Grid, Y, mu, mv, mw, dt, tend=None):
    Y, mu, mv, mw = _f64(Y), _f64(mu), _f64(mv), _f64(mw)
    tend = None if tend is None else _f64(tend)
    out = np.empty(g.shape)
    lib().orc_euler(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(tend), dt, _p(out))
    return out


def rk3(g: Grid, Y, mu, mv, mw, dt, tend=None):
    Y = _f64(Y).copy()
    mu, mv, mw = _f64(mu), _f64(mv), _f64(mw)
    tend = None if tend is None else _f64(tend)
    lib().orc_rk3(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(tend), dt)
    return Y


def column(g: Grid, Y, dt):
    """Column physics (relaxation, sedimentation, diffusion); returns (Y, precip per column)."""
    Y = _f64(Y).copy()
    pc = np.zeros((g.ny, g.nx))
    lib().orc_column(g.ref, _p(Y), dt, _p(pc))
    return Y, pc


def thomas(a, b, c, d):
    a, b, c, d = _f64(a), _f64(b), _f64(c), _f64(d)
    x = np.empty_like(d)
    lib().orc_thomas(len(d), _p(a), _p(b), _p(c), _p(d), _p(x))
    return x


def stencil7(field, c):
    """One explicit 7-point diffusion step of a [nz][ny][nx] field (periodic in i
    and j, zero flux through the lids)."""
    f = np.ascontiguousarray(_f64(field))
    nz, ny, nx = f.shape
    out = np.empty_like(f)
    lib().orc_stencil7(nx, ny, nz, float(c), _p(f), _p(out))
    return out


def damping(Y, ref, b0, b1, tratio, dt, *, width, ntop, nu_lat, nu_top, mtratio=None, ijk=None, shape=None):
    """Lateral and upper damping toward boundary data (Sec. 2.1's damping kernel
    target, relaxed implicitly).  Whole domain: Y, ref, b0, b1 are [F][nz][ny][nx].
    Sampled cells: ijk is an [n][3] int array of (i, j, k), the arrays are
    [F][n], and shape = (nx, ny, nz) gives the domain.  Returns the new Y."""
    if mtratio is None:
        mtratio = 1.0 - tratio
    y = np.array(_f64(Y), dtype=np.float64, order="C", copy=True)
    r, p0, p1 = (np.ascontiguousarray(_f64(a)) for a in (ref, b0, b1))
    assert r.shape == y.shape and p0.shape == y.shape and p1.shape == y.shape
    if ijk is None:
        F, nz, ny, nx = y.shape
        n, ip = 0, None
    else:
        nx, ny, nz = shape
        idx = np.ascontiguousarray(ijk, dtype=np.int32)
        F, n = y.shape
        assert idx.shape == (n, 3)
        ip = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    lib().orc_damping(nx, ny, nz, F, int(width), int(ntop), float(nu_lat), float(nu_top), float(mtratio),
                      float(tratio), float(dt), int(n), ip, _p(y), _p(r), _p(p0), _p(p1))
    return y


def acoustic(U, V, W, S, dz, rho0c, rho0f, cs2, beta, dtau, nshort, dx=2000.0, dy=2000.0):
    """nshort HEVI short steps of the linear acoustic-gravity system (Sec. 1.1).
    U, V, S: [nz][ny][nx]; W: [nz+1][ny][nx] (W[0], W[nz] rigid lids, kept).
    Returns new (U, V, W, S) arrays."""
    U, V, W, S = (np.array(_f64(a), dtype=np.float64, order="C", copy=True) for a in (U, V, W, S))
    nz, ny, nx = S.shape
    assert U.shape == S.shape and V.shape == S.shape and W.shape == (nz + 1, ny, nx)
    dz, r0c, r0f = (np.ascontiguousarray(_f64(a)) for a in (dz, rho0c, rho0f))
    assert dz.shape == (nz,) and r0c.shape == (nz,) and r0f.shape == (nz + 1,)
    lib().orc_acoustic(nx, ny, nz, float(dx), float(dy), _p(dz), _p(r0c), _p(r0f), float(cs2), float(beta),
                       float(dtau), int(nshort), _p(U), _p(V), _p(W), _p(S))
    return U, V, W, S


def budgets(g: Grid, Y, precip=0.0):
    out = np.empty(g.F + 1)
    lib().orc_budgets(g.ref, _p(_f64(Y)), float(precip), _p(out))
    return out


def step(g: Grid, Y, mu, mv, mw, dt, nsteps, tend=None):
    """nsteps full steps; returns (Y, budgets[F+1]: mass, rho*theta, tracers, precip)."""
    Y = _f64(Y).copy()
    mu, mv, mw = _f64(mu), _f64(mv), _f64(mw)
    tend = None if tend is None else _f64(tend)
    bud = np.empty(g.F + 1)
    lib().orc_step(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(tend), dt, nsteps, _p(bud))
    return Y, bud


def hevi_short_steps(ns: int, q: int) -> int:
    return int(lib().orc_hevi_short_steps(int(ns), int(q)))


def step_hevi(g: Grid, Y, U, V, W, rho0c, rho0f, cs2, beta, ns, dt, nsteps, tend=None, stage_rho=False):
    """nsteps long steps with the acoustic short steps nested in the RK3 stages;
    returns (Y, U, V, W, s_final, budgets[F+1]), and with stage_rho the density
    of the last step's first two RK stages ([2][nz][ny][nx]) as a seventh item."""
    Y, U, V, W = (_f64(a).copy() for a in (Y, U, V, W))
    rho0c, rho0f = _f64(rho0c), _f64(rho0f)
    tend = None if tend is None else _f64(tend)
    s_final = np.zeros(g.shape[1:])
    bud = np.empty(g.F + 1)
    srho = np.zeros((2,) + tuple(g.shape[1:])) if stage_rho else None
    lib().orc_step_hevi(g.ref, _p(Y), _p(U), _p(V), _p(W), _p(tend), _p(rho0c), _p(rho0f), float(cs2),
                        float(beta), int(ns), float(dt), int(nsteps), _p(s_final), _p(bud), _p(srho))
    if stage_rho:
        return Y, U, V, W, s_final, bud, srho
    return Y, U, V, W, s_final, bud


def halo_size(g: Grid) -> int:
    """values of one halo-layout array: 2 (2 ny + 2 nx) nz (F - 1)"""
    return 2 * (2 * g.ny + 2 * g.nx) * g.nz * (g.F - 1)


def rhs_open(g: Grid, Y, mu_x, mv_x, mw, ghost, tend=None):
    """R of an open domain (ghost phi in the halo layout, extended face fluxes)."""
    Y, mu_x, mv_x, mw, ghost = map(_f64, (Y, mu_x, mv_x, mw, ghost))
    assert mu_x.shape == (g.nz, g.ny, g.nx + 1) and mv_x.shape == (g.nz, g.ny + 1, g.nx)
    assert ghost.size == halo_size(g)
    tend = None if tend is None else _f64(tend)
    R = np.empty(g.shape)
    lib().orc_rhs_open(g.ref, _p(Y), _p(mu_x), _p(mv_x), _p(mw), _p(tend), _p(ghost), _p(R))
    return R


def step_open(g: Grid, Y, mu_x, mv_x, mw, ghost, dt, nsteps, tend=None):
    """nsteps steps of an open domain; returns (Y, budgets[F+1])."""
    Y = _f64(Y).copy()
    mu_x, mv_x, mw, ghost = map(_f64, (mu_x, mv_x, mw, ghost))
    assert mu_x.shape == (g.nz, g.ny, g.nx + 1) and mv_x.shape == (g.nz, g.ny + 1, g.nx)
    assert ghost.size == halo_size(g)
    tend = None if tend is None else _f64(tend)
    bud = np.empty(g.F + 1)
    lib().orc_step_open(g.ref, _p(Y), _p(mu_x), _p(mv_x), _p(mw), _p(tend), _p(ghost), dt, nsteps, _p(bud))
    return Y, bud


def step_window(g: Grid, Y, mu, mv, mw, dt, nsteps, i0, j0, w, h, tend=None):
    """nsteps steps evaluated only on the cone of the window; returns [F][nz][h][w]."""
    Y, mu, mv, mw = _f64(Y), _f64(mu), _f64(mv), _f64(mw)
    tend = None if tend is None else _f64(tend)
    out = np.empty((g.F, g.nz, h, w))
    rc = lib().orc_step_window(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(tend), dt, nsteps,
                               i0, j0, w, h, _p(out))
    if rc:
        raise RuntimeError(f"orc_step_window failed ({rc})")
    return out


def set_threads(n: int):
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


# ---------------------------------------------------------------- tangent-linear / adjoint

def _sig_tl():
    L = lib()
    if not getattr(L, "_tl_ready", False):
        G = ctypes.POINTER(OrcGrid)
        L.orc_rhs_tl.argtypes = [G, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.orc_rhs_adj.argtypes = [G, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.orc_column_tl.argtypes = [G, _D, _D, ctypes.c_double, _D]
        L.orc_column_adj.argtypes = [G, _D, _D, ctypes.c_double]
        L.orc_step_tl.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_step_adj.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_trajectory_branches.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _U8]
        L.orc_step_tl_br.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D, _D, _D, _U8, _D]
        L.orc_step_adj_br.argtypes = [G, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _U8, _D, _D, _D, _D]
        L._tl_ready = True
    return L


def rhs_tl(g: Grid, Y, mu, mv, mw, dY, dmu=None, dmv=None, dmw=None):
    L = _sig_tl()
    Y, mu, mv, mw, dY = map(_f64, (Y, mu, mv, mw, dY))
    dm = [None if a is None else _f64(a) for a in (dmu, dmv, dmw)]
    out = np.empty(g.shape)
    L.orc_rhs_tl(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(dY), _p(dm[0]), _p(dm[1]), _p(dm[2]), _p(out))
    return out


def rhs_adj(g: Grid, Y, mu, mv, mw, lamR):
    """((dR/dY)^T lamR, (dR/dMU)^T lamR, (dR/dMV)^T lamR, (dR/dMW)^T lamR)"""
    L = _sig_tl()
    Y, mu, mv, mw, lamR = map(_f64, (Y, mu, mv, mw, lamR))
    lY = np.zeros(g.shape)
    gmu, gmv, gmw = np.zeros_like(mu), np.zeros_like(mv), np.zeros_like(mw)
    L.orc_rhs_adj(g.ref, _p(Y), _p(mu), _p(mv), _p(mw), _p(lamR), _p(lY), _p(gmu), _p(gmv), _p(gmw))
    return lY, gmu, gmv, gmw


def column_tl(g: Grid, Y3, dY3, dt):
    L = _sig_tl()
    out = np.empty(g.shape)
    L.orc_column_tl(g.ref, _p(_f64(Y3)), _p(_f64(dY3)), dt, _p(out))
    return out


def column_adj(g: Grid, Y3, lam, dt):
    L = _sig_tl()
    lam = _f64(lam).copy()
    L.orc_column_adj(g.ref, _p(_f64(Y3)), _p(lam), dt)
    return lam


def _traj_br(g, nsteps, traj_br):
    if traj_br is None:
        return None
    b = np.ascontiguousarray(traj_br, dtype=np.uint8)
    assert b.shape == (nsteps, 3) + g.shape, b.shape
    return b


def step_tl(g: Grid, Y0, mu, mv, mw, dt, nsteps, dY0, dmu=None, dmv=None, dmw=None, tend=None,
            traj_br=None):
    """traj_br ([nsteps][3][F][nz][ny][nx] bytes), when given, fixes every face's branch"""
    L = _sig_tl()
    Y0, mu, mv, mw, dY0 = map(_f64, (Y0, mu, mv, mw, dY0))
    dm = [None if a is None else _f64(a) for a in (dmu, dmv, dmw)]
    tend = None if tend is None else _f64(tend)
    out = np.empty(g.shape)
    br = _traj_br(g, nsteps, traj_br)
    L.orc_step_tl_br(g.ref, _p(Y0), _p(mu), _p(mv), _p(mw), _p(tend), dt, nsteps, _p(dY0),
                     _p(dm[0]), _p(dm[1]), _p(dm[2]), None if br is None else br.ctypes.data_as(_U8),
                     _p(out))
    return out


def step_adj(g: Grid, Y0, mu, mv, mw, dt, nsteps, lam_final, tend=None, traj_br=None):
    """adjoint of nsteps steps: (lam0 [F][nz][ny][nx], g_mu, g_mv, g_mw); traj_br as in step_tl"""
    L = _sig_tl()
    Y0, mu, mv, mw, lam_final = map(_f64, (Y0, mu, mv, mw, lam_final))
    tend = None if tend is None else _f64(tend)
    lam0 = np.empty(g.shape)
    gmu, gmv, gmw = np.empty_like(mu), np.empty_like(mv), np.empty_like(mw)
    br = _traj_br(g, nsteps, traj_br)
    L.orc_step_adj_br(g.ref, _p(Y0), _p(mu), _p(mv), _p(mw), _p(tend), dt, nsteps, _p(lam_final),
                      None if br is None else br.ctypes.data_as(_U8), _p(lam0), _p(gmu), _p(gmv), _p(gmw))
    return lam0, gmu, gmv, gmw


def trajectory_branches(g: Grid, Y0, mu, mv, mw, dt, nsteps, tend=None):
    """limiter branch bytes of every face of every stage of nsteps steps"""
    L = _sig_tl()
    Y0, mu, mv, mw = map(_f64, (Y0, mu, mv, mw))
    tend = None if tend is None else _f64(tend)
    out = np.zeros((max(nsteps, 1), 3) + g.shape, dtype=np.uint8)
    L.orc_trajectory_branches(g.ref, _p(Y0), _p(mu), _p(mv), _p(mw), _p(tend), dt, nsteps,
                              out.ctypes.data_as(_U8))
    return out


def tracer_cost(g: Grid, Y, q_target):
    """J = 1/2 sum over cells and tracers of (q_n - q_target_n)^2, q = rho q / rho,
    and its gradient with respect to Y (all F fields)."""
    Y = _f64(Y)
    q = Y[2:] / Y[0]
    r = q - q_target
    J = 0.5 * float(np.sum(r * r))
    lam = np.zeros(g.shape)
    lam[2:] = r / Y[0]
    lam[0] = -np.sum(r * q, axis=0) / Y[0]
    return J, lam
