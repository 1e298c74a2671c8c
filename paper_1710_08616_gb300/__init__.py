"""Python binding of libasuca (the C ABI in include/asuca.h).

Argument marshalling only: every step of the time step runs in the CUDA
kernels of libasuca.so.  PyTorch supplies device memory (tensors) and
streams.  There is no CPU fallback: if the compiled library is missing,
every entry point raises.

The computation is the ASUCA-style step that the Hybrid Fortran paper
(arXiv 1710.08616) ports to GPUs: Wicker-Skamarock RK3 of flux-form rho,
rho*theta and rho*q_n with Koren-limited i/j/k fluxes on a periodic
Arakawa-C grid (Sec. 1.1 "ASUCA on GPU"), then per-column physics and an
FP64 implicit vertical-diffusion solve (Sec. 1.2 "Parallelization
Granularity"), with i-fastest fields (Sec. 1.3 "Memory Layout").
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _DEFAULT_LIB

# ASUCA_LIBRARY selects another build of the library for this process (the
# bounds-check build, libasuca_bc.so, in its tests); it must exist, as the
# default must: there is no fallback.
_LIB_PATH = os.environ.get("ASUCA_LIBRARY") or _DEFAULT_LIB

OK, ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_BOUNDS = range(8)
FP64, FP32_MIXED = 0, 1
LIM_KOREN, LIM_LINEAR, LIM_UPWIND1 = 0, 1, 2
OP_STEP, OP_ADJOINT, OP_ENSEMBLE = 0, 1, 2
MAX_TRACERS = 8
MAX_NZ = 128

_STATUS = {OK: "ok", ERR_ARG: "invalid argument", ERR_CUDA: "CUDA runtime error",
           ERR_WORKSPACE: "workspace missing, misaligned or too small",
           ERR_NONFINITE: "non-finite budget", ERR_TIMEOUT: "device barrier timed out",
           ERR_UNSUPPORTED: "unsupported size", ERR_BOUNDS: "a kernel index fell outside its buffer"}


class AsucaError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, 'unknown')} ({status})")


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ntracers", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.POINTER(ctypes.c_double)), ("tau_theta", ctypes.c_double),
                ("k0", ctypes.c_double), ("k_h", ctypes.c_double), ("v_sed", ctypes.c_double),
                ("sed_tracer", ctypes.c_int), ("lim", ctypes.c_int), ("prec", ctypes.c_int)]


class StateStruct(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_void_p), ("rhotheta", ctypes.c_void_p), ("rhoq", ctypes.c_void_p),
                ("mu", ctypes.c_void_p), ("mv", ctypes.c_void_p), ("mw", ctypes.c_void_p)]


class DampingDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("ntop", ctypes.c_int), ("nu_lat", ctypes.c_double),
                ("nu_top", ctypes.c_double)]


class AcousticDesc(ctypes.Structure):
    _fields_ = [("rho0c", ctypes.POINTER(ctypes.c_double)), ("rho0f", ctypes.POINTER(ctypes.c_double)),
                ("cs2", ctypes.c_double), ("beta", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p

# every symbol the C ABI exports, with its ctypes signature
SIGNATURES = {
    "asuca_init_grid": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.POINTER(_VP)]),
    "asuca_free_grid": (ctypes.c_int, [_VP]),
    "asuca_workspace_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int, ctypes.c_int]),
    "asuca_step": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double,
                                  ctypes.c_int, _VP, ctypes.c_size_t, _VP, _VP]),
    "asuca_get_status": (ctypes.c_int, [_VP]),
    "asuca_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "asuca_bounds_checked": (ctypes.c_int, []),
    "asuca_debug_stage": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), ctypes.POINTER(StateStruct),
                                         ctypes.POINTER(StateStruct), _VP, ctypes.c_double, _VP]),
    "asuca_debug_column": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), ctypes.c_double, _VP,
                                          _VP, ctypes.c_size_t, _VP]),
    "asuca_debug_numerics": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "asuca_column_noalloc": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), ctypes.c_double, _VP, _VP]),
    "asuca_stencil7": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, _VP]),
    "asuca_damping": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, _VP, _VP, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.POINTER(DampingDesc), _VP]),
    "asuca_damping_zone_cells": (ctypes.c_size_t, [ctypes.c_int] * 5),
    "asuca_debug_damping_cells": (ctypes.c_int, [ctypes.c_int] * 5 + [_VP, ctypes.c_size_t]),
    "asuca_acoustic_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "asuca_acoustic_steps": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(AcousticDesc), ctypes.c_double,
                                            ctypes.c_int, _VP, ctypes.c_size_t, _VP]),
    "asuca_adjoint_workspace_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int, ctypes.c_int]),
    "asuca_adjoint_step": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "asuca_checkpoint_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int, ctypes.c_int]),
    "asuca_forward_checkpointed": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double,
                                                  ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t, _VP,
                                                  ctypes.c_size_t, _VP, _VP]),
    "asuca_adjoint_from_checkpoints": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double,
                                                      ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP,
                                                      ctypes.c_size_t, _VP]),
    "asuca_debug_record_branches": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double,
                                                   ctypes.c_int, _VP, _VP, ctypes.c_size_t, _VP]),
    "asuca_ensemble_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(_VP), ctypes.c_int]),
    "asuca_ensemble_step": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(StateStruct),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int, _VP,
                                           ctypes.c_size_t, _VP, _VP]),
    "asuca_set_tuning": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "asuca_get_tuning": (ctypes.c_int, [_VP, ctypes.c_int]),
    "asuca_debug_dataflow_order": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP]),
    "asuca_open_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "asuca_halo_count": (ctypes.c_size_t, [_VP]),
    "asuca_open_prepare": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), ctypes.c_int, _VP, ctypes.c_size_t,
                                          _VP]),
    "asuca_open_stage": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double, ctypes.c_int, _VP,
                                        ctypes.c_size_t, _VP, _VP]),
    "asuca_halo_pack": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.c_int, _VP, _VP]),
    "asuca_halo_unpack": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.c_int, _VP, _VP, ctypes.c_double, _VP]),
    "asuca_step_open": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double, ctypes.c_int, _VP,
                                       _VP, ctypes.c_double, _VP, ctypes.c_size_t, _VP, _VP]),
    "asuca_hevi_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "asuca_step_hevi": (ctypes.c_int, [_VP, ctypes.POINTER(StateStruct), _VP, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(AcousticDesc), ctypes.c_int, _VP, _VP, ctypes.c_size_t, _VP, _VP]),
    "asuca_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "asuca_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
}
KERNEL_STAGE, KERNEL_COLUMN, KERNEL_REDUCE, KERNEL_ADJ_STAGE, KERNEL_ADJ_COLUMN, KERNEL_ENSEMBLE = 0, 1, 2, 3, 4, 5
TUNE_COL_BLOCKS_PER_SM, TUNE_BARRIER_EXTRA, TUNE_STAGE_TILE_ROWS, TUNE_ENSEMBLE_TILE_ROWS, TUNE_STEP_MODE = 0, 1, 2, 3, 4
TUNE_FUSED_COLUMN = 5
KERNEL_DATAFLOW = 6
KERNEL_STAGE_COLUMN = 7
KERNEL_ACOUSTIC = 8
KERNEL_STAGE_FACTOR = 9
KERNEL_KINDS = 10


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libasuca.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libasuca.so is not built ({_LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def bounds_checked() -> bool:
    """Whether the loaded library is the bounds-check build (asuca_bounds_checked)."""
    return bool(lib().asuca_bounds_checked())


def _check(status: int, where: str):
    if status != OK:
        raise AsucaError(status, where)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Grid:
    """Grid, physics constants and precision (asuca_init_grid)."""

    def __init__(self, nx, ny, nz, ntracers, dz, dx=2000.0, dy=2000.0, *, tau_theta=3600.0,
                 k0=50.0, k_h=1000.0, v_sed=2.0, sed_tracer=None, lim=LIM_KOREN,
                 prec=FP32_MIXED):
        self.dz = np.ascontiguousarray(dz, dtype=np.float64)
        if sed_tracer is None:
            sed_tracer = ntracers - 1
        self.desc = GridDesc(nx, ny, nz, ntracers, dx, dy,
                             self.dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             tau_theta, k0, k_h, v_sed, sed_tracer, lim, prec)
        self.nx, self.ny, self.nz, self.ntracers = nx, ny, nz, ntracers
        self.dx, self.dy, self.prec = dx, dy, prec
        h = ctypes.c_void_p()
        _check(lib().asuca_init_grid(ctypes.byref(self.desc), ctypes.byref(h)), "asuca_init_grid")
        self.handle = h

    @classmethod
    def from_case(cls, case, **kw):
        return cls(case.nx, case.ny, case.nz, case.ntracers, case.dz, case.dx, case.dy, **kw)

    @property
    def nfields(self):
        return 2 + self.ntracers

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.prec == FP64 else torch.float32

    def workspace_bytes(self, op=OP_STEP, param=0) -> int:
        return int(lib().asuca_workspace_bytes(self.handle, op, param))

    def workspace(self, op=OP_STEP, param=0, device="cuda"):
        import torch
        n = self.workspace_bytes(op, param)
        return torch.empty(max(n, 256), dtype=torch.uint8, device=device)

    def close(self):
        if getattr(self, "handle", None):
            lib().asuca_free_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Caller-owned device fields: rho, rhotheta [nz][ny][nx], rhoq [N][nz][ny][nx],
    mu, mv [nz][ny][nx], mw [nz+1][ny][nx] (i fastest)."""

    def __init__(self, rho, rhotheta, rhoq, mu, mv, mw):
        self.rho, self.rhotheta, self.rhoq = rho, rhotheta, rhoq
        self.mu, self.mv, self.mw = mu, mv, mw

    @classmethod
    def from_case(cls, case, prec=FP32_MIXED, device="cuda"):
        import torch
        dt = torch.float64 if prec == FP64 else torch.float32
        t = lambda a: torch.as_tensor(np.require(a, requirements=['C', 'W'])).to(device=device, dtype=dt).contiguous()
        rhoq = case.rhoq if case.ntracers > 0 else np.zeros((0,) + case.rho.shape)
        return cls(t(case.rho), t(case.rhotheta), t(rhoq), t(case.mu), t(case.mv), t(case.mw))

    def clone(self):
        return State(self.rho.clone(), self.rhotheta.clone(), self.rhoq.clone(), self.mu, self.mv, self.mw)

    def fields(self):
        """[F][nz][ny][nx] stacked copy (rho, rho*theta, tracers)."""
        import torch
        return torch.cat([self.rho[None], self.rhotheta[None], self.rhoq], 0)

    def struct(self) -> StateStruct:
        ptr = lambda t: t.data_ptr() if t is not None and t.numel() else None
        return StateStruct(ptr(self.rho), ptr(self.rhotheta), ptr(self.rhoq), ptr(self.mu), ptr(self.mv),
                           ptr(self.mw))


def _check_state(grid: Grid, st: State):
    dt = grid.torch_dtype
    nz, ny, nx, N = grid.nz, grid.ny, grid.nx, grid.ntracers
    for name, shape in (("rho", (nz, ny, nx)), ("rhotheta", (nz, ny, nx)), ("rhoq", (N, nz, ny, nx)),
                        ("mu", (nz, ny, nx)), ("mv", (nz, ny, nx)), ("mw", (nz + 1, ny, nx))):
        t = getattr(st, name)
        if tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"state.{name}: need contiguous CUDA {dt} of shape {shape}, "
                             f"got {t.dtype} {tuple(t.shape)}")


def step(grid: Grid, state: State, dt: float, nsteps: int, *, tendencies=None, workspace=None,
         budgets=None, stream=None):
    """Advance `state` in place by nsteps (asuca_step).  Returns the budgets tensor
    (N+3 doubles on the device) if `budgets` is given or True."""
    import torch
    _check_state(grid, state)
    if tendencies is not None:
        shape = (grid.ntracers + 1, grid.nz, grid.ny, grid.nx)
        if tuple(tendencies.shape) != shape or tendencies.dtype != grid.torch_dtype or \
                not tendencies.is_contiguous():
            raise ValueError(f"tendencies: need contiguous {grid.torch_dtype} of shape {shape}")
    if workspace is None:
        workspace = grid.workspace(device=state.rho.device)
    if budgets is True:
        budgets = torch.empty(grid.nfields + 1, dtype=torch.float64, device=state.rho.device)
    s = state.struct()
    _check(lib().asuca_step(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt), int(nsteps),
                            _ptr(workspace), workspace.numel() * workspace.element_size(),
                            _ptr(budgets), _stream_ptr(stream)), "asuca_step")
    return budgets


# ---------------------------------------------------------------- open lateral boundaries

def _check_open_state(grid: Grid, st: State):
    """Fields as for step; mu, mv are the open domain's face fluxes
    [nz][ny][nx+1] and [nz][ny+1][nx] (entry i, j: face i-1/2, j-1/2)."""
    dt = grid.torch_dtype
    nz, ny, nx, N = grid.nz, grid.ny, grid.nx, grid.ntracers
    for name, shape in (("rho", (nz, ny, nx)), ("rhotheta", (nz, ny, nx)), ("rhoq", (N, nz, ny, nx)),
                        ("mu", (nz, ny, nx + 1)), ("mv", (nz, ny + 1, nx)), ("mw", (nz + 1, ny, nx))):
        t = getattr(st, name)
        if tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"open state.{name}: need contiguous CUDA {dt} of shape {shape}, "
                             f"got {t.dtype} {tuple(t.shape)}")


def _check_halo(grid: Grid, t, what):
    n = halo_count(grid)
    if t is None or t.numel() != n or t.dtype != grid.torch_dtype or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"{what}: need a contiguous CUDA {grid.torch_dtype} halo array of {n} values")


def open_workspace_bytes(grid: Grid) -> int:
    return int(lib().asuca_open_workspace_bytes(grid.handle))


def open_workspace(grid: Grid, device="cuda"):
    import torch
    return torch.empty(open_workspace_bytes(grid), dtype=torch.uint8, device=device)


def halo_count(grid: Grid) -> int:
    """values of one halo-layout array: 2 (2 nx + 2 ny) nz (F - 1)"""
    return int(lib().asuca_halo_count(grid.handle))


def open_prepare(grid: Grid, state: State, workspace, *, first: bool = True, stream=None):
    """Buffer 0's interior = phi of the state (asuca_open_prepare)."""
    _check_open_state(grid, state)
    s = state.struct()
    _check(lib().asuca_open_prepare(grid.handle, ctypes.byref(s), int(bool(first)), _ptr(workspace),
                                    workspace.numel(), _stream_ptr(stream)), "asuca_open_prepare")


def open_stage(grid: Grid, state: State, dt: float, stage: int, workspace, *, tendencies=None, budgets=None,
               stream=None):
    """RK stage 0, 1 or 2 of an open domain (asuca_open_stage); stage 2 runs the column pass."""
    _check_open_state(grid, state)
    s = state.struct()
    _check(lib().asuca_open_stage(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt), int(stage),
                                  _ptr(workspace), workspace.numel(), _ptr(budgets), _stream_ptr(stream)),
           "asuca_open_stage")
    return budgets


def halo_pack(grid: Grid, workspace, buffer: int, send, *, stream=None):
    _check_halo(grid, send, "send")
    _check(lib().asuca_halo_pack(grid.handle, _ptr(workspace), workspace.numel(), int(buffer), _ptr(send),
                                 _stream_ptr(stream)), "asuca_halo_pack")


def halo_unpack(grid: Grid, workspace, buffer: int, recv, *, bnd1=None, tratio: float = 0.0, stream=None):
    _check_halo(grid, recv, "recv")
    if bnd1 is not None:
        _check_halo(grid, bnd1, "bnd1")
    _check(lib().asuca_halo_unpack(grid.handle, _ptr(workspace), workspace.numel(), int(buffer), _ptr(recv),
                                   _ptr(bnd1), float(tratio), _stream_ptr(stream)), "asuca_halo_unpack")


def step_open(grid: Grid, state: State, dt: float, nsteps: int, bnd0, *, bnd1=None, tratio: float = 0.0,
              tendencies=None, workspace=None, budgets=None, stream=None):
    """nsteps steps of a limited-area domain (asuca_step_open): the ghosts of every
    stage are (1 - tratio) bnd0 + tratio bnd1 (bnd0 alone without bnd1)."""
    import torch
    _check_open_state(grid, state)
    _check_halo(grid, bnd0, "bnd0")
    if bnd1 is not None:
        _check_halo(grid, bnd1, "bnd1")
    if workspace is None:
        workspace = open_workspace(grid, device=state.rho.device)
    if budgets is True:
        budgets = torch.empty(grid.nfields + 1, dtype=torch.float64, device=state.rho.device)
    s = state.struct()
    _check(lib().asuca_step_open(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt), int(nsteps),
                                 _ptr(bnd0), _ptr(bnd1), float(tratio), _ptr(workspace), workspace.numel(),
                                 _ptr(budgets), _stream_ptr(stream)), "asuca_step_open")
    return budgets


def get_status(grid: Grid) -> int:
    return int(lib().asuca_get_status(grid.handle))


def debug_stage(grid: Grid, yin: State, ybase: State, yout: State, cdt: float, *, tendencies=None,
                stream=None):
    """One RK stage: yout = ybase + cdt * R(yin) (asuca_debug_stage)."""
    a, b, c = yin.struct(), ybase.struct(), yout.struct()
    _check(lib().asuca_debug_stage(grid.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                   _ptr(tendencies), float(cdt), _stream_ptr(stream)),
           "asuca_debug_stage")


def debug_column(grid: Grid, state: State, dt: float, precip_col, *, workspace=None, stream=None):
    """The column pass alone (asuca_debug_column); precip_col [ny][nx] float64 is incremented."""
    if workspace is None:
        workspace = grid.workspace(device=state.rho.device)
    s = state.struct()
    _check(lib().asuca_debug_column(grid.handle, ctypes.byref(s), float(dt), _ptr(precip_col),
                                    _ptr(workspace), workspace.numel(), _stream_ptr(stream)),
           "asuca_debug_column")


def debug_numerics(in_f, in_d, *, stream=None):
    """(widen(in_f), narrow(in_d), rcp(in_d)) computed by the library's column-solve helpers."""
    import torch
    n = in_f.numel()
    assert in_d.numel() == n and in_f.dtype == torch.float32 and in_d.dtype == torch.float64
    w = torch.empty(n, dtype=torch.float64, device=in_f.device)
    nr = torch.empty(n, dtype=torch.float32, device=in_f.device)
    r = torch.empty(n, dtype=torch.float64, device=in_f.device)
    _check(lib().asuca_debug_numerics(_ptr(in_f), _ptr(in_d), n, _ptr(w), _ptr(nr), _ptr(r),
                                      _stream_ptr(stream)), "asuca_debug_numerics")
    return w, nr, r


def column_noalloc(grid: Grid, state: State, dt: float, precip_col, *, stream=None):
    """The column pass without a workspace (asuca_column_noalloc): for callers that
    cannot allocate device memory; its scratch is an array compiled into the library."""
    s = state.struct()
    _check(lib().asuca_column_noalloc(grid.handle, ctypes.byref(s), float(dt), _ptr(precip_col),
                                      _stream_ptr(stream)), "asuca_column_noalloc")


LAYOUT_IJK, LAYOUT_KIJ = 0, 1


def stencil7(inp, out, c: float, layout: int = LAYOUT_IJK, *, stream=None):
    """One explicit 7-point diffusion step (asuca_stencil7): out = in + c (sum of
    the six neighbours - 6 in).  inp, out: contiguous CUDA tensors of nx ny nz
    float32 or float64 elements, [nz][ny][nx] for LAYOUT_IJK, [ny][nx][nz] for
    LAYOUT_KIJ; the shape gives (nx, ny, nz)."""
    import torch
    if inp.dtype not in (torch.float32, torch.float64) or out.dtype != inp.dtype or inp.shape != out.shape \
            or inp.dim() != 3 or not inp.is_contiguous() or not out.is_contiguous() or not inp.is_cuda:
        raise ValueError("stencil7: need two contiguous CUDA float tensors of the same 3D shape")
    if layout == LAYOUT_IJK:
        nz, ny, nx = inp.shape
    else:
        ny, nx, nz = inp.shape
    prec = FP64 if inp.dtype == torch.float64 else FP32_MIXED
    _check(lib().asuca_stencil7(_ptr(inp), _ptr(out), nx, ny, nz, int(layout), prec, float(c), _stream_ptr(stream)),
           "asuca_stencil7")
    return out


DAMP_MAX_WIDTH = 64


def damping(grid: Grid, state: State, ref, bnd0, bnd1, tratio: float, dt: float, *, width: int, ntop: int,
            nu_lat: float, nu_top: float, mtratio=None, stream=None):
    """Lateral and upper damping toward boundary data (asuca_damping), in place:
    target = ref + mtratio (ref + bnd0) + tratio (ref + bnd1) - ref, y relaxed
    implicitly toward it with rate nu in the zone of `width` edge cells and
    `ntop` top levels.  ref, bnd0, bnd1: contiguous CUDA [F][nz][ny][nx] tensors
    of the grid's dtype; mtratio defaults to 1 - tratio."""
    _check_state(grid, state)
    shape = (grid.nfields, grid.nz, grid.ny, grid.nx)
    for name, t in (("ref", ref), ("bnd0", bnd0), ("bnd1", bnd1)):
        if tuple(t.shape) != shape or t.dtype != grid.torch_dtype or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name}: need contiguous CUDA {grid.torch_dtype} of shape {shape}")
    if mtratio is None:
        mtratio = 1.0 - tratio
    d = DampingDesc(int(width), int(ntop), float(nu_lat), float(nu_top))
    s = state.struct()
    _check(lib().asuca_damping(grid.handle, ctypes.byref(s), _ptr(ref), _ptr(bnd0), _ptr(bnd1), float(mtratio),
                               float(tratio), float(dt), ctypes.byref(d), _stream_ptr(stream)), "asuca_damping")


def acoustic_workspace_bytes(grid: Grid) -> int:
    return int(lib().asuca_acoustic_workspace_bytes(grid.handle))


def acoustic_steps(grid: Grid, U, V, W, S, rho0c, rho0f, cs2: float, beta: float, dtau: float, nshort: int, *,
                   workspace=None, stream=None):
    """nshort HEVI acoustic short steps (asuca_acoustic_steps), in place.  U, V, S:
    contiguous CUDA [nz][ny][nx] tensors of the grid's dtype; W: [nz+1][ny][nx]
    (W[0], W[nz] rigid lids, untouched); rho0c (nz) and rho0f (nz+1): host arrays."""
    import torch
    nz, ny, nx = grid.nz, grid.ny, grid.nx
    for name, t, shape in (("U", U, (nz, ny, nx)), ("V", V, (nz, ny, nx)), ("W", W, (nz + 1, ny, nx)),
                           ("S", S, (nz, ny, nx))):
        if tuple(t.shape) != shape or t.dtype != grid.torch_dtype or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name}: need contiguous CUDA {grid.torch_dtype} of shape {shape}")
    r0c = np.ascontiguousarray(rho0c, dtype=np.float64)
    r0f = np.ascontiguousarray(rho0f, dtype=np.float64)
    if r0c.shape != (nz,) or r0f.shape != (nz + 1,):
        raise ValueError("rho0c: nz values, rho0f: nz + 1 values")
    if workspace is None:
        workspace = torch.empty(max(acoustic_workspace_bytes(grid), 256), dtype=torch.uint8, device=S.device)
    dp = ctypes.POINTER(ctypes.c_double)
    d = AcousticDesc(r0c.ctypes.data_as(dp), r0f.ctypes.data_as(dp), float(cs2), float(beta))
    _check(lib().asuca_acoustic_steps(grid.handle, _ptr(U), _ptr(V), _ptr(W), _ptr(S), ctypes.byref(d), float(dtau),
                                      int(nshort), _ptr(workspace), workspace.numel(), _stream_ptr(stream)),
           "asuca_acoustic_steps")


def hevi_workspace_bytes(grid: Grid) -> int:
    return int(lib().asuca_hevi_workspace_bytes(grid.handle))


def step_hevi(grid: Grid, state: State, dt: float, nsteps: int, rho0c, rho0f, cs2: float, beta: float, nshort: int,
              *, tendencies=None, s_final=None, workspace=None, budgets=None, stream=None):
    """nsteps long steps with the acoustic short steps nested in the RK3 stages
    (asuca_step_hevi): state.mu, mv, mw are the prognostic momenta U, V, W,
    updated in place with the scalars.  s_final, if given ([nz][ny][nx] of the
    grid's dtype), receives s of the last third-stage integration."""
    import torch
    _check_state(grid, state)
    if workspace is None:
        workspace = torch.empty(hevi_workspace_bytes(grid), dtype=torch.uint8, device=state.rho.device)
    if budgets is True:
        budgets = torch.empty(grid.nfields + 1, dtype=torch.float64, device=state.rho.device)
    r0c = np.ascontiguousarray(rho0c, dtype=np.float64)
    r0f = np.ascontiguousarray(rho0f, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    d = AcousticDesc(r0c.ctypes.data_as(dp), r0f.ctypes.data_as(dp), float(cs2), float(beta))
    s = state.struct()
    _check(lib().asuca_step_hevi(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt), int(nsteps),
                                 ctypes.byref(d), int(nshort), _ptr(s_final), _ptr(workspace), workspace.numel(),
                                 _ptr(budgets), _stream_ptr(stream)), "asuca_step_hevi")
    return budgets


def profile_enable(grid: Grid, on: bool = True):
    _check(lib().asuca_profile_enable(grid.handle, int(bool(on))), "asuca_profile_enable")


def profile_read(grid: Grid):
    """{kind: (total_ms, launches)} of the kernels launched since the last read."""
    ms = (ctypes.c_double * KERNEL_KINDS)()
    n = (ctypes.c_int * KERNEL_KINDS)()
    _check(lib().asuca_profile_read(grid.handle, ms, n, KERNEL_KINDS), "asuca_profile_read")
    return {k: (ms[k], n[k]) for k in range(KERNEL_KINDS) if n[k]}


# ---------------------------------------------------------------- adjoint

def adjoint_workspace_bytes(grid: Grid, nsteps: int, checkpoint_every: int = 10) -> int:
    return int(lib().asuca_adjoint_workspace_bytes(grid.handle, int(nsteps), int(checkpoint_every)))


def adjoint_step(grid: Grid, initial: State, dt: float, nsteps: int, lam_final, *, checkpoint_every: int = 10,
                 tendencies=None, workspace=None, stream=None):
    """Adjoint of nsteps steps (asuca_adjoint_step): lam_final = dJ/dY_final as a
    [F][nz][ny][nx] tensor; returns (dJ/dY_initial [F][nz][ny][nx], dJ/dmu,
    dJ/dmv, dJ/dmw).  `initial` is not modified."""
    import torch
    _check_state(grid, initial)
    F = grid.nfields
    shape = (F, grid.nz, grid.ny, grid.nx)
    if tuple(lam_final.shape) != shape or lam_final.dtype != grid.torch_dtype or not lam_final.is_contiguous():
        raise ValueError(f"lam_final: need contiguous {grid.torch_dtype} of shape {shape}")
    dev = initial.rho.device
    if workspace is None:
        n = adjoint_workspace_bytes(grid, nsteps, checkpoint_every)
        workspace = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
    g0 = torch.empty(shape, dtype=grid.torch_dtype, device=dev)
    gmu = torch.empty_like(initial.mu)
    gmv = torch.empty_like(initial.mv)
    gmw = torch.empty_like(initial.mw)
    s = initial.struct()
    _check(lib().asuca_adjoint_step(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt), int(nsteps),
                                    int(checkpoint_every), _ptr(lam_final), _ptr(g0), _ptr(gmu), _ptr(gmv),
                                    _ptr(gmw), _ptr(workspace), workspace.numel(), _stream_ptr(stream)),
           "asuca_adjoint_step")
    return g0, gmu, gmv, gmw


def checkpoint_bytes(grid: Grid, nsteps: int, checkpoint_every: int = 10) -> int:
    return int(lib().asuca_checkpoint_bytes(grid.handle, int(nsteps), int(checkpoint_every)))


def forward_checkpointed(grid: Grid, state: State, dt: float, nsteps: int, *, checkpoint_every: int = 10,
                         tendencies=None, workspace=None, checkpoints=None, budgets=None, stream=None):
    """asuca_forward_checkpointed: advance `state` in place by nsteps (as step())
    and return the uint8 checkpoint tensor (the state every checkpoint_every
    steps) that adjoint_from_checkpoints reverses from."""
    import torch
    _check_state(grid, state)
    dev = state.rho.device
    if workspace is None:
        workspace = grid.workspace(device=dev)
    n = checkpoint_bytes(grid, nsteps, checkpoint_every)
    if checkpoints is None:
        checkpoints = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
    if budgets is True:
        budgets = torch.empty(grid.nfields + 1, dtype=torch.float64, device=dev)
    s = state.struct()
    _check(lib().asuca_forward_checkpointed(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt), int(nsteps),
                                            int(checkpoint_every), _ptr(checkpoints), checkpoints.numel(),
                                            _ptr(workspace), workspace.numel(), _ptr(budgets), _stream_ptr(stream)),
           "asuca_forward_checkpointed")
    return checkpoints


def adjoint_from_checkpoints(grid: Grid, checkpoints, fluxes: State, dt: float, nsteps: int, lam_final, *,
                             checkpoint_every: int = 10, tendencies=None, workspace=None, stream=None):
    """asuca_adjoint_from_checkpoints: the adjoint_step result, reversing from
    the checkpoints forward_checkpointed kept (fluxes supplies mu, mv, mw)."""
    import torch
    F = grid.nfields
    shape = (F, grid.nz, grid.ny, grid.nx)
    if tuple(lam_final.shape) != shape or lam_final.dtype != grid.torch_dtype or not lam_final.is_contiguous():
        raise ValueError(f"lam_final: need contiguous {grid.torch_dtype} of shape {shape}")
    dev = fluxes.mu.device
    if workspace is None:
        n = adjoint_workspace_bytes(grid, nsteps, checkpoint_every)
        workspace = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
    g0 = torch.empty(shape, dtype=grid.torch_dtype, device=dev)
    gmu = torch.empty_like(fluxes.mu)
    gmv = torch.empty_like(fluxes.mv)
    gmw = torch.empty_like(fluxes.mw)
    s = fluxes.struct()
    _check(lib().asuca_adjoint_from_checkpoints(grid.handle, _ptr(checkpoints), ctypes.byref(s), _ptr(tendencies),
                                                float(dt), int(nsteps), int(checkpoint_every), _ptr(lam_final),
                                                _ptr(g0), _ptr(gmu), _ptr(gmv), _ptr(gmw), _ptr(workspace),
                                                workspace.numel(), _stream_ptr(stream)),
           "asuca_adjoint_from_checkpoints")
    return g0, gmu, gmv, gmw


def record_branches(grid: Grid, initial: State, dt: float, nsteps: int, *, tendencies=None, stream=None):
    """Limiter branch bytes [nsteps][3][F-1][nz][ny][nx] of a forward trajectory."""
    import torch
    dev = initial.rho.device
    out = torch.empty((nsteps, 3, grid.nfields - 1, grid.nz, grid.ny, grid.nx), dtype=torch.uint8, device=dev)
    n = adjoint_workspace_bytes(grid, 1, 1)
    ws = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
    s = initial.struct()
    _check(lib().asuca_debug_record_branches(grid.handle, ctypes.byref(s), _ptr(tendencies), float(dt),
                                             int(nsteps), _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream)),
           "asuca_debug_record_branches")
    return out


def _autograd_function():
    import torch

    class AdjointFn(torch.autograd.Function):
        """Y_final = step^nsteps(Y_initial; mu, mv, mw) with a hand-written adjoint.

        forward(rho0, rhotheta0, rhoq0, mu, mv, mw, grid, dt, nsteps, checkpoint_every)
        -> (rho, rhotheta, rhoq) after nsteps steps.  The forward pass keeps the
        state every checkpoint_every steps (asuca_forward_checkpointed); backward
        runs asuca_adjoint_from_checkpoints, which recomputes each segment from
        its checkpoint and reverses it."""

        @staticmethod
        def forward(ctx, rho0, rhotheta0, rhoq0, mu, mv, mw, grid, dt, nsteps, checkpoint_every=10):
            st = State(rho0.detach().clone().contiguous(), rhotheta0.detach().clone().contiguous(),
                       rhoq0.detach().clone().contiguous(), mu.detach().contiguous(), mv.detach().contiguous(),
                       mw.detach().contiguous())
            ckpt = forward_checkpointed(grid, st, dt, nsteps, checkpoint_every=checkpoint_every)
            ctx.save_for_backward(mu, mv, mw, ckpt)
            ctx.grid, ctx.dt, ctx.nsteps, ctx.k = grid, dt, nsteps, checkpoint_every
            ctx.like = [(t.shape, t.dtype, t.device) for t in (rho0, rhotheta0, rhoq0)]
            return st.rho, st.rhotheta, st.rhoq

        @staticmethod
        def backward(ctx, g_rho, g_rt, g_q):
            mu, mv, mw, ckpt = ctx.saved_tensors
            grid = ctx.grid
            z = lambda t, like: torch.zeros(like[0], dtype=like[1], device=like[2]) if t is None else t
            lam = torch.cat([z(g_rho, ctx.like[0])[None], z(g_rt, ctx.like[1])[None], z(g_q, ctx.like[2])],
                            0).contiguous()
            fl = State(None, None, None, mu.detach().contiguous(), mv.detach().contiguous(), mw.detach().contiguous())
            g0, gmu, gmv, gmw = adjoint_from_checkpoints(grid, ckpt, fl, ctx.dt, ctx.nsteps,
                                                         lam.to(grid.torch_dtype), checkpoint_every=ctx.k)
            return g0[0], g0[1], g0[2:], gmu, gmv, gmw, None, None, None, None

    return AdjointFn


_ADJOINT_FN = None


def __getattr__(name):
    global _ADJOINT_FN
    if name == "AdjointFn":
        if _ADJOINT_FN is None:
            _ADJOINT_FN = _autograd_function()
        return _ADJOINT_FN
    raise AttributeError(name)


# ---------------------------------------------------------------- ensemble and tuning

def set_tuning(grid: Grid, key: int, value: int):
    _check(lib().asuca_set_tuning(grid.handle, int(key), int(value)), "asuca_set_tuning")


def get_tuning(grid: Grid, key: int) -> int:
    return int(lib().asuca_get_tuning(grid.handle, int(key)))


def _grid_array(grids):
    arr = (_VP * len(grids))()
    for m, g in enumerate(grids):
        arr[m] = g.handle.value if isinstance(g.handle, ctypes.c_void_p) else g.handle
    return arr


def ensemble_workspace_bytes(grids) -> int:
    return int(lib().asuca_ensemble_workspace_bytes(_grid_array(grids), len(grids)))


_side_streams = {}


def ensemble_step(grids, states, dts, nsteps: int, *, workspace=None, budgets=None, stream=None):
    """Advance every member by nsteps in one persistent launch (asuca_ensemble_step).
    Without an explicit stream the call runs on a side stream ordered after the
    current stream, so that its launch sequence can be captured into (and later
    replayed from) a CUDA graph.  Returns the budgets tensor [M][N+3] if asked."""
    import torch
    M = len(grids)
    assert len(states) == M and len(dts) == M and M > 0
    for g, st in zip(grids, states):
        _check_state(g, st)
    dev = states[0].rho.device
    if workspace is None:
        n = ensemble_workspace_bytes(grids)
        if n == 0:
            raise AsucaError(ERR_CUDA, "asuca_ensemble_workspace_bytes")
        workspace = torch.empty(n, dtype=torch.uint8, device=dev)
    if budgets is True:
        budgets = torch.empty((M, grids[0].nfields + 1), dtype=torch.float64, device=dev)
    sts = (StateStruct * M)(*[st.struct() for st in states])
    dd = (ctypes.c_double * M)(*[float(x) for x in dts])
    cur = torch.cuda.current_stream(dev)
    run = stream
    if run is None:
        run = _side_streams.get(dev.index)
        if run is None:
            run = _side_streams[dev.index] = torch.cuda.Stream(device=dev)
        run.wait_stream(cur)
    _check(lib().asuca_ensemble_step(_grid_array(grids), sts, dd, M, int(nsteps), _ptr(workspace),
                                     workspace.numel(), _ptr(budgets), ctypes.c_void_p(run.cuda_stream)),
           "asuca_ensemble_step")
    if stream is None:
        cur.wait_stream(run)
        workspace.record_stream(run)
    return budgets
