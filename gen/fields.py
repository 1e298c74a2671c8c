"""Seeded synthetic fields with the structure of the paper's workload.

The paper ran ASUCA on real JMA data (Sec. 4, "Productivity- and Performance
Results"): a rectangular grid with 2 km spacing and 58 levels (Sec. 1.1,
"ASUCA on GPU").  That data is not available, so these generators build
stand-ins of the same shape:

* dz stretched geometrically from 40 m to 1 km, dx = dy = 2 km;
* rho0(z) = 1.2 exp(-z / 8000) kg/m^3, horizontally uniform;
* theta = 300 + 0.004 z K plus four Gaussian bubbles of +-2 K;
* tracer mixing ratios from four Gaussian blobs each, in [0, 0.02];
* horizontally non-divergent C-grid mass fluxes MU, MV from an 8-mode sine
  streamfunction scaled to max |u|, |v| = 20 m/s, plus one x-z overturning
  mode (max 2 m/s) whose vertical mass flux MW follows from discrete
  continuity, so the 3D mass divergence is zero up to rounding;
* dt from a Courant number of 0.8;
* for the damping: a level-mean reference state and two boundary datasets
  (the state's deviation from it, the second one shifted, both with 1%
  noise);
* for the acoustic short steps: a base density rho_s exp(-g z / c^2) and
  perturbations taken from the case (s from the theta bubbles, momenta
  from 5% of the mass fluxes).

Array layout (all C order, i fastest):
  rho, rhotheta : [nz][ny][nx]
  rhoq          : [ntracers][nz][ny][nx]
  mu            : [nz][ny][nx], mu[k, j, i] is the flux through face i+1/2
  mv            : [nz][ny][nx], mv[k, j, i] is the flux through face j+1/2
  mw            : [nz+1][ny][nx], mw[k, j, i] is the flux through the face
                  below cell k (mw[0] and mw[nz] are the rigid lids, zero).

Nothing here is arithmetic of the time step; the same arrays feed the FP64
oracle and the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 171008616
DX = 2000.0
DY = 2000.0
COURANT = 0.8
UMAX = 20.0          # max |u|, |v| of the streamfunction winds (m/s)
OVERTURN_DU = 2.0    # max |du| of the x-z overturning mode (m/s)

# Workloads by what they are; "index" offsets the seed.
CONFIGS = {
    "fp64_32x32x16": dict(index=0, nx=32, ny=32, nz=16, ntracers=3, nsteps=20),
    "precision_256x256x58": dict(index=1, nx=256, ny=256, nz=58, ntracers=6, nsteps=100),
    "adjoint_128x128x58": dict(index=2, nx=128, ny=128, nz=58, ntracers=4, nsteps=50),
    "ensemble_32x_64to320x58": dict(index=3, members=32, nmin=64, nmax=320, nz=58,
                                    ntracers=4, nsteps=100),
    "large_1024x1024x58": dict(index=4, nx=1024, ny=1024, nz=58, ntracers=8, nsteps=200),
}


@dataclass
class Case:
    nx: int
    ny: int
    nz: int
    ntracers: int
    dx: float
    dy: float
    dz: np.ndarray
    rho: np.ndarray
    rhotheta: np.ndarray
    rhoq: np.ndarray
    mu: np.ndarray
    mv: np.ndarray
    mw: np.ndarray
    dt: float
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def nfields(self) -> int:
        return 2 + self.ntracers

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def state(self) -> np.ndarray:
        """All prognostic fields stacked as [F][nz][ny][nx]: rho, rho*theta, rho*q_1..N."""
        return np.concatenate([self.rho[None], self.rhotheta[None], self.rhoq], axis=0)


def make_dz(nz: int) -> np.ndarray:
    """Geometric stretching, 40 m at the ground to 1 km at the top level."""
    if nz < 2:
        return np.full(nz, 40.0)
    k = np.arange(nz, dtype=np.float64)
    return 40.0 * 25.0 ** (k / (nz - 1))


def _levels(dz: np.ndarray):
    zf = np.concatenate([[0.0], np.cumsum(dz)])     # faces, zf[k] below cell k
    zc = zf[:-1] + 0.5 * dz                          # cell centres
    return zf, zc


def _rho0(z):
    return 1.2 * np.exp(-np.asarray(z) / 8000.0)


def _draw_pattern(rng: np.random.Generator, ntracers: int) -> dict:
    """Shape parameters in domain-relative coordinates; the draw order is fixed."""
    p = {}
    p["bub_c"] = np.stack([rng.uniform(0, 1, 4), rng.uniform(0, 1, 4), rng.uniform(0, 0.5, 4)], 1)
    p["bub_a"] = rng.uniform(-2.0, 2.0, 4)
    blobs = []
    for _ in range(ntracers):
        c = np.stack([rng.uniform(0, 1, 4), rng.uniform(0, 1, 4), rng.uniform(0, 0.5, 4)], 1)
        a = rng.uniform(0.0, 1.0, 4)
        blobs.append((c, a))
    p["blobs"] = blobs
    modes = []
    while len(modes) < 8:
        kx, ky = int(rng.integers(-3, 4)), int(rng.integers(-3, 4))
        if kx == 0 and ky == 0:
            continue
        modes.append((kx, ky, rng.uniform(0.5, 1.0), rng.uniform(0, 2 * math.pi)))
    p["modes"] = modes
    p["ot_phase"] = rng.uniform(0, 2 * math.pi)
    return p


def _periodic_offset(x, c, L):
    d = x - c
    return d - L * np.round(d / L)


def _gauss_sep(nx, ny, nz, dx, dy, zc, H, centre):
    """exp(-r^2) on cell centres as a separable product; minimum-image in x, y."""
    Lx, Ly = nx * dx, ny * dy
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    ex = np.exp(-(_periodic_offset(x, centre[0] * Lx, Lx) / (Lx / 8)) ** 2)
    ey = np.exp(-(_periodic_offset(y, centre[1] * Ly, Ly) / (Ly / 8)) ** 2)
    ez = np.exp(-((zc - centre[2] * H) / (H / 8)) ** 2)
    return ez[:, None, None] * ey[None, :, None] * ex[None, None, :]


def _streamfunction(nx, ny, dx, dy, modes):
    """psi at cell corners (i+1/2, j+1/2) -> array [ny][nx]."""
    Lx, Ly = nx * dx, ny * dy
    xc = (np.arange(nx) + 1.0) * dx
    yc = (np.arange(ny) + 1.0) * dy
    psi = np.zeros((ny, nx))
    for kx, ky, a, ph in modes:
        psi += a * np.sin(2 * math.pi * (kx * xc[None, :] / Lx + ky * yc[:, None] / Ly) + ph)
    return psi


def _winds_from_psi(psi, dx, dy):
    """u at faces i+1/2 and v at faces j+1/2 (per unit density) from corner psi."""
    u = -(psi - np.roll(psi, 1, axis=0)) / dy
    v = (psi - np.roll(psi, 1, axis=1)) / dx
    return u, v


def make_case(nx: int, ny: int, nz: int, ntracers: int, seed: int, *,
              overturning: bool = True, pattern_seed: int | None = None,
              perturb_seed: int | None = None, smooth_tracers: bool = False,
              dx: float = DX, dy: float = DY, dtype=np.float64) -> Case:
    """Build one seeded case (horizontal spacing dx, dy; 2 km by default).

    pattern_seed draws the bubble/blob/mode parameters (domain-relative, so
    domains of different sizes share a pattern); perturb_seed, when given, adds
    an ensemble member's perturbation: one more bubble set of +-0.5 K and one
    more streamfunction mode scaled to max 1 m/s.
    """
    if nx < 1 or ny < 1 or nz < 1 or ntracers < 0:
        raise ValueError("bad grid size")
    rng = np.random.default_rng(seed if pattern_seed is None else pattern_seed)
    pat = _draw_pattern(rng, ntracers)
    dx, dy = float(dx), float(dy)
    dz = make_dz(nz)
    zf, zc = _levels(dz)
    H = zf[-1]
    rho0c = _rho0(zc)

    theta = np.broadcast_to((300.0 + 0.004 * zc)[:, None, None], (nz, ny, nx)).copy()
    for b in range(4):
        theta += pat["bub_a"][b] * _gauss_sep(nx, ny, nz, dx, dy, zc, H, pat["bub_c"][b])
    q = np.zeros((ntracers, nz, ny, nx))
    for n, (c, a) in enumerate(pat["blobs"]):
        acc = np.zeros((nz, ny, nx))
        for b in range(4):
            np.maximum(acc, a[b] * _gauss_sep(nx, ny, nz, dx, dy, zc, H, c[b]), out=acc)
        q[n] = 0.02 * acc

    if smooth_tracers and ntracers > 0:
        srng = np.random.default_rng(seed + 77)
        x = (np.arange(nx) + 0.5) / nx
        y = (np.arange(ny) + 0.5) / ny
        zz = zc / H
        for n in range(ntracers):
            acc = np.zeros((nz, ny, nx))
            for _ in range(3):
                kx, ky = int(srng.integers(1, 3)), int(srng.integers(1, 3))
                kz = srng.uniform(0.5, 1.5)
                ph = srng.uniform(0, 2 * math.pi, 3)
                acc += (np.sin(2 * math.pi * kx * x + ph[0])[None, None, :] *
                        np.sin(2 * math.pi * ky * y + ph[1])[None, :, None] *
                        np.sin(math.pi * kz * zz + ph[2])[:, None, None])
            q[n] = 0.0125 + 0.0075 * acc / 3.0

    psi = _streamfunction(nx, ny, dx, dy, pat["modes"])
    u, v = _winds_from_psi(psi, dx, dy)
    s = UMAX / max(np.abs(u).max(), np.abs(v).max())
    u *= s
    v *= s

    if perturb_seed is not None:
        prng = np.random.default_rng(perturb_seed)
        pc = np.stack([prng.uniform(0, 1, 4), prng.uniform(0, 1, 4), prng.uniform(0, 0.5, 4)], 1)
        pa = prng.uniform(-0.5, 0.5, 4)
        for b in range(4):
            theta += pa[b] * _gauss_sep(nx, ny, nz, dx, dy, zc, H, pc[b])
        while True:
            kx, ky = int(prng.integers(-3, 4)), int(prng.integers(-3, 4))
            if kx or ky:
                break
        ppsi = _streamfunction(nx, ny, dx, dy, [(kx, ky, 1.0, prng.uniform(0, 2 * math.pi))])
        pu, pv = _winds_from_psi(ppsi, dx, dy)
        ps = 1.0 / max(np.abs(pu).max(), np.abs(pv).max(), 1e-300)
        u += ps * pu
        v += ps * pv

    mu = rho0c[:, None, None] * u[None, :, :]
    mv = rho0c[:, None, None] * v[None, :, :]
    mu = np.ascontiguousarray(np.broadcast_to(mu, (nz, ny, nx)))
    mv = np.ascontiguousarray(np.broadcast_to(mv, (nz, ny, nx)))

    mw = np.zeros((nz + 1, ny, nx))
    if overturning and nz >= 2:
        # mass streamfunction Phi at (i+1/2, k+1/2) edges, zero on both lids;
        # a whole number of wavelengths near 32 dx keeps it periodic.
        waves = max(1, int(round(nx / 32.0)))
        lam = nx * dx / waves
        xe = (np.arange(nx) + 1.0) * dx
        phi = np.sin(2 * math.pi * xe / lam + pat["ot_phase"])[None, :] * \
            np.sin(math.pi * zf / H)[:, None]
        phi[0] = 0.0
        phi[-1] = 0.0
        dmu = -(phi[1:] - phi[:-1]) / dz[:, None]              # [nz][nx]
        amp = OVERTURN_DU / np.abs(dmu / rho0c[:, None]).max()
        mu = mu + amp * dmu[:, None, :]
        # discrete continuity, bottom-up from the lower lid
        div_h = (mu - np.roll(mu, 1, axis=2)) / dx + (mv - np.roll(mv, 1, axis=1)) / dy
        for k in range(nz):
            mw[k + 1] = mw[k] - dz[k] * div_h[k]
        mw[nz] = 0.0
    rho = np.ascontiguousarray(np.broadcast_to(rho0c[:, None, None], (nz, ny, nx)))

    umax = np.abs(mu / rho0c[:, None, None]).max()
    vmax = np.abs(mv / rho0c[:, None, None]).max()
    wmax = 0.0
    for kf in range(1, nz):
        w = np.abs(mw[kf]).max() / _rho0(zf[kf]) / min(dz[kf - 1], dz[kf])
        wmax = max(wmax, w)
    dt = COURANT / (umax / dx + vmax / dy + wmax)

    cast = (lambda a: np.ascontiguousarray(a, dtype=dtype))
    return Case(nx=nx, ny=ny, nz=nz, ntracers=ntracers, dx=dx, dy=dy, dz=dz,
                rho=cast(rho), rhotheta=cast(rho * theta), rhoq=cast(rho[None] * q),
                mu=cast(mu), mv=cast(mv), mw=cast(mw), dt=float(dt), seed=seed,
                meta=dict(umax=float(umax), vmax=float(vmax), wmax_over_dz=float(wmax),
                          top=float(H)))


def make_config_case(name: str, *, dtype=np.float64, nx=None, ny=None, nz=None,
                     ntracers=None, overturning=True) -> Case:
    """The named workload's fields; sizes may be overridden for scaled-down tests."""
    c = CONFIGS[name]
    if "members" in c:
        raise ValueError("use make_ensemble_cases for the ensemble workload")
    return make_case(nx or c["nx"], ny or c["ny"], nz or c["nz"],
                     c["ntracers"] if ntracers is None else ntracers,
                     SEED_BASE + c["index"], overturning=overturning, dtype=dtype)


def ensemble_sizes(members: int | None = None, nmin: int | None = None,
                   nmax: int | None = None) -> list[int]:
    c = CONFIGS["ensemble_32x_64to320x58"]
    rng = np.random.default_rng(SEED_BASE + c["index"])
    return [int(v) for v in rng.integers(nmin or c["nmin"], (nmax or c["nmax"]) + 1,
                                         members or c["members"])]


def make_ensemble_cases(members: int | None = None, *, sizes=None, nz=None, ntracers=None,
                        dtype=np.float64) -> list[Case]:
    """Uneven ensemble: member m has nx = ny drawn from U{64..320} and its own
    perturbation seeded with SEED_BASE + index + 1000 (m + 1)."""
    c = CONFIGS["ensemble_32x_64to320x58"]
    seed = SEED_BASE + c["index"]
    if sizes is None:
        sizes = ensemble_sizes(members)
    out = []
    for m, n in enumerate(sizes):
        out.append(make_case(n, n, nz or c["nz"], c["ntracers"] if ntracers is None else ntracers,
                             seed + 1000 * (m + 1), pattern_seed=seed,
                             perturb_seed=seed + 1000 * (m + 1), dtype=dtype))
    return out


# Damping zone of the limited-area workloads: 16 edge cells (32 km), the top 8
# levels, relaxation times of 5 and 10 minutes, a quarter into the boundary interval.
DAMPING = dict(width=16, ntop=8, nu_lat=1.0 / 300.0, nu_top=1.0 / 600.0, tratio=0.25)


def make_boundary_data(Y: np.ndarray, seed: int, *, dtype=np.float64):
    """Reference state and two boundary datasets for a [F][nz][ny][nx] state Y:
    ref = the level mean of each field (horizontally uniform, like a reference
    atmosphere); bnd0 = Y - ref plus 1% noise (the perturbation at the start of
    the boundary interval); bnd1 = bnd0 shifted by three cells in i and one in j
    plus fresh noise (the perturbation moved on by the end of the interval).
    Returns (ref, bnd0, bnd1), each [F][nz][ny][nx] of dtype."""
    rng = np.random.default_rng(seed)
    Y = np.asarray(Y)
    ref = np.broadcast_to(Y.mean(axis=(2, 3), dtype=np.float64)[:, :, None, None], Y.shape).astype(dtype)
    dev = Y.astype(dtype) - ref
    scale = (0.01 * np.abs(ref[:, :, :1, :1])).astype(dtype)      # 1% of each field's level mean
    b0 = dev + scale * rng.standard_normal(Y.shape, dtype=np.float32).astype(dtype)
    b1 = np.roll(dev, (1, 3), axis=(2, 3)) + scale * rng.standard_normal(Y.shape, dtype=np.float32).astype(dtype)
    return np.ascontiguousarray(ref), np.ascontiguousarray(b0), np.ascontiguousarray(b1)


# Acoustic short steps: sound speed 340 m/s, off-centred implicit weight 0.6,
# 2 s short steps (horizontal acoustic Courant number 0.34 at 2 km), six short
# steps per call.
ACOUSTIC = dict(cs2=340.0 ** 2, beta=0.6, dtau=2.0, nshort=6, g=9.81, rho_s=1.2)


def make_acoustic_state(case: Case, *, dtype=np.float64):
    """Inputs of the acoustic short steps on a case's grid: the base density
    rho0 = rho_s exp(-g z / c^2) at level centres and faces (a base state in
    hydrostatic balance with p0 = c^2 rho0), and perturbations taken from the
    case: s = rho'/rho0 = 5e-4 (theta - theta_ref) from its theta bubbles
    (|s| <= 1e-3), momenta U, V, W = 0.05 MU, MV, MW (|u'| about 1 m/s).
    Returns (U, V, W, S, rho0c, rho0f)."""
    A = ACOUSTIC
    dz = np.asarray(case.dz, dtype=np.float64)
    zf = np.concatenate([[0.0], np.cumsum(dz)])
    zc = zf[:-1] + 0.5 * dz
    rho0c = A["rho_s"] * np.exp(-A["g"] * zc / A["cs2"])
    rho0f = A["rho_s"] * np.exp(-A["g"] * zf / A["cs2"])
    theta = np.asarray(case.rhotheta, np.float64) / np.asarray(case.rho, np.float64)
    S = 5e-4 * (theta - (300.0 + 0.004 * zc)[:, None, None])
    cast = (lambda a: np.ascontiguousarray(a, dtype=dtype))
    return (cast(0.05 * np.asarray(case.mu)), cast(0.05 * np.asarray(case.mv)), cast(0.05 * np.asarray(case.mw)),
            cast(S), rho0c, rho0f)


HEVI = dict(dt=12.0, nshort=6)   # long step and short steps of the coupled workload (h = 2 s)


def make_hevi_state(case: Case, *, dtype=np.float64):
    """Inputs of the long step with nested acoustic short steps on a case's grid:
    the acoustic base state of make_acoustic_state, the density
    rho = rho0 (1 + s) with s = 5e-4 (theta - theta_ref) (|s| <= 1e-3), the
    case's theta and mixing ratios carried by that density, and the case's
    mass fluxes as the initial momenta U, V, W.  A 12 s long step of six 2 s
    short steps keeps the horizontal acoustic Courant number at 0.34.
    Returns (Y [F][nz][ny][nx], U, V, W, rho0c, rho0f, dt, nshort)."""
    _, _, _, S, rho0c, rho0f = make_acoustic_state(case)
    rho_case = np.asarray(case.rho, np.float64)
    theta = np.asarray(case.rhotheta, np.float64) / rho_case
    q = np.asarray(case.rhoq, np.float64) / rho_case[None]
    rho = rho0c[:, None, None] * (1.0 + S)
    Y = np.concatenate([rho[None], (rho * theta)[None], rho[None] * q])
    cast = (lambda a: np.ascontiguousarray(a, dtype=dtype))
    return (cast(Y), cast(case.mu), cast(case.mv), cast(case.mw), rho0c, rho0f, HEVI["dt"], HEVI["nshort"])


# ---------------------------------------------------------------- open lateral boundaries
#
# Halo layout of the ghost cells of an open domain (limited-area or one block
# of a decomposed domain): four strips one after another,
#   W: i = c - 2,  E: i = nx + c  (c = 0, 1; every j), each [T][nz][2][ny]
#   S: j = c - 2,  N: j = ny + c  (c = 0, 1; every i), each [T][nz][2][nx]
# for T fields.  Face mass fluxes of an open domain: mu_x [nz][ny][nx+1] and
# mv_x [nz][ny+1][nx], index i (j) holding face i-1/2 (j-1/2).

def halo_periodic(fields: np.ndarray) -> np.ndarray:
    """The halo-layout ghosts of [T][nz][ny][nx] values continued periodically."""
    f = np.asarray(fields)
    nx, ny = f.shape[3], f.shape[2]
    w = np.stack([f[..., :, nx - 2], f[..., :, nx - 1]], axis=2)      # [T][nz][2][ny]
    e = np.stack([f[..., :, 0], f[..., :, 1]], axis=2)
    s = np.stack([f[..., ny - 2, :], f[..., ny - 1, :]], axis=2)      # [T][nz][2][nx]
    n = np.stack([f[..., 0, :], f[..., 1, :]], axis=2)
    return np.concatenate([a.reshape(-1) for a in (w, e, s, n)])


def halo_strips(halo: np.ndarray, T: int, nz: int, ny: int, nx: int):
    """(W, E, S, N) views of a halo-layout array: [T][nz][2][ny] twice, then [T][nz][2][nx] twice."""
    sw, ss = T * nz * 2 * ny, T * nz * 2 * nx
    h = np.asarray(halo).reshape(-1)
    return (h[:sw].reshape(T, nz, 2, ny), h[sw:2 * sw].reshape(T, nz, 2, ny),
            h[2 * sw:2 * sw + ss].reshape(T, nz, 2, nx), h[2 * sw + ss:].reshape(T, nz, 2, nx))


def extend_fluxes(mu: np.ndarray, mv: np.ndarray):
    """Open-domain face fluxes (mu_x, mv_x) of periodic ones: face -1/2 is face nx-1/2."""
    mu_x = np.concatenate([mu[:, :, -1:], mu], axis=2)
    mv_x = np.concatenate([mv[:, -1:, :], mv], axis=1)
    return np.ascontiguousarray(mu_x), np.ascontiguousarray(mv_x)


def split_extent(n: int, parts: int) -> list[tuple[int, int]]:
    """[start, stop) of each of `parts` blocks of n cells, sizes differing by at most 1."""
    if parts < 1 or parts > n:
        raise ValueError("bad block count")
    base, extra = divmod(n, parts)
    out, s = [], 0
    for p in range(parts):
        e = s + base + (1 if p < extra else 0)
        out.append((s, e))
        s = e
    return out


def subdomain(case: Case, px: int, py: int, rx: int, ry: int) -> dict:
    """Block (rx, ry) of a px x py decomposition of a periodic case: its state
    [F][nz][h][w], its open-domain face fluxes (the faces on its low edges
    taken from the neighbouring block, periodically) and mw."""
    (i0, i1), (j0, j1) = split_extent(case.nx, px)[rx], split_extent(case.ny, py)[ry]
    Y = case.state()[:, :, j0:j1, i0:i1]
    ii = np.arange(i0 - 1, i1) % case.nx
    jj = np.arange(j0 - 1, j1) % case.ny
    mu_x = case.mu[:, j0:j1, :][:, :, ii]
    mv_x = case.mv[:, :, i0:i1][:, jj, :]
    mw = case.mw[:, j0:j1, i0:i1]
    c = lambda a: np.ascontiguousarray(a)
    return dict(i0=i0, i1=i1, j0=j0, j1=j1, nx=i1 - i0, ny=j1 - j0, Y=c(Y), mu_x=c(mu_x), mv_x=c(mv_x),
                mw=c(mw))


def make_open_boundary(case: Case, seed: int, *, dtype=np.float64):
    """Two boundary datasets of a limited-area domain in the halo layout, for
    the F-1 transported quantities (theta and the mixing ratios): the case's
    own values continued periodically past its edges (so that the boundary
    joins the interior smoothly), with 1% noise, the second one shifted by
    one cell in i and with fresh noise (a later time of the outer model)."""
    rng = np.random.default_rng(seed)
    phi = case.state()[1:] / case.state()[0][None]
    h0 = halo_periodic(phi)
    h1 = halo_periodic(np.roll(phi, 1, axis=3))
    scale = np.abs(phi).reshape(phi.shape[0], -1).max(axis=1)
    T = phi.shape[0]

    def noisy(h):
        out = []
        for a in halo_strips(h, T, case.nz, case.ny, case.nx):
            out.append((a + 0.01 * scale[:, None, None, None] * rng.standard_normal(a.shape)).reshape(-1))
        return np.concatenate(out)

    return np.ascontiguousarray(noisy(h0), dtype=dtype), np.ascontiguousarray(noisy(h1), dtype=dtype)
