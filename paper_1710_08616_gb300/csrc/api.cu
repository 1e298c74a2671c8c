// Host side of the C ABI declared in include/asuca.h: argument checks,
// level tables, workspace layout and the launch sequence of one call.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <new>
#include <cstdlib>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "adjoint_params.cuh"
#include "ensemble_params.cuh"
#include "dataflow_params.cuh"
#include "damping.cuh"
#include "acoustic.cuh"
#include "common.cuh"
#include "open.cuh"

using namespace asuca;

struct asuca_grid {
    asuca_grid_desc d;
    double dz[MAXNZ], zf[MAXNZ + 1], zc[MAXNZ];
    int F;
    long long plane, cells;
    int device, nsm;
    int col_grid;                 // persistent column-kernel grid
    int col_blocks_per_sm;        // tuning knob behind col_grid
    int barrier_extra;            // test hook: extra arrivals the ensemble barrier waits for
    int stage_ty;                 // tile rows of the stage kernel (tuned; 8 for FP64)
    int step_mode;                // 0: one launch per stage and column pass; 1: persistent dataflow kernel
    int fused_col;                // step mode 0: stage 3 fused with the top-down column pass (1) or not (0)
    int df_grid;                  // co-resident CTAs of the dataflow kernel (0 until queried)
    unsigned *df_order_host[2];   // pinned wave-order tables: a full chunk and the remainder chunk
    int df_order_q[2];
    int ens_ty;                   // tile rows of the ensemble kernel (tuned; 8 for FP64)
    std::vector<void *> *kept_pinned;   // parameter buffers referenced by a caller's captured graphs
    volatile int *status_host;    // pinned, mapped; the device writes error codes here
    int *status_dev;
    cudaStream_t last_stream;
    // TMA descriptors of the two padded stage buffers, for the workspace they were made for
    void *map_ws;
    int map_ty;
    CUtensorMap map_ystar, map_ystar2;
    const void *umap_key[3];      // caller fields the cached user maps describe (rho, rho theta, rho q)
    int umap_ty, umap_ok;
    CUtensorMap umap[3];
    // TMA descriptors of the open domain's three padded stage inputs, for the workspace they were made for
    void *omap_ws;
    int omap_ty;
    CUtensorMap omap[3];
    // opt-in per-kernel timing: events recorded around every launch
    bool prof_on;
    cudaEvent_t *prof_ev;
    int prof_cap, prof_used;
    int *prof_kind;               // kind of the launch bracketed by events 2q, 2q+1
    // the adjoint's second stream (the recomputation of the next segment runs on it
    // while the caller's stream reverses the current one) and its events: fork, join,
    // segment recomputed (two buffer sets), segment reversed (two buffer sets)
    cudaStream_t aux_stream;
    cudaEvent_t aux_ev[6];
};

namespace {

// A named range on the host timeline of a profiler (NVTX; free when no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

constexpr size_t ALIGN = 256;
// column-kernel blocks resident per SM; the Thomas scratch is sized to match
int col_blocks_per_sm() {
    const char *e = std::getenv("ASUCA_COL_BLOCKS_PER_SM");
    const int v = e ? std::atoi(e) : 0;
    return v > 0 ? v : 3;
}

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

void set_col_grid(asuca_grid *g) {
    long long need = (g->plane + COL_TPB - 1) / COL_TPB;
    long long cap = (long long)g->nsm * g->col_blocks_per_sm;
    g->col_grid = (int)(need < cap ? need : cap);
}

size_t elem_size(const asuca_grid *g) { return g->d.prec == ASUCA_FP64 ? 8 : 4; }

long long col_slots(const asuca_grid *g) { return (long long)g->col_grid * COL_TPB; }

struct StepLayout {
    size_t ystar, ystar2, precip, partials, scratch, fscratch, falpha, df_order, df_counter, df_flags, df_partials, df_scratch,
        total;
};

// the fused stage-3/column path is taken (step mode 0, diffusion on, not disabled)
// (with 8-row stage tiles: the fused kernel is built for those, and the stage
// buffers' tensor maps follow the tuned tile height)
bool fused_path(const asuca_grid *g) {
    return g->step_mode == 0 && g->fused_col && g->d.k0 > 0.0 && g->stage_ty == 8;
}

constexpr int DF_CHUNK = 16;   // steps per dataflow launch

int df_tiles_x(const asuca_grid *g) { return (g->d.nx + 31) / 32; }
int df_tiles_y(const asuca_grid *g) { return (g->d.ny + 7) / 8; }
int df_grid_size(asuca_grid *g);

size_t padded_field_elems(const asuca_grid *g) {
    return (size_t)g->d.nz * (g->d.ny + 4) * padded_pitch(g->d.nx);
}

// elements of a padded stage buffer: the F fields in pairs (pair layout)
size_t padded_state_elems(const asuca_grid *g) { return 2 * (size_t)pair_count(g->F) * padded_field_elems(g); }

StepLayout step_layout(const asuca_grid *g) {
    StepLayout L;
    const size_t state = padded_state_elems(g) * elem_size(g);
    size_t off = 0;
    L.ystar = off;
    off = align_up(off + state);
    L.ystar2 = off;
    off = align_up(off + state);
    L.precip = off;
    off = align_up(off + (size_t)g->plane * sizeof(double));
    L.partials = off;
    off = align_up(off + (size_t)g->col_grid * (g->F + 1) * sizeof(double));
    L.scratch = off;
    off = align_up(off + (size_t)g->d.nz * (g->F + 1) * col_slots(g) * sizeof(double));
    L.fscratch = off;
    if (fused_path(g)) off = align_up(off + (size_t)g->d.nz * fscratch_level(g->plane, g->F + 1) * sizeof(double));
    L.falpha = off;
    if (fused_path(g)) off = align_up(off + (size_t)g->d.nz * (size_t)g->plane * sizeof(double));
    L.df_order = L.df_counter = L.df_flags = L.df_partials = L.df_scratch = off;
    if (g->step_mode == 1) {
        const size_t R = (size_t)df_tiles_y(g), tiles = R * df_tiles_x(g);
        L.df_order = off;
        off = align_up(off + 2 * (4 * DF_CHUNK * R) * sizeof(unsigned));
        L.df_counter = off;
        off = align_up(off + sizeof(unsigned));
        L.df_flags = off;
        off = align_up(off + tiles * sizeof(unsigned));
        L.df_partials = off;
        off = align_up(off + tiles * (g->F + 1) * sizeof(double));
        L.df_scratch = off;
        // the co-resident grid is a property of the device and the kernel; it is cached in the grid
        const int dg = df_grid_size(const_cast<asuca_grid *>(g));
        off = align_up(off + (size_t)g->d.nz * (g->F + 1) * (size_t)dg * 256 * sizeof(double));
    }
    L.total = off;
    return L;
}

asuca_status take_status(asuca_grid *g) {
    int s = g->status_host[0];
    if (s != 0) {
        g->status_host[0] = 0;
        return (asuca_status)s;
    }
    return ASUCA_OK;
}

bool state_ok(const asuca_grid *g, const asuca_state *s) {
    return s && s->rho && s->rhotheta && (g->d.ntracers == 0 || s->rhoq) && s->mu && s->mv && s->mw;
}

template <typename T>
void field_ptrs(const asuca_grid *g, void *rho, void *rhotheta, void *rhoq, T **out) {
    out[0] = (T *)rho;
    out[1] = (T *)rhotheta;
    for (int n = 0; n < g->d.ntracers; n++) out[2 + n] = (T *)rhoq + (size_t)n * g->cells;
    for (int f = g->F; f < MAXF; f++) out[f] = nullptr;
}

// per-field views of a padded stage buffer in the workspace (pair layout):
// field f's element (k, j, i) at view[f][k plev + (j + 2) prow + 2 (i + 4)];
// field 1 (pair 0, lane 0) is the buffer's base
template <typename T>
void workspace_fields(const asuca_grid *g, char *ws, size_t off, T **out) {
    const long long P = padded_pitch(g->d.nx);
    for (int f = 0; f < g->F; f++) {
        const int pos = pair_pos(f, g->F);
        out[f] = (T *)(ws + off) + (pos / 2) * 2 * P + (pos % 2);
    }
    for (int f = g->F; f < MAXF; f++) out[f] = nullptr;
}

// row and level strides (elements) of the pair layout
long long pair_row(const asuca_grid *g) { return 2LL * pair_count(g->F) * padded_pitch(g->d.nx); }
long long pair_level(const asuca_grid *g) { return pair_row(g) * (g->d.ny + 4); }

template <typename T>
StageParams<T> stage_params(const asuca_grid *g, const asuca_state *fl, const void *tend) {
    StageParams<T> p;
    std::memset(&p, 0, sizeof(p));
    p.mu = (const T *)fl->mu;
    p.mv = (const T *)fl->mv;
    p.mw = (const T *)fl->mw;
    p.tend = (const T *)tend;
    p.nx = g->d.nx;
    p.ny = g->d.ny;
    p.nz = g->d.nz;
    p.lim = (int)g->d.lim;
    p.plane = g->plane;
    p.plane_u = p.plane_v = g->plane;
    p.status = g->status_dev;
    p.ty = g->stage_ty;
    p.opitch = padded_pitch(g->d.nx);
    p.oplane = (long long)(g->d.ny + 4) * p.opitch;
    p.prow = pair_row(g);
    p.plev = pair_level(g);
    p.rdx = (T)(1.0 / g->d.dx);
    p.rdy = (T)(1.0 / g->d.dy);
    for (int k = 0; k < g->d.nz; k++) p.rdz[k] = (T)(1.0 / g->dz[k]);
    return p;
}

template <typename T>
ColumnParams<T> column_params(const asuca_grid *g, double dt) {
    ColumnParams<T> p;
    std::memset(&p, 0, sizeof(p));
    const asuca_grid_desc &d = g->d;
    const int nz = d.nz;
    p.nx = d.nx;
    p.ny = d.ny;
    p.nz = nz;
    p.plane = g->plane;
    p.status = g->status_dev;
    p.do_relax = d.tau_theta > 0.0;
    p.do_sed = d.v_sed > 0.0 && d.sed_tracer >= 0 && d.sed_tracer < d.ntracers;
    p.sed = p.do_sed ? 2 + d.sed_tracer : -1;
    p.do_diff = d.k0 > 0.0;
    p.do_phys = 1;
    p.relax_r = p.do_relax ? (T)(dt / d.tau_theta) : T(0);
    p.relax_inv = p.do_relax ? (T)(1.0 / (1.0 + dt / d.tau_theta)) : T(1);
    p.sed_dt = (T)dt;
    p.sed_v = (T)d.v_sed;
    p.dt = dt;
    p.dxdy = d.dx * d.dy;
    p.nslots = col_slots(g);
    for (int k = 0; k < nz; k++) {
        p.dz[k] = g->dz[k];
        p.dzT[k] = (T)g->dz[k];
        p.dzlo[k] = (float)(g->dz[k] - (double)(float)g->dz[k]);
        p.sedr[k] = (T)(1.0 / (g->dz[k] + dt * d.v_sed));
        p.thref[k] = (T)(300.0 + 0.004 * g->zc[k]);
        p.dzr_up[k] = (k + 1 < nz) ? g->dz[k + 1] / g->dz[k] : 0.0;
        p.dzr_dn[k] = (k > 0) ? g->dz[k - 1] / g->dz[k] : 0.0;
        p.rdz64[k] = 1.0 / g->dz[k];
        p.rdzT[k] = (T)(1.0 / g->dz[k]);
        if (k + 1 < nz && p.do_diff) {
            const double K = d.k0 * std::exp(-g->zf[k + 1] / d.k_h);
            p.kc[k] = 0.5 * dt * K / (g->zc[k + 1] - g->zc[k]);
        } else {
            p.kc[k] = 0.0;
        }
        p.kcT[k] = (T)p.kc[k];
    }
    return p;
}

asuca_status cuda_status(cudaError_t e) { return e == cudaSuccess ? ASUCA_OK : ASUCA_ERR_CUDA; }

// Launch through f(), bracketed by two events when profiling is on.
template <typename Fn>
cudaError_t timed(asuca_grid *g, int kind, cudaStream_t s, Fn f) {
    if (!g->prof_on) return f();
    if (2 * (g->prof_used + 1) > g->prof_cap) {
        int cap = g->prof_cap ? 2 * g->prof_cap : 256;
        cudaEvent_t *ev = (cudaEvent_t *)std::realloc(g->prof_ev, sizeof(cudaEvent_t) * cap);
        int *kd = (int *)std::realloc(g->prof_kind, sizeof(int) * cap / 2);
        if (!ev || !kd) return cudaErrorMemoryAllocation;
        g->prof_ev = ev;
        g->prof_kind = kd;
        for (int q = g->prof_cap; q < cap; q++) {
            cudaError_t e = cudaEventCreate(&g->prof_ev[q]);
            if (e != cudaSuccess) return e;
        }
        g->prof_cap = cap;
    }
    const int q = g->prof_used;
    cudaError_t e = cudaEventRecord(g->prof_ev[2 * q], s);
    if (e != cudaSuccess) return e;
    if ((e = f()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(g->prof_ev[2 * q + 1], s)) != cudaSuccess) return e;
    g->prof_kind[q] = kind;
    g->prof_used = q + 1;
    return cudaSuccess;
}

// Order of the dataflow tasks for Q phases on R tile rows, entries (q << 12) | r.
// Phase q of row r reads phase q-1 of rows r-1, r, r+1, periodic in the row
// index, so the rows form a ring.  Entries are sorted by the slot
// 2 q + d(r) with d(r) = min(r, R - r): ring neighbours differ by at most 1
// in d, hence every input comes at least one slot earlier, and rows far from
// row 0 lag behind by up to R/2 slots, so phases of different steps
// interleave across the ring.
void df_fill_order(unsigned *out, int Q, int R) {
    int n = 0;
    const int dmax = R / 2;
    for (int w = 0; w <= 2 * (Q - 1) + dmax; w++)
        for (int r = 0; r < R; r++) {
            const int d = r < R - r ? r : R - r;
            const int t = w - d;
            if (t < 0 || (t & 1)) continue;
            const int q = t / 2;
            if (q < Q) out[n++] = ((unsigned)q << 12) | (unsigned)r;
        }
}

// Tensor maps over the caller's fields for stage 1, cached on the grid for the
// last fields seen.  False when the fields do not meet TMA's alignment rules
// (16-byte bases, rows a multiple of 16 bytes) or the domain has no interior tile.
template <typename T>
bool user_maps(asuca_grid *g, const asuca_state *st, int ty) {
    const int nx = g->d.nx, ny = g->d.ny, ntr = g->d.ntracers;
    const void *key[3] = {st->rho, st->rhotheta, ntr > 0 ? st->rhoq : nullptr};
    if (g->umap_ok && g->umap_ty == ty && key[0] == g->umap_key[0] && key[1] == g->umap_key[1] &&
        key[2] == g->umap_key[2])
        return true;
    g->umap_ok = 0;
    if (((size_t)nx * sizeof(T)) % 16 != 0 || nx < 40 || ny < ty + 4) return false;
    for (int q = 0; q < 3; q++)
        if (key[q] && ((uintptr_t)key[q] % 16) != 0) return false;
    if (encode_user_maps<T>(g->umap, key[0], key[1], key[2], ntr, nx, ny, g->d.nz, ty) != cudaSuccess) return false;
    for (int q = 0; q < 3; q++) g->umap_key[q] = key[q];
    g->umap_ty = ty;
    g->umap_ok = 1;
    return true;
}

template <typename T>
asuca_status run_step_dataflow(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps,
                               char *ws, double *budgets, cudaStream_t s);

// No work before the stages: the mass fluxes are the caller's.
struct NoPre {
    static constexpr bool none = true;
    template <typename T>
    cudaError_t operator()(int, int, StageParams<T> &) { return cudaSuccess; }
};

// zero_precip = false continues the precipitation total of a previous call
// on the same workspace (the checkpointed forward runs one call per segment).
// pre(n, -1, sp) runs at the start of step n and pre(n, stage, sp) before each
// RK stage's launch; it may launch work of its own and set the stage's mass
// fluxes (the nested acoustic short steps do both).
template <typename T, typename Pre = NoPre>
asuca_status run_step(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps,
                      char *ws, double *budgets, cudaStream_t s, bool zero_precip = true, Pre pre = Pre()) {
    if (g->step_mode == 1 && zero_precip && Pre::none)
        return run_step_dataflow<T>(g, st, tend, dt, nsteps, ws, budgets, s);
    const StepLayout L = step_layout(g);
    const int F = g->F;
    T *yn[MAXF], *y1[MAXF], *y2[MAXF];
    field_ptrs<T>(g, st->rho, st->rhotheta, st->rhoq, yn);
    workspace_fields<T>(g, ws, L.ystar, y1);
    workspace_fields<T>(g, ws, L.ystar2, y2);
    StageParams<T> sp = stage_params<T>(g, st, tend);
    ColumnParams<T> cp = column_params<T>(g, dt);
    for (int f = 0; f < MAXF; f++) cp.y[f] = yn[f];
    cp.precip_col = (double *)(ws + L.precip);
    cp.partials = (double *)(ws + L.partials);
    cp.scratch = (double *)(ws + L.scratch);

    cudaError_t e = zero_precip ? cudaMemsetAsync(ws + L.precip, 0, (size_t)g->plane * sizeof(double), s) : cudaSuccess;
    if (e != cudaSuccess) return ASUCA_ERR_CUDA;
    if (g->map_ws != (void *)ws || g->map_ty != g->stage_ty) {
        if (encode_stage_map<T>(&g->map_ystar, ws + L.ystar, F, g->d.nx, g->d.ny, g->d.nz, g->stage_ty) != cudaSuccess ||
            encode_stage_map<T>(&g->map_ystar2, ws + L.ystar2, F, g->d.nx, g->d.ny, g->d.nz, g->stage_ty) != cudaSuccess) {
            g->map_ws = nullptr;
            return ASUCA_ERR_CUDA;
        }
        g->map_ws = (void *)ws;
        g->map_ty = g->stage_ty;
    }
    const bool umaps = user_maps<T>(g, st, g->stage_ty);
    const T cdt[3] = {(T)(dt / 3.0), (T)(dt / 2.0), (T)dt};
    for (int f = 0; f < MAXF; f++) sp.ybase[f] = yn[f];
    for (int q = 0; q < 3 && umaps; q++) sp.umap[q] = g->umap[q];
    const bool fused = fused_path(g);
    // with the caller's mass fluxes (no per-stage work) the density after the
    // step is known before stage 2, which then carries the factorisation
    constexpr bool split = Pre::none;
    FusedParams<T> fp;
    if (fused) {
        fp.c = cp;
        fp.c.scratch = (double *)(ws + L.fscratch);
        fp.c.alpha = (double *)(ws + L.falpha);
        fp.c.nslots = g->plane;
    }
    for (int n = 0; n < nsteps; n++) {
        Range step_range("asuca step");
        if ((e = pre(n, -1, sp)) != cudaSuccess) return ASUCA_ERR_CUDA;
        for (int stg = 0; stg < (fused ? 2 : 3); stg++) {
            Range stage_range(stg == 0 ? "RK stage 1" : (stg == 1 ? "RK stage 2" : "RK stage 3"));
            // stage 1 reads the caller's fields (TMA for interior tiles, cp.async at the
            // periodic edges), stages 2 and 3 the padded buffers of phi the previous
            // stage wrote (TMA); stage 3 writes the caller's fields
            sp.tma_in = stg > 0;
            sp.user_tma = (stg == 0) && umaps;
            if (stg == 1) sp.tmap = g->map_ystar;
            if (stg == 2) sp.tmap = g->map_ystar2;
            sp.out_padded = stg < 2;
            T **out = stg == 0 ? y1 : (stg == 1 ? y2 : yn);
            for (int f = 0; f < MAXF; f++) {
                sp.yin[f] = yn[f];
                sp.yout[f] = out[f];
            }
            sp.cdt = cdt[stg];
            if ((e = pre(n, stg, sp)) != cudaSuccess) return ASUCA_ERR_CUDA;
            if (fused && split && stg == 1) {
                // stage 2 marching downward with the factorisation of every column
                FusedParams<T> f2 = fp;
                f2.s = sp;
                f2.s.hcdt = cdt[2];
                e = timed(g, ASUCA_KERNEL_STAGE_FACTOR, s, [&] { return launch_stage2_factor<T>(f2, F, s); });
            } else {
                e = timed(g, ASUCA_KERNEL_STAGE, s, [&] { return launch_stage<T>(sp, F, s); });
            }
            if (e != cudaSuccess) return ASUCA_ERR_CUDA;
        }
        cp.budgets = (budgets != nullptr) && (n == nsteps - 1);
        Range col_range(fused ? "RK stage 3 + column pass" : "column pass");
        if (fused) {
            if ((e = pre(n, 2, sp)) != cudaSuccess) return ASUCA_ERR_CUDA;
            // stage 3 marching downward with the relaxation, sedimentation and
            // elimination of every column, then the bottom-up back substitution
            fp.s = sp;
            fp.s.tma_in = 1;
            fp.s.user_tma = 0;
            fp.s.tmap = g->map_ystar2;
            fp.s.out_padded = 0;
            fp.s.ty = 8;
            for (int f = 0; f < MAXF; f++) {
                fp.s.yin[f] = yn[f];
                fp.s.yout[f] = yn[f];
            }
            fp.s.cdt = cdt[2];
            if ((e = timed(g, ASUCA_KERNEL_STAGE_COLUMN, s, [&] {
                     return split ? launch_stage3_sweep<T>(fp, F, s) : launch_stage3_column<T>(fp, F, s);
                 })) != cudaSuccess)
                return ASUCA_ERR_CUDA;
            ColumnParams<T> cu = fp.c;
            for (int f = 0; f < MAXF; f++) cu.y[f] = yn[f];
            cu.budgets = cp.budgets;
            if ((e = timed(g, ASUCA_KERNEL_COLUMN, s, [&] { return launch_column_up<T>(cu, F, g->col_grid, s); })) !=
                cudaSuccess)
                return ASUCA_ERR_CUDA;
        } else if ((e = timed(g, ASUCA_KERNEL_COLUMN, s,
                              [&] { return launch_column<T>(cp, F, g->col_grid, COL_TPB, s); })) != cudaSuccess) {
            return ASUCA_ERR_CUDA;
        }
    }
    if (budgets) {
        if (nsteps == 0) {
            cp.do_phys = 0;
            cp.budgets = 1;
            if ((e = timed(g, ASUCA_KERNEL_COLUMN, s, [&] { return launch_column<T>(cp, F, g->col_grid, COL_TPB, s); })) != cudaSuccess)
                return ASUCA_ERR_CUDA;
        }
        e = timed(g, ASUCA_KERNEL_REDUCE, s, [&] {
            return launch_budget_reduce(cp.partials, g->col_grid, F + 1, F, g->d.dx * g->d.dy, budgets,
                                        g->status_dev, s);
        });
        if (e != cudaSuccess) return ASUCA_ERR_CUDA;
    }
    return ASUCA_OK;
}

int df_grid_size(asuca_grid *g) {
    if (g->df_grid <= 0) {
        DfParams<double> d64;
        DfParams<float> d32;
        int grid = 0;
        cudaError_t e = g->d.prec == ASUCA_FP64 ? launch_dataflow<double>(d64, g->F, (int)g->d.lim, 0, nullptr, &grid)
                                                : launch_dataflow<float>(d32, g->F, (int)g->d.lim, 0, nullptr, &grid);
        g->df_grid = (e == cudaSuccess && grid > 0) ? grid : 0;
    }
    return g->df_grid;
}

template <typename T>
asuca_status run_step_dataflow(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps,
                               char *ws, double *budgets, cudaStream_t s) {
    const StepLayout L = step_layout(g);
    const int F = g->F, R = df_tiles_y(g), TXn = df_tiles_x(g);
    const int grid = df_grid_size(g);
    if (grid <= 0 || R > 4095) return ASUCA_ERR_UNSUPPORTED;
    T *yn[MAXF], *y1[MAXF], *y2[MAXF];
    field_ptrs<T>(g, st->rho, st->rhotheta, st->rhoq, yn);
    workspace_fields<T>(g, ws, L.ystar, y1);
    workspace_fields<T>(g, ws, L.ystar2, y2);
    if (cudaMemsetAsync(ws + L.precip, 0, (size_t)g->plane * sizeof(double), s) != cudaSuccess) return ASUCA_ERR_CUDA;
    if (g->map_ws != (void *)ws || g->map_ty != 8) {
        if (encode_stage_map<T>(&g->map_ystar, ws + L.ystar, F, g->d.nx, g->d.ny, g->d.nz, 8) != cudaSuccess ||
            encode_stage_map<T>(&g->map_ystar2, ws + L.ystar2, F, g->d.nx, g->d.ny, g->d.nz, 8) != cudaSuccess) {
            g->map_ws = nullptr;
            return ASUCA_ERR_CUDA;
        }
        g->map_ws = (void *)ws;
        g->map_ty = 8;
    }
    DfParams<T> p;
    std::memset(&p, 0, sizeof(p));
    const T cdt[3] = {(T)(dt / 3.0), (T)(dt / 2.0), (T)dt};
    for (int stg = 0; stg < 3; stg++) {
        StageParams<T> sp = stage_params<T>(g, st, tend);
        sp.ty = 8;
        sp.tma_in = stg > 0;
        if (stg == 1) sp.tmap = g->map_ystar;
        if (stg == 2) sp.tmap = g->map_ystar2;
        sp.out_padded = stg < 2;
        T **out = stg == 0 ? y1 : (stg == 1 ? y2 : yn);
        for (int f = 0; f < MAXF; f++) {
            sp.yin[f] = yn[f];
            sp.ybase[f] = yn[f];
            sp.yout[f] = out[f];
        }
        sp.cdt = cdt[stg];
        p.stage[stg] = sp;
    }
    p.col = column_params<T>(g, dt);
    for (int f = 0; f < MAXF; f++) p.col.y[f] = yn[f];
    p.col.precip_col = (double *)(ws + L.precip);
    p.col.budgets = 0;
    p.col_last = p.col;
    p.col_last.budgets = budgets != nullptr;
    p.txn = TXn;
    p.tyn = R;
    p.counter = (unsigned *)(ws + L.df_counter);
    p.flags = (unsigned *)(ws + L.df_flags);
    p.scratch = (double *)(ws + L.df_scratch);
    p.partials = (double *)(ws + L.df_partials);
    p.status = g->status_dev;
    // the column tasks' scratch: one slot per thread of the persistent grid
    // (the column parameters carry it for the bounds-check build's extents)
    p.col.scratch = p.col_last.scratch = p.scratch;
    p.col.nslots = p.col_last.nslots = (long long)df_grid_size(g) * 32 * 8;
    const size_t tiles = (size_t)R * TXn;
    for (int c0 = 0; c0 < nsteps; c0 += DF_CHUNK) {
        const int n = (nsteps - c0) < DF_CHUNK ? (nsteps - c0) : DF_CHUNK;
        const int which = n == DF_CHUNK ? 0 : 1, Q = 4 * n;
        if (!g->df_order_host[which]) {
            void *h = nullptr;
            if (cudaHostAlloc(&h, (size_t)4 * DF_CHUNK * R * sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess)
                return ASUCA_ERR_CUDA;
            g->df_order_host[which] = (unsigned *)h;
            g->df_order_q[which] = -1;
        }
        if (g->df_order_q[which] != Q) {   // contents only change with Q (the grid fixes R)
            df_fill_order(g->df_order_host[which], Q, R);
            g->df_order_q[which] = Q;
        }
        unsigned *dorder = (unsigned *)(ws + L.df_order) + (size_t)which * 4 * DF_CHUNK * R;
        if (cudaMemcpyAsync(dorder, g->df_order_host[which], (size_t)Q * R * sizeof(unsigned), cudaMemcpyHostToDevice,
                            s) != cudaSuccess ||
            cudaMemsetAsync(ws + L.df_counter, 0, sizeof(unsigned), s) != cudaSuccess ||
            cudaMemsetAsync(ws + L.df_flags, 0, tiles * sizeof(unsigned), s) != cudaSuccess)
            return ASUCA_ERR_CUDA;
        p.order = dorder;
        p.nslot = Q * R;
        const bool last_chunk = c0 + n >= nsteps;
        p.last_q0 = (last_chunk && budgets) ? 4 * (n - 1) + 3 : Q + 1;
        if (timed(g, ASUCA_KERNEL_DATAFLOW, s, [&] { return launch_dataflow<T>(p, F, (int)g->d.lim, grid, s, nullptr); }) !=
            cudaSuccess)
            return ASUCA_ERR_CUDA;
    }
    if (budgets) {
        if (nsteps == 0) {
            ColumnParams<T> cp = column_params<T>(g, dt);
            for (int f = 0; f < MAXF; f++) cp.y[f] = yn[f];
            cp.do_phys = 0;
            cp.budgets = 1;
            cp.precip_col = (double *)(ws + L.precip);
            cp.partials = (double *)(ws + L.partials);
            if (launch_column<T>(cp, F, g->col_grid, COL_TPB, s) != cudaSuccess ||
                launch_budget_reduce(cp.partials, g->col_grid, F + 1, F, g->d.dx * g->d.dy, budgets, g->status_dev, s) !=
                    cudaSuccess)
                return ASUCA_ERR_CUDA;
        } else if (timed(g, ASUCA_KERNEL_REDUCE, s, [&] {
                       return launch_budget_reduce(p.partials, (int)tiles, F + 1, F, g->d.dx * g->d.dy, budgets,
                                                   g->status_dev, s);
                   }) != cudaSuccess) {
            return ASUCA_ERR_CUDA;
        }
    }
    return ASUCA_OK;
}

// ---- adjoint -------------------------------------------------------------

struct AdjLayout {
    size_t step, W, ckpt, segYn, segY1, segY2, segY3, branch, facev, rec, lam, l2, l1, acc, scratch, total;
    size_t nrec_step, nfacev_stage;
    size_t setbytes;   // one set of segment buffers (segYn .. rec); set b starts b * setbytes after segYn
    int nsets;         // 2 when there are several segments (recompute and reverse overlap), else 1
    int ncp;
    size_t ustate, pstate, nbranch_step;
    long long slots;
};

int adj_col_grid(const asuca_grid *g) { return g->col_grid; }

// Tile rows of the branch-recording stage launches: the grid's tuned stage
// tile height where a recording variant exists (4 or 8 rows), else 8.
int rec_tile_rows(const asuca_grid *g) { return g->stage_ty == 4 ? 4 : 8; }

// Blocks of the column transpose: 32 columns each (one warp per field), at
// most as many column slots as the scratch holds (adj_col_grid * COL_TPB).
int adj_col_blocks(const asuca_grid *g) {
    const long long need = (g->plane + 31) / 32, cap = (long long)adj_col_grid(g) * COL_TPB / 32;
    return (int)(need < cap ? need : cap);
}


AdjLayout adj_layout(const asuca_grid *g, int nsteps, int K) {
    AdjLayout L;
    const size_t s = elem_size(g);
    L.ustate = (size_t)g->F * g->cells * s;
    L.pstate = padded_state_elems(g) * s;
    L.nbranch_step = (size_t)3 * (g->F - 1) * g->cells;
    L.ncp = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    L.slots = (long long)adj_col_grid(g) * COL_TPB;
    size_t off = 0;
    L.step = off;
    off = align_up(off + step_layout(g).total);
    L.W = off;
    off = align_up(off + L.ustate);
    L.ckpt = off;
    off = align_up(off + (size_t)L.ncp * align_up(L.ustate));
    L.nsets = L.ncp >= 2 ? 2 : 1;
    L.segYn = off;
    off = align_up(off + (size_t)(K + 1) * align_up(L.ustate));
    L.segY1 = off;
    off = align_up(off + (size_t)K * align_up(L.pstate));
    L.segY2 = off;
    off = align_up(off + (size_t)K * align_up(L.pstate));
    L.segY3 = off;
    off = align_up(off + (size_t)K * align_up(L.ustate));
    L.branch = off;
    off = align_up(off + (size_t)K * align_up(L.nbranch_step));
    // per recorded stage: the face values of every cell's three +1/2 faces, [3][F-1][nz][ny][nx]
    L.nfacev_stage = (size_t)3 * (g->F - 1) * g->cells * elem_size(g);
    L.facev = off;
    off = align_up(off + (size_t)K * 3 * align_up(L.nfacev_stage));
    // per recorded step: the column pass's factorisation and solution, [nz][F + 2][ny][nx] doubles
    L.nrec_step = (size_t)g->d.nz * (g->F + 2) * (size_t)g->plane * sizeof(double);
    L.rec = off;
    off = align_up(off + (g->d.k0 > 0.0 ? (size_t)K * align_up(L.nrec_step) : 0));
    L.setbytes = off - L.segYn;
    off = L.segYn + (size_t)L.nsets * L.setbytes;
    L.lam = off;
    off = align_up(off + L.ustate);
    L.l2 = off;
    off = align_up(off + L.ustate);
    L.l1 = off;
    off = align_up(off + L.ustate);
    L.acc = off;
    off = align_up(off + L.ustate);
    L.scratch = off;
    off = align_up(off + (size_t)g->d.nz * (4 + 2 * (g->F - 1)) * L.slots * sizeof(double));
    L.total = off;
    return L;
}

// fields of a contiguous [F][nz][ny][nx] block (user layout)
template <typename T>
void block_fields(const asuca_grid *g, void *base, T **out) {
    for (int f = 0; f < g->F; f++) out[f] = (T *)base + (size_t)f * g->cells;
    for (int f = g->F; f < MAXF; f++) out[f] = nullptr;
}

template <typename T>
asuca_state block_state(const asuca_grid *g, void *base, const asuca_state *m) {
    asuca_state st;
    st.rho = base;
    st.rhotheta = (T *)base + g->cells;
    st.rhoq = (T *)base + 2 * g->cells;
    st.mu = m->mu;
    st.mv = m->mv;
    st.mw = m->mw;
    return st;
}

template <typename T>
asuca_status run_adjoint(asuca_grid *g, const asuca_state *init, const void *tend, double dt, int nsteps,
                         int K, const T *lam_final, T *grad0, T *gmu, T *gmv, T *gmw, char *ws,
                         const char *ckpt_ext, cudaStream_t s) {
    const AdjLayout L = adj_layout(g, nsteps, K);
    const int F = g->F;
    const size_t cb = (size_t)g->cells * sizeof(T);
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
    // checkpoints: the caller's (kept by its forward pass), or made here
    const char *ckbase = ckpt_ext ? ckpt_ext : ws + L.ckpt;
    if (!ckpt_ext) {
        // ---- forward pass from the initial state, keeping a checkpoint every K steps;
        // the last segment's checkpoint is all that is needed of it
        T *Wf[MAXF];
        block_fields<T>(g, ws + L.W, Wf);
        T *init_f[MAXF];
        field_ptrs<T>(g, init->rho, init->rhotheta, init->rhoq, init_f);
        for (int f = 0; f < F; f++) ck(cudaMemcpyAsync(Wf[f], init_f[f], cb, cudaMemcpyDeviceToDevice, s));
        asuca_state Ws = block_state<T>(g, ws + L.W, init);
        const int last_start = L.ncp > 0 ? (L.ncp - 1) * K : 0;
        for (int n = 0; n < last_start; n++) {
            if (n % K == 0)
                ck(cudaMemcpyAsync(ws + L.ckpt + (size_t)(n / K) * align_up(L.ustate), ws + L.W, L.ustate,
                                   cudaMemcpyDeviceToDevice, s));
            if (e != cudaSuccess) return ASUCA_ERR_CUDA;
            asuca_status r = run_step<T>(g, &Ws, tend, dt, 1, ws + L.step, nullptr, s);
            if (r != ASUCA_OK) return r;
        }
        if (L.ncp > 0)
            ck(cudaMemcpyAsync(ws + L.ckpt + (size_t)(L.ncp - 1) * align_up(L.ustate), ws + L.W, L.ustate,
                               cudaMemcpyDeviceToDevice, s));
    }
    // ---- adjoint accumulators
    const size_t mb = (size_t)g->cells * sizeof(T), mwb = (size_t)(g->d.nz + 1) * g->plane * sizeof(T);
    ck(cudaMemsetAsync(gmu, 0, mb, s));
    ck(cudaMemsetAsync(gmv, 0, mb, s));
    ck(cudaMemsetAsync(gmw, 0, mwb, s));
    ck(cudaMemcpyAsync(ws + L.lam, lam_final, L.ustate, cudaMemcpyDeviceToDevice, s));
    if (e != cudaSuccess) return ASUCA_ERR_CUDA;
    T *lam[MAXF], *l2[MAXF], *l1[MAXF], *acc[MAXF];
    block_fields<T>(g, ws + L.lam, lam);
    block_fields<T>(g, ws + L.l2, l2);
    block_fields<T>(g, ws + L.l1, l1);
    block_fields<T>(g, ws + L.acc, acc);
    const T cdt[3] = {(T)(dt / 3.0), (T)(dt / 2.0), (T)dt};
    const StepLayout SL = step_layout(g);
    char *sws = ws + L.step;
    // the recomputation records branches with the grid's tuned tile height (4 or 8 rows)
    const int rty = rec_tile_rows(g);
    // With several segments the buffers come in two sets: the recomputation of
    // segment c - 1 runs on the grid's auxiliary stream into one set while the
    // caller's stream reverses segment c from the other.  A set is recomputed
    // only after the reversal that last read it (segment c + 2) has finished.
    std::vector<CUtensorMap> maps(2 * (size_t)K * L.nsets);
    for (int b = 0; b < L.nsets; b++)
        for (int q = 0; q < K; q++) {
            char *y1 = ws + L.segY1 + (size_t)b * L.setbytes + (size_t)q * align_up(L.pstate);
            char *y2 = ws + L.segY2 + (size_t)b * L.setbytes + (size_t)q * align_up(L.pstate);
            if (encode_stage_map<T>(&maps[2 * ((size_t)b * K + q)], y1, F, g->d.nx, g->d.ny, g->d.nz, rty) !=
                    cudaSuccess ||
                encode_stage_map<T>(&maps[2 * ((size_t)b * K + q) + 1], y2, F, g->d.nx, g->d.ny, g->d.nz, rty) !=
                    cudaSuccess)
                return ASUCA_ERR_CUDA;
        }
    cudaStream_t s2 = g->aux_stream;
    cudaEvent_t ev_fork = g->aux_ev[0], ev_join = g->aux_ev[1];
    cudaEvent_t ev_rec[2] = {g->aux_ev[2], g->aux_ev[3]}, ev_rev[2] = {g->aux_ev[4], g->aux_ev[5]};
    ck(cudaEventRecord(ev_fork, s));
    ck(cudaStreamWaitEvent(s2, ev_fork, 0));
    if (e != cudaSuccess) return ASUCA_ERR_CUDA;
    for (int c = L.ncp - 1; c >= 0; c--) {
        const int start = c * K, len = (nsteps - start) < K ? (nsteps - start) : K;
        const int b = L.nsets == 2 ? (c & 1) : 0;
        const size_t so = (size_t)b * L.setbytes;
        auto segYn = [&](int q) { return ws + L.segYn + so + (size_t)q * align_up(L.ustate); };
        auto segY1 = [&](int q) { return ws + L.segY1 + so + (size_t)q * align_up(L.pstate); };
        auto segY2 = [&](int q) { return ws + L.segY2 + so + (size_t)q * align_up(L.pstate); };
        auto segY3 = [&](int q) { return ws + L.segY3 + so + (size_t)q * align_up(L.ustate); };
        auto rec = [&](int q) { return (double *)(ws + L.rec + so + (size_t)q * align_up(L.nrec_step)); };
        auto fvs = [&](int q, int stg) {
            return (T *)(ws + L.facev + so + ((size_t)q * 3 + stg) * align_up(L.nfacev_stage));
        };
        auto brs = [&](int q, int stg) {
            return (uint8_t *)(ws + L.branch + so + (size_t)q * align_up(L.nbranch_step)) +
                   (size_t)stg * (F - 1) * g->cells;
        };
        if (c + L.nsets < L.ncp) ck(cudaStreamWaitEvent(s2, ev_rev[b], 0));
        ck(cudaMemcpyAsync(segYn(0), ckbase + (size_t)c * align_up(L.ustate), L.ustate,
                           cudaMemcpyDeviceToDevice, s2));
        if (e != cudaSuccess) return ASUCA_ERR_CUDA;
        // ---- recompute the segment (auxiliary stream), recording stage states and limiter branches
        Range seg_range("adjoint segment");
        for (int q = 0; q < len; q++) {
            Range rec_range("adjoint recompute step");
            T *yn[MAXF], *y1[MAXF], *y2[MAXF], *y3[MAXF];
            block_fields<T>(g, segYn(q), yn);
            workspace_fields<T>(g, segY1(q), 0, y1);
            workspace_fields<T>(g, segY2(q), 0, y2);
            block_fields<T>(g, segY3(q), y3);
            StageParams<T> sp = stage_params<T>(g, init, tend);
            sp.ty = rty;
            for (int f = 0; f < MAXF; f++) sp.ybase[f] = yn[f];
            for (int stg = 0; stg < 3; stg++) {
                sp.tma_in = stg > 0;
                if (stg > 0) sp.tmap = maps[2 * ((size_t)b * K + q) + (stg - 1)];
                sp.out_padded = stg < 2;
                T **out = stg == 0 ? y1 : (stg == 1 ? y2 : y3);
                for (int f = 0; f < MAXF; f++) {
                    sp.yin[f] = yn[f];
                    sp.yout[f] = out[f];
                }
                sp.cdt = cdt[stg];
                sp.branch = brs(q, stg);
                sp.facev = fvs(q, stg);
                if (timed(g, ASUCA_KERNEL_STAGE, s2, [&] { return launch_stage<T>(sp, F, s2); }) != cudaSuccess)
                    return ASUCA_ERR_CUDA;
            }
            ck(cudaMemcpyAsync(segYn(q + 1), segY3(q), L.ustate, cudaMemcpyDeviceToDevice, s2));
            ColumnParams<T> cp = column_params<T>(g, dt);
            block_fields<T>(g, segYn(q + 1), cp.y);
            cp.precip_col = (double *)(sws + SL.precip);
            cp.partials = (double *)(sws + SL.partials);
            cp.scratch = (double *)(sws + SL.scratch);
            cp.budgets = 0;
            cp.rec = cp.do_diff ? rec(q) : nullptr;
            if (e != cudaSuccess ||
                timed(g, ASUCA_KERNEL_COLUMN, s2,
                      [&] { return launch_column<T>(cp, F, g->col_grid, COL_TPB, s2); }) != cudaSuccess)
                return ASUCA_ERR_CUDA;
        }
        ck(cudaEventRecord(ev_rec[b], s2));
        ck(cudaStreamWaitEvent(s, ev_rec[b], 0));
        if (e != cudaSuccess) return ASUCA_ERR_CUDA;
        // ---- reverse through the segment
        for (int q = len - 1; q >= 0; q--) {
            Range rev_range("adjoint reverse step");
            AdjColParams<T> ac;
            std::memset(&ac, 0, sizeof(ac));
            ac.c = column_params<T>(g, dt);
            block_fields<T>(g, segY3(q), ac.c.y);
            ac.c.scratch = (double *)(ws + L.scratch);
            ac.c.nslots = L.slots;
            ac.c.rec = ac.c.do_diff ? rec(q) : nullptr;
            for (int f = 0; f < MAXF; f++) ac.lam[f] = lam[f];
            if (timed(g, ASUCA_KERNEL_ADJ_COLUMN, s, [&] { return launch_adj_column<T>(ac, F, adj_col_blocks(g), s); }) !=
                cudaSuccess)
                return ASUCA_ERR_CUDA;
            for (int stg = 2; stg >= 0; stg--) {
                AdjStageParams<T> ap;
                std::memset(&ap, 0, sizeof(ap));
                if (stg == 0) {
                    block_fields<T>(g, segYn(q), (T **)ap.ys);
                    ap.ys_pitch = g->d.nx;
                    ap.ys_plane = g->plane;
                    ap.ys_xs = 1;
                    ap.ys_ox = ap.ys_oy = 0;
                } else {
                    workspace_fields<T>(g, stg == 1 ? segY1(q) : segY2(q), 0, (T **)ap.ys);
                    ap.ys_pitch = pair_row(g);
                    ap.ys_plane = pair_level(g);
                    ap.ys_xs = 2;
                    ap.ys_ox = 4;
                    ap.ys_oy = 2;
                    ap.ys_phi = 1;
                }
                T **lin = stg == 2 ? lam : (stg == 1 ? l2 : l1);
                for (int f = 0; f < MAXF; f++) ap.lam[f] = lin[f];
                ap.cs = cdt[stg];
                ap.branch = brs(q, stg);
                ap.facev = fvs(q, stg);
                ap.mu = (const T *)init->mu;
                ap.mv = (const T *)init->mv;
                ap.mw = (const T *)init->mw;
                for (int f = 0; f < MAXF; f++) {
                    ap.out1[f] = stg == 2 ? l2[f] : (stg == 1 ? l1[f] : nullptr);
                    ap.out2[f] = stg == 0 ? lam[f] : acc[f];
                    ap.base2[f] = stg == 2 ? nullptr : acc[f];
                }
                ap.add_self = stg == 2;
                ap.gmu = gmu;
                ap.gmv = gmv;
                ap.gmw = gmw;
                ap.nx = g->d.nx;
                ap.ny = g->d.ny;
                ap.nz = g->d.nz;
                ap.plane = g->plane;
                ap.rdx = (T)(1.0 / g->d.dx);
                ap.rdy = (T)(1.0 / g->d.dy);
                for (int k = 0; k < g->d.nz; k++) ap.rdz[k] = (T)(1.0 / g->dz[k]);
                if (timed(g, ASUCA_KERNEL_ADJ_STAGE, s, [&] { return launch_adj_stage<T>(ap, F, (int)g->d.lim, s); }) !=
                    cudaSuccess)
                    return ASUCA_ERR_CUDA;
            }
        }
        ck(cudaEventRecord(ev_rev[b], s));
    }
    // the auxiliary stream's work joins the caller's stream
    ck(cudaEventRecord(ev_join, s2));
    ck(cudaStreamWaitEvent(s, ev_join, 0));
    ck(cudaMemcpyAsync(grad0, ws + L.lam, L.ustate, cudaMemcpyDeviceToDevice, s));
    return e == cudaSuccess ? ASUCA_OK : ASUCA_ERR_CUDA;
}

// Forward steps (asuca_step's) that also keep the state before steps 0, K,
// 2K, ... in ckpt ([ceil(nsteps / K)] blocks of F fields, each block padded
// to 256 bytes), the checkpoints run_adjoint reverses from.
template <typename T>
asuca_status run_forward_ckpt(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps, int K,
                              char *ckpt, char *ws, double *budgets, cudaStream_t s) {
    const int F = g->F;
    const size_t cb = (size_t)g->cells * sizeof(T), us = align_up((size_t)F * cb);
    T *yf[MAXF];
    field_ptrs<T>(g, st->rho, st->rhotheta, st->rhoq, yf);
    if (nsteps == 0) return run_step<T>(g, st, tend, dt, 0, ws, budgets, s);
    for (int c = 0; c * K < nsteps; c++) {
        for (int f = 0; f < F; f++)
            if (cudaMemcpyAsync(ckpt + (size_t)c * us + (size_t)f * cb, yf[f], cb, cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess)
                return ASUCA_ERR_CUDA;
        const int n = (nsteps - c * K) < K ? (nsteps - c * K) : K;
        const bool last = (c + 1) * K >= nsteps;
        asuca_status r = run_step<T>(g, st, tend, dt, n, ws, last ? budgets : nullptr, s, c == 0);
        if (r != ASUCA_OK) return r;
    }
    return ASUCA_OK;
}

// Forward steps that record every stage's limiter branches into out
// ([nsteps][3][F-1][nz][ny][nx] bytes), using the one-step adjoint layout.
template <typename T>
asuca_status run_record(asuca_grid *g, const asuca_state *init, const void *tend, double dt, int nsteps,
                        unsigned char *out, char *ws, cudaStream_t s) {
    const AdjLayout L = adj_layout(g, 1, 1);
    const int F = g->F;
    const size_t cb = (size_t)g->cells * sizeof(T);
    CUtensorMap m1, m2;
    if (encode_stage_map<T>(&m1, ws + L.segY1, F, g->d.nx, g->d.ny, g->d.nz, 8) != cudaSuccess ||
        encode_stage_map<T>(&m2, ws + L.segY2, F, g->d.nx, g->d.ny, g->d.nz, 8) != cudaSuccess)
        return ASUCA_ERR_CUDA;
    T *yn[MAXF], *y1[MAXF], *y2[MAXF], *y3[MAXF], *init_f[MAXF];
    block_fields<T>(g, ws + L.segYn, yn);
    workspace_fields<T>(g, ws + L.segY1, 0, y1);
    workspace_fields<T>(g, ws + L.segY2, 0, y2);
    block_fields<T>(g, ws + L.segY3, y3);
    field_ptrs<T>(g, init->rho, init->rhotheta, init->rhoq, init_f);
    for (int f = 0; f < F; f++)
        if (cudaMemcpyAsync(yn[f], init_f[f], cb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return ASUCA_ERR_CUDA;
    const StepLayout SL = step_layout(g);
    char *sws = ws + L.step;
    const T cdt[3] = {(T)(dt / 3.0), (T)(dt / 2.0), (T)dt};
    for (int n = 0; n < nsteps; n++) {
        StageParams<T> sp = stage_params<T>(g, init, tend);
        sp.ty = 8;
        for (int f = 0; f < MAXF; f++) sp.ybase[f] = yn[f];
        for (int stg = 0; stg < 3; stg++) {
            sp.tma_in = stg > 0;
            if (stg > 0) sp.tmap = stg == 1 ? m1 : m2;
            sp.out_padded = stg < 2;
            T **o = stg == 0 ? y1 : (stg == 1 ? y2 : y3);
            for (int f = 0; f < MAXF; f++) {
                sp.yin[f] = yn[f];
                sp.yout[f] = o[f];
            }
            sp.cdt = cdt[stg];
            sp.branch = out + ((size_t)n * 3 + stg) * (F - 1) * g->cells;
            if (launch_stage<T>(sp, F, s) != cudaSuccess) return ASUCA_ERR_CUDA;
        }
        if (cudaMemcpyAsync(ws + L.segYn, ws + L.segY3, L.ustate, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return ASUCA_ERR_CUDA;
        ColumnParams<T> cp = column_params<T>(g, dt);
        for (int f = 0; f < MAXF; f++) cp.y[f] = yn[f];
        cp.precip_col = (double *)(sws + SL.precip);
        cp.partials = (double *)(sws + SL.partials);
        cp.scratch = (double *)(sws + SL.scratch);
        cp.budgets = 0;
        if (launch_column<T>(cp, F, g->col_grid, COL_TPB, s) != cudaSuccess) return ASUCA_ERR_CUDA;
    }
    return ASUCA_OK;
}

// ---- ensemble ------------------------------------------------------------

struct EnsLayout {
    size_t members, bar, per_member, partials, total;
    std::vector<size_t> ystar, ystar2, precip, fscratch, falpha;
    int grid, threads;
};

template <typename T>
cudaError_t ens_grid(const asuca_grid *g0, int nzmax, int *grid) {
    EnsParams<T> dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    dummy.nzmax = nzmax;
    return launch_ensemble<T>(dummy, g0->F, (int)g0->d.lim, g0->ens_ty, 0, nullptr, grid);
}

int ens_nzmax(asuca_grid *const *grids, int M) {
    int nz = 0;
    for (int m = 0; m < M; m++) nz = grids[m]->d.nz > nz ? grids[m]->d.nz : nz;
    return nz;
}

bool ens_layout(asuca_grid *const *grids, int M, EnsLayout *L) {
    const asuca_grid *g0 = grids[0];
    int grid = 0;
    const int nzmax = ens_nzmax(grids, M);
    cudaError_t e = g0->d.prec == ASUCA_FP64 ? ens_grid<double>(g0, nzmax, &grid)
                                             : ens_grid<float>(g0, nzmax, &grid);
    if (e != cudaSuccess || grid <= 0) return false;
    L->grid = grid;
    L->threads = 32 * g0->ens_ty;
    const size_t msize = g0->d.prec == ASUCA_FP64 ? sizeof(EnsMember<double>) : sizeof(EnsMember<float>);
    size_t off = 0;
    L->members = off;
    off = align_up(off + (size_t)M * msize);
    L->bar = off;
    off = align_up(off + 2 * sizeof(unsigned));
    L->ystar.resize(M);
    L->ystar2.resize(M);
    L->precip.resize(M);
    L->fscratch.resize(M);
    L->falpha.resize(M);
    int maxcol = 0;
    for (int m = 0; m < M; m++) {
        const size_t ps = padded_state_elems(grids[m]) * elem_size(grids[m]);
        L->ystar[m] = off;
        off = align_up(off + ps);
        L->ystar2[m] = off;
        off = align_up(off + ps);
        L->precip[m] = off;
        off = align_up(off + (size_t)grids[m]->plane * sizeof(double));
        // the column pass split over stages 2 and 3 (fused scratch, alpha)
        L->fscratch[m] = off;
        off = align_up(off + (size_t)grids[m]->d.nz * fscratch_level(grids[m]->plane, g0->F + 1) * sizeof(double));
        L->falpha[m] = off;
        off = align_up(off + (size_t)grids[m]->d.nz * (size_t)grids[m]->plane * sizeof(double));
        if (grids[m]->col_grid > maxcol) maxcol = grids[m]->col_grid;
    }
    L->partials = off;
    off = align_up(off + (size_t)maxcol * (g0->F + 1) * sizeof(double));
    L->total = off;
    return true;
}

struct EnsGraph {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    void *staging = nullptr;
};
std::mutex g_ens_mu;
EnsGraph g_ens_cache[4];
int g_ens_next = 0;

template <typename T>
asuca_status ens_enqueue(asuca_grid *const *grids, asuca_state *states, const double *dts, int M, int nsteps,
                         char *ws, const EnsLayout &L, double *budgets, void *staging, cudaStream_t s) {
    asuca_grid *g0 = grids[0];
    const int F = g0->F;
    EnsMember<T> *mb = (EnsMember<T> *)staging;
    long long tile0 = 0, col0 = 0;
    const int TX = 32, TY = g0->ens_ty;
    for (int m = 0; m < M; m++) {
        asuca_grid *g = grids[m];
        const double dt = dts[m];
        std::memset((void *)&mb[m], 0, sizeof(EnsMember<T>));
        T *yn[MAXF], *y1[MAXF], *y2[MAXF];
        field_ptrs<T>(g, states[m].rho, states[m].rhotheta, states[m].rhoq, yn);
        workspace_fields<T>(g, ws, L.ystar[m], y1);
        workspace_fields<T>(g, ws, L.ystar2[m], y2);
        CUtensorMap m1, m2;
        if (encode_stage_map<T>(&m1, ws + L.ystar[m], F, g->d.nx, g->d.ny, g->d.nz, TY) != cudaSuccess ||
            encode_stage_map<T>(&m2, ws + L.ystar2[m], F, g->d.nx, g->d.ny, g->d.nz, TY) != cudaSuccess)
            return ASUCA_ERR_CUDA;
        const T cdt[3] = {(T)(dt / 3.0), (T)(dt / 2.0), (T)dt};
        for (int stg = 0; stg < 3; stg++) {
            StageParams<T> sp = stage_params<T>(g, &states[m], nullptr);
            sp.status = g0->status_dev;
            sp.ty = TY;
            sp.tma_in = stg > 0;
            if (stg == 1) sp.tmap = m1;
            if (stg == 2) sp.tmap = m2;
            sp.out_padded = stg < 2;
            T **out = stg == 0 ? y1 : (stg == 1 ? y2 : yn);
            for (int f = 0; f < MAXF; f++) {
                sp.yin[f] = yn[f];
                sp.ybase[f] = yn[f];
                sp.yout[f] = out[f];
            }
            sp.cdt = cdt[stg];
            sp.hcdt = cdt[2];   // stage 2's factorisation takes the density after the step
            // stage 1 reads the member's fields by TMA where their rows allow (the kernel
            // takes the maps from the member table in global memory)
            if (stg == 0 && user_maps<T>(g, &states[m], TY)) {
                for (int q = 0; q < 3; q++) sp.umap[q] = g->umap[q];
                sp.user_tma = 1;
            }
            mb[m].stage[stg] = sp;
        }
        ColumnParams<T> cp = column_params<T>(g, dt);
        for (int f = 0; f < MAXF; f++) cp.y[f] = yn[f];
        cp.precip_col = (double *)(ws + L.precip[m]);
        cp.scratch = (double *)(ws + L.fscratch[m]);
        cp.alpha = (double *)(ws + L.falpha[m]);
        cp.nslots = g->plane;
        cp.status = g0->status_dev;   // the ensemble reports through the first member's grid
        cp.budgets = 0;
        mb[m].col = cp;
        const int tx = (g->d.nx + TX - 1) / TX, ty = (g->d.ny + TY - 1) / TY;
        mb[m].tiles_x = tx;
        mb[m].tile0 = tile0;
        mb[m].col0 = col0;
        tile0 += (long long)tx * ty;
        col0 += g->plane;
    }
    cudaError_t e = cudaMemcpyAsync(ws + L.members, staging, (size_t)M * sizeof(EnsMember<T>),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.bar, 0, 2 * sizeof(unsigned), s);
    for (int m = 0; m < M && e == cudaSuccess; m++)
        e = cudaMemsetAsync(ws + L.precip[m], 0, (size_t)grids[m]->plane * sizeof(double), s);
    if (e != cudaSuccess) return ASUCA_ERR_CUDA;
    EnsParams<T> ep;
    std::memset(&ep, 0, sizeof(ep));
    ep.members = (const EnsMember<T> *)(ws + L.members);
    ep.nmembers = M;
    ep.nsteps = nsteps;
    ep.nzmax = ens_nzmax(grids, M);
    ep.total_tiles = tile0;
    ep.total_cols = col0;
    ep.bar_count = (unsigned *)(ws + L.bar);
    ep.bar_gen = ep.bar_count + 1;
    ep.bar_extra = g0->barrier_extra;
    ep.status = g0->status_dev;
    if (nsteps > 0 &&
        timed(g0, ASUCA_KERNEL_ENSEMBLE, s, [&] { return launch_ensemble<T>(ep, F, (int)g0->d.lim, TY, L.grid, s, nullptr); }) !=
            cudaSuccess)
        return ASUCA_ERR_CUDA;
    if (budgets) {
        for (int m = 0; m < M; m++) {
            asuca_grid *g = grids[m];
            ColumnParams<T> cp = column_params<T>(g, dts[m]);
            field_ptrs<T>(g, states[m].rho, states[m].rhotheta, states[m].rhoq, cp.y);
            cp.do_phys = 0;
            cp.budgets = 1;
            cp.precip_col = (double *)(ws + L.precip[m]);
            cp.partials = (double *)(ws + L.partials);
            cp.nslots = col_slots(g);
            if (launch_column<T>(cp, F, g->col_grid, COL_TPB, s) != cudaSuccess ||
                launch_budget_reduce(cp.partials, g->col_grid, F + 1, F, g->d.dx * g->d.dy, budgets + (size_t)m * (F + 1),
                                     g0->status_dev, s) != cudaSuccess)
                return ASUCA_ERR_CUDA;
        }
    }
    return ASUCA_OK;
}

// ---- open lateral boundaries ----------------------------------------------
// Workspace of an open domain: the step workspace (its two padded stage
// buffers hold phi* and phi**) followed by a third padded buffer for phi^n.
size_t open_b0_offset(const asuca_grid *g) { return step_layout(g).total; }
size_t open_total(const asuca_grid *g) {
    return align_up(open_b0_offset(g) + padded_state_elems(g) * elem_size(g));
}
size_t open_buffer_offset(const asuca_grid *g, int b) {
    const StepLayout L = step_layout(g);
    return b == 0 ? open_b0_offset(g) : (b == 1 ? L.ystar : L.ystar2);
}
bool open_fits(const asuca_grid *g) {
    return (long long)g->d.nz * (g->d.ny + 1) * (long long)(g->d.nx + 1) < (1LL << 32);
}

template <typename T>
bool open_maps(asuca_grid *g, char *ws) {
    if (g->omap_ws == (void *)ws && g->omap_ty == g->stage_ty) return true;
    for (int b = 0; b < 3; b++)
        if (encode_stage_map<T>(&g->omap[b], ws + open_buffer_offset(g, b), g->F, g->d.nx, g->d.ny, g->d.nz,
                                g->stage_ty) != cudaSuccess) {
            g->omap_ws = nullptr;
            return false;
        }
    g->omap_ws = (void *)ws;
    g->omap_ty = g->stage_ty;
    return true;
}

template <typename T>
OpenParams<T> open_params(const asuca_grid *g, char *ws, int b) {
    OpenParams<T> p;
    std::memset(&p, 0, sizeof(p));
    workspace_fields<T>(g, ws, open_buffer_offset(g, b), p.pad);
    p.pitch = pair_row(g);
    p.pplane = pair_level(g);
    p.nx = g->d.nx;
    p.ny = g->d.ny;
    p.nz = g->d.nz;
    p.nt = g->F - 1;
    return p;
}

template <typename T>
asuca_status run_open_prepare(asuca_grid *g, const asuca_state *st, bool first, char *ws, cudaStream_t s) {
    if (first && cudaMemsetAsync(ws + step_layout(g).precip, 0, (size_t)g->plane * sizeof(double), s) != cudaSuccess)
        return ASUCA_ERR_CUDA;
    OpenParams<T> p = open_params<T>(g, ws, 0);
    T *y[MAXF];
    field_ptrs<T>(g, st->rho, st->rhotheta, st->rhoq, y);
    for (int f = 0; f < MAXF; f++) p.y[f] = y[f];
    return cuda_status(timed(g, ASUCA_KERNEL_STAGE, s, [&] { return launch_open_prepare<T>(p, s); }));
}

template <typename T>
asuca_status run_open_halo(asuca_grid *g, char *ws, int b, bool pack, const void *in0, const void *in1,
                           double tratio, void *out, cudaStream_t s) {
    OpenParams<T> p = open_params<T>(g, ws, b);
    p.hin0 = (const T *)in0;
    p.hin1 = (const T *)in1;
    p.hout = (T *)out;
    p.w0 = (T)(1.0 - tratio);
    p.w1 = (T)tratio;
    return cuda_status(launch_halo<T>(p, pack, g->nsm, s));
}

template <typename T>
asuca_status run_open_stage(asuca_grid *g, asuca_state *st, const void *tend, double dt, int stage, char *ws,
                            double *budgets, cudaStream_t s) {
    if (!open_maps<T>(g, ws)) return ASUCA_ERR_CUDA;
    const StepLayout L = step_layout(g);
    const int F = g->F;
    T *yn[MAXF], *next[MAXF];
    field_ptrs<T>(g, st->rho, st->rhotheta, st->rhoq, yn);
    StageParams<T> sp = stage_params<T>(g, st, tend);
    sp.open = 1;
    sp.plane_u = (long long)g->d.ny * (g->d.nx + 1);
    sp.plane_v = (long long)(g->d.ny + 1) * g->d.nx;
    sp.tma_in = 1;
    sp.user_tma = 0;
    sp.tmap = g->omap[stage];
    for (int f = 0; f < MAXF; f++) sp.ybase[f] = sp.yin[f] = yn[f];
    const T cdt[3] = {(T)(dt / 3.0), (T)(dt / 2.0), (T)dt};
    sp.cdt = cdt[stage];
    cudaError_t e;
    if (stage < 2) {
        workspace_fields<T>(g, ws, open_buffer_offset(g, stage + 1), next);
        sp.out_padded = 1;
        for (int f = 0; f < MAXF; f++) sp.yout[f] = next[f];
        return cuda_status(timed(g, ASUCA_KERNEL_STAGE, s, [&] { return launch_stage<T>(sp, F, s); }));
    }
    ColumnParams<T> cp = column_params<T>(g, dt);
    for (int f = 0; f < MAXF; f++) cp.y[f] = yn[f];
    cp.precip_col = (double *)(ws + L.precip);
    cp.partials = (double *)(ws + L.partials);
    cp.scratch = (double *)(ws + L.scratch);
    cp.budgets = budgets != nullptr;
    sp.out_padded = 0;
    for (int f = 0; f < MAXF; f++) sp.yout[f] = yn[f];
    if (fused_path(g)) {
        FusedParams<T> fp;
        fp.c = cp;
        fp.c.scratch = (double *)(ws + L.fscratch);
        fp.c.nslots = g->plane;
        fp.s = sp;
        fp.s.ty = 8;
        if ((e = timed(g, ASUCA_KERNEL_STAGE_COLUMN, s, [&] { return launch_stage3_column<T>(fp, F, s); })) !=
            cudaSuccess)
            return ASUCA_ERR_CUDA;
        ColumnParams<T> cu = fp.c;
        cu.budgets = cp.budgets;
        if ((e = timed(g, ASUCA_KERNEL_COLUMN, s, [&] { return launch_column_up<T>(cu, F, g->col_grid, s); })) !=
            cudaSuccess)
            return ASUCA_ERR_CUDA;
    } else {
        if ((e = timed(g, ASUCA_KERNEL_STAGE, s, [&] { return launch_stage<T>(sp, F, s); })) != cudaSuccess)
            return ASUCA_ERR_CUDA;
        if ((e = timed(g, ASUCA_KERNEL_COLUMN, s,
                       [&] { return launch_column<T>(cp, F, g->col_grid, COL_TPB, s); })) != cudaSuccess)
            return ASUCA_ERR_CUDA;
    }
    if (budgets) {
        e = timed(g, ASUCA_KERNEL_REDUCE, s, [&] {
            return launch_budget_reduce(cp.partials, g->col_grid, F + 1, F, g->d.dx * g->d.dy, budgets,
                                        g->status_dev, s);
        });
        if (e != cudaSuccess) return ASUCA_ERR_CUDA;
    }
    return ASUCA_OK;
}

template <typename T>
asuca_status run_step_open(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps, const void *b0,
                           const void *b1, double tratio, char *ws, double *budgets, cudaStream_t s) {
    if (nsteps == 0) return run_step<T>(g, st, tend, dt, 0, ws, budgets, s);
    for (int n = 0; n < nsteps; n++) {
        Range step_range("asuca open step");
        asuca_status r = run_open_prepare<T>(g, st, n == 0, ws, s);
        for (int stg = 0; stg < 3 && r == ASUCA_OK; stg++) {
            r = run_open_halo<T>(g, ws, stg, false, b0, b1, tratio, nullptr, s);
            if (r == ASUCA_OK)
                r = run_open_stage<T>(g, st, tend, dt, stg, ws, n == nsteps - 1 ? budgets : nullptr, s);
        }
        if (r != ASUCA_OK) return r;
    }
    return ASUCA_OK;
}

bool open_ws_ok(const asuca_grid *g, const void *ws, size_t bytes) {
    return ws && ((uintptr_t)ws % ALIGN) == 0 && bytes >= open_total(g);
}

}  // namespace

// ---- column pass without a caller workspace ------------------------------
// Scratch for the Thomas intermediates of asuca_column_noalloc().  It lives in
// a file-scope device array, so every GPU that loads this library holds these
// bytes until the process exits; all calls on one device share it.
#define ASUCA_NOALLOC_BYTES (16u << 20)
static __device__ __align__(256) double g_noalloc_scratch[ASUCA_NOALLOC_BYTES / sizeof(double)];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
asuca_status noalloc_scratch(int dev, double **out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return ASUCA_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ASUCA_ERR_CUDA;
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return ASUCA_OK;
}

template <typename T>
cudaError_t launch_column_noalloc(asuca_grid *g, asuca_state *st, double dt, double *precip_col,
                                  double *scratch, int blocks, cudaStream_t s) {
    ColumnParams<T> p = column_params<T>(g, dt);
    field_ptrs<T>(g, st->rho, st->rhotheta, st->rhoq, p.y);
    p.precip_col = precip_col;
    p.partials = nullptr;          // budgets stay off: the kernel never touches partials
    p.budgets = 0;
    p.scratch = scratch;
    p.nslots = (long long)blocks * COL_TPB;
    return launch_column<T>(p, g->F, blocks, COL_TPB, s);
}
}  // namespace

extern "C" {

int asuca_bounds_checked(void) {
#ifdef ASUCA_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

const char *asuca_status_string(asuca_status s) {
    switch (s) {
        case ASUCA_OK: return "ok";
        case ASUCA_ERR_ARG: return "invalid argument";
        case ASUCA_ERR_CUDA: return "CUDA runtime error";
        case ASUCA_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case ASUCA_ERR_NONFINITE: return "non-finite budget";
        case ASUCA_ERR_TIMEOUT: return "device barrier timed out";
        case ASUCA_ERR_UNSUPPORTED: return "unsupported size";
        case ASUCA_ERR_BOUNDS: return "a kernel index fell outside its buffer";
    }
    return "unknown status";
}

asuca_status asuca_init_grid(const asuca_grid_desc *desc, asuca_grid **out) {
    if (!desc || !out) return ASUCA_ERR_ARG;
    *out = nullptr;
    const asuca_grid_desc &d = *desc;
    if (d.nx < 4 || d.ny < 4 || d.nz < 3 || d.ntracers < 0 || !d.dz) return ASUCA_ERR_ARG;
    if (d.nz > ASUCA_MAX_NZ || d.ntracers > ASUCA_MAX_TRACERS) return ASUCA_ERR_UNSUPPORTED;
    if (!(d.dx > 0.0) || !(d.dy > 0.0) || !std::isfinite(d.dx) || !std::isfinite(d.dy)) return ASUCA_ERR_ARG;
    if (!(d.tau_theta >= 0.0) || !(d.k0 >= 0.0) || !(d.v_sed >= 0.0)) return ASUCA_ERR_ARG;
    if (d.k0 > 0.0 && !(d.k_h > 0.0)) return ASUCA_ERR_ARG;
    if (d.sed_tracer < -1 || d.sed_tracer >= d.ntracers) return ASUCA_ERR_ARG;
    if (d.lim != ASUCA_LIM_KOREN && d.lim != ASUCA_LIM_LINEAR && d.lim != ASUCA_LIM_UPWIND1) return ASUCA_ERR_ARG;
    if (d.prec != ASUCA_FP64 && d.prec != ASUCA_FP32_MIXED) return ASUCA_ERR_ARG;
    for (int k = 0; k < d.nz; k++)
        if (!(d.dz[k] > 0.0) || !std::isfinite(d.dz[k])) return ASUCA_ERR_ARG;
    if ((long long)d.nx * d.ny > (1LL << 31)) return ASUCA_ERR_UNSUPPORTED;
    // element offsets within one field (caller layout with nz + 1 levels of MW,
    // and the padded stage buffers) are 32-bit in the kernels
    if ((long long)d.nx * d.ny * (d.nz + 1) >= (1LL << 32) ||
        2LL * pair_count(2 + d.ntracers) * padded_pitch(d.nx) * (d.ny + 4) * (long long)d.nz >= (1LL << 32))
        return ASUCA_ERR_UNSUPPORTED;

    asuca_grid *g = new (std::nothrow) asuca_grid;
    if (!g) return ASUCA_ERR_ARG;
    std::memset((void *)g, 0, sizeof(*g));
    g->d = d;
    g->d.dz = nullptr;
    g->zf[0] = 0.0;
    for (int k = 0; k < d.nz; k++) {
        g->dz[k] = d.dz[k];
        g->zf[k + 1] = g->zf[k] + d.dz[k];
        g->zc[k] = g->zf[k] + 0.5 * d.dz[k];
    }
    g->F = 2 + d.ntracers;
    g->plane = (long long)d.nx * d.ny;
    g->cells = g->plane * d.nz;
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        delete g;
        return ASUCA_ERR_CUDA;
    }
    g->col_blocks_per_sm = col_blocks_per_sm();
    g->stage_ty = 8;
    g->ens_ty = 8;
    g->step_mode = 0;
    g->fused_col = 1;
    set_col_grid(g);
    void *h = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocMapped) != cudaSuccess) {
        delete g;
        return ASUCA_ERR_CUDA;
    }
    std::memset(h, 0, 64);
    g->status_host = (volatile int *)h;
    if (cudaHostGetDevicePointer((void **)&g->status_dev, h, 0) != cudaSuccess) {
        cudaFreeHost(h);
        delete g;
        return ASUCA_ERR_CUDA;
    }
    g->last_stream = nullptr;
    bool aux_ok = cudaStreamCreateWithFlags(&g->aux_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int q = 0; q < 6; q++)
        aux_ok = aux_ok && cudaEventCreateWithFlags(&g->aux_ev[q], cudaEventDisableTiming) == cudaSuccess;
    if (!aux_ok) {
        cudaFreeHost(h);
        delete g;
        return ASUCA_ERR_CUDA;
    }
    *out = g;
    return ASUCA_OK;
}

asuca_status asuca_free_grid(asuca_grid *g) {
    if (!g) return ASUCA_ERR_ARG;
    if (g->status_host) cudaFreeHost((void *)g->status_host);
    for (int q = 0; q < g->prof_cap; q++) cudaEventDestroy(g->prof_ev[q]);
    for (int w = 0; w < 2; w++)
        if (g->df_order_host[w]) cudaFreeHost(g->df_order_host[w]);
    if (g->kept_pinned) {
        for (void *p : *g->kept_pinned) cudaFreeHost(p);
        delete g->kept_pinned;
    }
    std::free(g->prof_ev);
    std::free(g->prof_kind);
    for (int q = 0; q < 6; q++) cudaEventDestroy(g->aux_ev[q]);
    cudaStreamDestroy(g->aux_stream);
    delete g;
    return ASUCA_OK;
}

size_t asuca_workspace_bytes(const asuca_grid *g, int op, int param) {
    if (!g) return 0;
    if (op == ASUCA_OP_STEP) return step_layout(g).total;
    if (op == ASUCA_OP_ADJOINT) return param >= 0 ? adj_layout(g, param, 10).total : 0;
    return 0;
}

size_t asuca_adjoint_workspace_bytes(const asuca_grid *g, int nsteps, int checkpoint_every) {
    if (!g || nsteps < 0 || checkpoint_every < 1) return 0;
    return adj_layout(g, nsteps, checkpoint_every).total;
}

asuca_status asuca_adjoint_step(asuca_grid *g, const asuca_state *initial, const void *tendencies, double dt,
                                int nsteps, int checkpoint_every, const void *lambda_final, void *grad_initial,
                                void *grad_mu, void *grad_mv, void *grad_mw, void *workspace,
                                size_t workspace_bytes, void *cuda_stream) {
    if (!g || !state_ok(g, initial) || nsteps < 0 || checkpoint_every < 1 || !std::isfinite(dt) || dt < 0.0 ||
        !lambda_final || !grad_initial || !grad_mu || !grad_mv || !grad_mw)
        return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 ||
        workspace_bytes < adj_layout(g, nsteps, checkpoint_every).total)
        return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    if (g->d.prec == ASUCA_FP64)
        return run_adjoint<double>(g, initial, tendencies, dt, nsteps, checkpoint_every, (const double *)lambda_final,
                                   (double *)grad_initial, (double *)grad_mu, (double *)grad_mv, (double *)grad_mw,
                                   (char *)workspace, nullptr, s);
    return run_adjoint<float>(g, initial, tendencies, dt, nsteps, checkpoint_every, (const float *)lambda_final,
                              (float *)grad_initial, (float *)grad_mu, (float *)grad_mv, (float *)grad_mw,
                              (char *)workspace, nullptr, s);
}

size_t asuca_checkpoint_bytes(const asuca_grid *g, int nsteps, int checkpoint_every) {
    if (!g || nsteps < 0 || checkpoint_every < 1) return 0;
    const size_t n = nsteps > 0 ? (size_t)((nsteps + checkpoint_every - 1) / checkpoint_every) : 0;
    return n * align_up((size_t)g->F * g->cells * elem_size(g));
}

asuca_status asuca_forward_checkpointed(asuca_grid *g, asuca_state *state, const void *tendencies, double dt,
                                        int nsteps, int checkpoint_every, void *checkpoints,
                                        size_t checkpoint_bytes, void *workspace, size_t workspace_bytes,
                                        double *budgets_dev, void *cuda_stream) {
    if (!g || !state_ok(g, state) || nsteps < 0 || checkpoint_every < 1 || !std::isfinite(dt) || dt < 0.0)
        return ASUCA_ERR_ARG;
    if (nsteps > 0 && (!checkpoints || checkpoint_bytes < asuca_checkpoint_bytes(g, nsteps, checkpoint_every) ||
                       ((uintptr_t)checkpoints % ALIGN) != 0))
        return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < step_layout(g).total)
        return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    return g->d.prec == ASUCA_FP64
               ? run_forward_ckpt<double>(g, state, tendencies, dt, nsteps, checkpoint_every, (char *)checkpoints,
                                          (char *)workspace, budgets_dev, s)
               : run_forward_ckpt<float>(g, state, tendencies, dt, nsteps, checkpoint_every, (char *)checkpoints,
                                         (char *)workspace, budgets_dev, s);
}

asuca_status asuca_adjoint_from_checkpoints(asuca_grid *g, const void *checkpoints, const asuca_state *fluxes,
                                            const void *tendencies, double dt, int nsteps, int checkpoint_every,
                                            const void *lambda_final, void *grad_initial, void *grad_mu,
                                            void *grad_mv, void *grad_mw, void *workspace, size_t workspace_bytes,
                                            void *cuda_stream) {
    if (!g || !fluxes || !fluxes->mu || !fluxes->mv || !fluxes->mw || nsteps < 0 || checkpoint_every < 1 ||
        !std::isfinite(dt) || dt < 0.0 || !lambda_final || !grad_initial || !grad_mu || !grad_mv || !grad_mw ||
        (nsteps > 0 && (!checkpoints || ((uintptr_t)checkpoints % ALIGN) != 0)))
        return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 ||
        workspace_bytes < adj_layout(g, nsteps, checkpoint_every).total)
        return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    if (g->d.prec == ASUCA_FP64)
        return run_adjoint<double>(g, fluxes, tendencies, dt, nsteps, checkpoint_every, (const double *)lambda_final,
                                   (double *)grad_initial, (double *)grad_mu, (double *)grad_mv, (double *)grad_mw,
                                   (char *)workspace, (const char *)checkpoints, s);
    return run_adjoint<float>(g, fluxes, tendencies, dt, nsteps, checkpoint_every, (const float *)lambda_final,
                              (float *)grad_initial, (float *)grad_mu, (float *)grad_mv, (float *)grad_mw,
                              (char *)workspace, (const char *)checkpoints, s);
}

asuca_status asuca_debug_record_branches(asuca_grid *g, const asuca_state *initial, const void *tendencies,
                                         double dt, int nsteps, unsigned char *branches_dev, void *workspace,
                                         size_t workspace_bytes, void *cuda_stream) {
    if (!g || !state_ok(g, initial) || nsteps < 0 || !branches_dev || !std::isfinite(dt) || dt < 0.0)
        return ASUCA_ERR_ARG;
    const AdjLayout L = adj_layout(g, 1, 1);
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < L.total) return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    return g->d.prec == ASUCA_FP64
               ? run_record<double>(g, initial, tendencies, dt, nsteps, branches_dev, (char *)workspace, s)
               : run_record<float>(g, initial, tendencies, dt, nsteps, branches_dev, (char *)workspace, s);
}

size_t asuca_ensemble_workspace_bytes(asuca_grid *const *grids, int nmembers) {
    if (!grids || nmembers <= 0 || !grids[0]) return 0;
    EnsLayout L;
    if (!ens_layout(grids, nmembers, &L)) return 0;
    return L.total;
}

asuca_status asuca_ensemble_step(asuca_grid *const *grids, asuca_state *states, const double *dts, int nmembers,
                                 int nsteps, void *workspace, size_t workspace_bytes, double *budgets_dev,
                                 void *cuda_stream) {
    if (!grids || !states || !dts || nmembers <= 0 || nsteps < 0) return ASUCA_ERR_ARG;
    asuca_grid *g0 = grids[0];
    if (!g0) return ASUCA_ERR_ARG;
    for (int m = 0; m < nmembers; m++) {
        const asuca_grid *g = grids[m];
        if (!g || !state_ok(g, &states[m]) || !std::isfinite(dts[m]) || dts[m] < 0.0) return ASUCA_ERR_ARG;
        if (g->F != g0->F || g->d.nz != g0->d.nz || g->d.prec != g0->d.prec || g->d.lim != g0->d.lim ||
            g->device != g0->device || g->ens_ty != g0->ens_ty)
            return ASUCA_ERR_ARG;
    }
    asuca_status prev = take_status(g0);
    if (prev != ASUCA_OK) return prev;
    EnsLayout L;
    if (!ens_layout(grids, nmembers, &L)) return ASUCA_ERR_CUDA;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < L.total) return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g0->last_stream = s;
    const size_t msize = g0->d.prec == ASUCA_FP64 ? sizeof(EnsMember<double>) : sizeof(EnsMember<float>);
    // graph key: everything the captured launches depend on
    std::vector<unsigned char> key;
    auto put = [&](const void *p, size_t n) { key.insert(key.end(), (const unsigned char *)p, (const unsigned char *)p + n); };
    put(&nmembers, sizeof(int));
    put(&nsteps, sizeof(int));
    put(&workspace, sizeof(void *));
    put(&budgets_dev, sizeof(void *));
    for (int m = 0; m < nmembers; m++) {
        put(&grids[m], sizeof(void *));
        put(&states[m], sizeof(asuca_state));
        put(&dts[m], sizeof(double));
        put(&grids[m]->col_grid, sizeof(int));
        put(&grids[m]->d.nx, sizeof(int));
        put(&grids[m]->d.ny, sizeof(int));
        put(&grids[m]->barrier_extra, sizeof(int));
        put(&grids[m]->ens_ty, sizeof(int));
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (s != nullptr && cudaStreamIsCapturing(s, &cap) != cudaSuccess) return ASUCA_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) {
        // the caller is capturing: record the launches into the caller's graph; the
        // parameter buffer its copy node reads is kept until the first grid is freed
        void *pin = nullptr;
        if (cudaHostAlloc(&pin, (size_t)nmembers * msize, cudaHostAllocDefault) != cudaSuccess) return ASUCA_ERR_CUDA;
        if (!g0->kept_pinned) g0->kept_pinned = new (std::nothrow) std::vector<void *>();
        if (!g0->kept_pinned) {
            cudaFreeHost(pin);
            return ASUCA_ERR_CUDA;
        }
        g0->kept_pinned->push_back(pin);
        return g0->d.prec == ASUCA_FP64
                   ? ens_enqueue<double>(grids, states, dts, nmembers, nsteps, (char *)workspace, L, budgets_dev, pin, s)
                   : ens_enqueue<float>(grids, states, dts, nmembers, nsteps, (char *)workspace, L, budgets_dev, pin, s);
    }
    if (s == nullptr || g0->prof_on) {
        // the legacy stream cannot be captured, and per-kernel profiling needs the
        // event pairs: launch directly, then release the parameter buffer
        void *pin = nullptr;
        if (cudaHostAlloc(&pin, (size_t)nmembers * msize, cudaHostAllocDefault) != cudaSuccess) return ASUCA_ERR_CUDA;
        asuca_status r = g0->d.prec == ASUCA_FP64
                             ? ens_enqueue<double>(grids, states, dts, nmembers, nsteps, (char *)workspace, L, budgets_dev, pin, s)
                             : ens_enqueue<float>(grids, states, dts, nmembers, nsteps, (char *)workspace, L, budgets_dev, pin, s);
        if (cudaStreamSynchronize(s) != cudaSuccess && r == ASUCA_OK) r = ASUCA_ERR_CUDA;
        cudaFreeHost(pin);
        return r;
    }
    std::lock_guard<std::mutex> lock(g_ens_mu);
    for (EnsGraph &c : g_ens_cache) {
        if (c.exec && c.key == key) return cudaGraphLaunch(c.exec, s) == cudaSuccess ? ASUCA_OK : ASUCA_ERR_CUDA;
    }
    EnsGraph &c = g_ens_cache[g_ens_next];
    g_ens_next = (g_ens_next + 1) % 4;
    if (c.exec) {
        cudaGraphExecDestroy(c.exec);
        c.exec = nullptr;
    }
    if (c.staging) {
        cudaFreeHost(c.staging);
        c.staging = nullptr;
    }
    if (cudaHostAlloc(&c.staging, (size_t)nmembers * msize, cudaHostAllocDefault) != cudaSuccess) return ASUCA_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ASUCA_ERR_CUDA;
    asuca_status r = g0->d.prec == ASUCA_FP64
                         ? ens_enqueue<double>(grids, states, dts, nmembers, nsteps, (char *)workspace, L, budgets_dev, c.staging, s)
                         : ens_enqueue<float>(grids, states, dts, nmembers, nsteps, (char *)workspace, L, budgets_dev, c.staging, s);
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (r != ASUCA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (ee != cudaSuccess || cudaGraphInstantiate(&c.exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        c.exec = nullptr;
        return ASUCA_ERR_CUDA;
    }
    cudaGraphDestroy(graph);
    c.key = key;
    return cudaGraphLaunch(c.exec, s) == cudaSuccess ? ASUCA_OK : ASUCA_ERR_CUDA;
}

asuca_status asuca_set_tuning(asuca_grid *g, int key, int value) {
    if (!g) return ASUCA_ERR_ARG;
    switch (key) {
        case ASUCA_TUNE_COL_BLOCKS_PER_SM:
            if (value < 1 || value > 16) return ASUCA_ERR_ARG;
            g->col_blocks_per_sm = value;
            set_col_grid(g);
            return ASUCA_OK;
        case ASUCA_TUNE_BARRIER_EXTRA:
            if (value < 0) return ASUCA_ERR_ARG;
            g->barrier_extra = value;
            return ASUCA_OK;
        case ASUCA_TUNE_STAGE_TILE_ROWS:
            if (g->d.prec == ASUCA_FP64 ? value != 8 : (value != 4 && value != 8 && value != 16)) return ASUCA_ERR_ARG;
            g->stage_ty = value;
            return ASUCA_OK;
        case ASUCA_TUNE_ENSEMBLE_TILE_ROWS:
            if (g->d.prec == ASUCA_FP64 ? value != 8 : (value != 4 && value != 8)) return ASUCA_ERR_ARG;
            g->ens_ty = value;
            return ASUCA_OK;
        case ASUCA_TUNE_STEP_MODE:
            if (value != 0 && value != 1) return ASUCA_ERR_ARG;
            g->step_mode = value;
            return ASUCA_OK;
        case ASUCA_TUNE_FUSED_COLUMN:
            if (value != 0 && value != 1) return ASUCA_ERR_ARG;
            g->fused_col = value;
            return ASUCA_OK;
        default: return ASUCA_ERR_ARG;
    }
}

int asuca_get_tuning(const asuca_grid *g, int key) {
    if (!g) return -1;
    switch (key) {
        case ASUCA_TUNE_COL_BLOCKS_PER_SM: return g->col_blocks_per_sm;
        case ASUCA_TUNE_BARRIER_EXTRA: return g->barrier_extra;
        case ASUCA_TUNE_STAGE_TILE_ROWS: return g->stage_ty;
        case ASUCA_TUNE_ENSEMBLE_TILE_ROWS: return g->ens_ty;
        case ASUCA_TUNE_STEP_MODE: return g->step_mode;
        case ASUCA_TUNE_FUSED_COLUMN: return g->fused_col;
        default: return -1;
    }
}

asuca_status asuca_get_status(asuca_grid *g) {
    if (!g) return ASUCA_ERR_ARG;
    if (cudaStreamSynchronize(g->last_stream) != cudaSuccess) return ASUCA_ERR_CUDA;
    return take_status(g);
}

asuca_status asuca_step(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps,
                        void *workspace, size_t workspace_bytes, double *budgets_dev,
                        void *cuda_stream) {
    if (!g || !state_ok(g, st) || nsteps < 0 || !std::isfinite(dt) || dt < 0.0) return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    if (nsteps == 0 && !budgets_dev) return ASUCA_OK;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 ||
        workspace_bytes < step_layout(g).total)
        return ASUCA_ERR_WORKSPACE;
    if (g->d.prec == ASUCA_FP64)
        return run_step<double>(g, st, tend, dt, nsteps, (char *)workspace, budgets_dev, s);
    return run_step<float>(g, st, tend, dt, nsteps, (char *)workspace, budgets_dev, s);
}

asuca_status asuca_debug_stage(asuca_grid *g, const asuca_state *in, const asuca_state *base,
                               asuca_state *out, const void *tend, double cdt, void *cuda_stream) {
    if (!g || !state_ok(g, in) || !base || !out || !base->rho || !out->rho || !std::isfinite(cdt))
        return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    cudaError_t e;
    if (g->d.prec == ASUCA_FP64) {
        StageParams<double> p = stage_params<double>(g, in, tend);
        field_ptrs<double>(g, in->rho, in->rhotheta, in->rhoq, (double **)p.yin);
        field_ptrs<double>(g, base->rho, base->rhotheta, base->rhoq, (double **)p.ybase);
        field_ptrs<double>(g, out->rho, out->rhotheta, out->rhoq, p.yout);
        p.cdt = cdt;
        e = launch_stage<double>(p, g->F, s);
    } else {
        StageParams<float> p = stage_params<float>(g, in, tend);
        field_ptrs<float>(g, in->rho, in->rhotheta, in->rhoq, (float **)p.yin);
        field_ptrs<float>(g, base->rho, base->rhotheta, base->rhoq, (float **)p.ybase);
        field_ptrs<float>(g, out->rho, out->rhotheta, out->rhoq, p.yout);
        p.cdt = (float)cdt;
        e = launch_stage<float>(p, g->F, s);
    }
    return cuda_status(e);
}

asuca_status asuca_debug_column(asuca_grid *g, asuca_state *st, double dt, double *precip_col,
                                void *workspace, size_t workspace_bytes, void *cuda_stream) {
    if (!g || !st || !st->rho || !st->rhotheta || (g->d.ntracers && !st->rhoq) || !precip_col ||
        !std::isfinite(dt) || dt < 0.0)
        return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    const StepLayout L = step_layout(g);
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < L.total)
        return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    char *ws = (char *)workspace;
    cudaError_t e;
    if (g->d.prec == ASUCA_FP64) {
        ColumnParams<double> p = column_params<double>(g, dt);
        field_ptrs<double>(g, st->rho, st->rhotheta, st->rhoq, p.y);
        p.precip_col = precip_col;
        p.partials = (double *)(ws + L.partials);
        p.scratch = (double *)(ws + L.scratch);
        e = launch_column<double>(p, g->F, g->col_grid, COL_TPB, s);
    } else {
        ColumnParams<float> p = column_params<float>(g, dt);
        field_ptrs<float>(g, st->rho, st->rhotheta, st->rhoq, p.y);
        p.precip_col = precip_col;
        p.partials = (double *)(ws + L.partials);
        p.scratch = (double *)(ws + L.scratch);
        e = launch_column<float>(p, g->F, g->col_grid, COL_TPB, s);
    }
    return cuda_status(e);
}

asuca_status asuca_column_noalloc(asuca_grid *g, asuca_state *st, double dt, double *precip_col,
                                  void *cuda_stream) {
    if (!g || !st || !st->rho || !st->rhotheta || (g->d.ntracers && !st->rhoq) || !precip_col ||
        !std::isfinite(dt) || dt < 0.0)
        return ASUCA_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ASUCA_ERR_CUDA;
    if (dev != g->device) return ASUCA_ERR_ARG;
    // one 128-column block needs nz * (F + 1) doubles per column of scratch
    const size_t per_block = (size_t)g->d.nz * (g->F + 1) * COL_TPB * sizeof(double);
    const size_t fit = ASUCA_NOALLOC_BYTES / per_block;
    if (fit < 1) return ASUCA_ERR_UNSUPPORTED;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    double *scratch = nullptr;
    asuca_status rs = noalloc_scratch(dev, &scratch);
    if (rs != ASUCA_OK) return rs;
    const int blocks = (int)((size_t)g->col_grid < fit ? (size_t)g->col_grid : fit);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    cudaError_t e = g->d.prec == ASUCA_FP64
                        ? launch_column_noalloc<double>(g, st, dt, precip_col, scratch, blocks, s)
                        : launch_column_noalloc<float>(g, st, dt, precip_col, scratch, blocks, s);
    return cuda_status(e);
}

asuca_status asuca_debug_numerics(const float *in_f, const double *in_d, int n, double *widen,
                                  float *narrow, double *rcp, void *cuda_stream) {
    if (n < 0 || (n > 0 && ((widen && !in_f) || ((narrow || rcp) && !in_d)))) return ASUCA_ERR_ARG;
    return cuda_status(launch_numerics(in_f, in_d, n, widen, narrow, rcp, (cudaStream_t)cuda_stream));
}

asuca_status asuca_debug_dataflow_order(int nphases, int nrows, unsigned *out) {
    if (nphases < 1 || nrows < 1 || nrows > 4095 || nphases > 4 * DF_CHUNK || !out) return ASUCA_ERR_ARG;
    df_fill_order(out, nphases, nrows);
    return ASUCA_OK;
}

size_t asuca_open_workspace_bytes(const asuca_grid *g) { return g ? open_total(g) : 0; }

size_t asuca_halo_count(const asuca_grid *g) {
    return g ? (size_t)2 * (2 * (size_t)g->d.nx + 2 * (size_t)g->d.ny) * g->d.nz * (g->F - 1) : 0;
}

asuca_status asuca_open_prepare(asuca_grid *g, const asuca_state *st, int first, void *ws, size_t ws_bytes,
                                void *cuda_stream) {
    if (!g || !st || !st->rho || !st->rhotheta || (g->d.ntracers && !st->rhoq)) return ASUCA_ERR_ARG;
    if (!open_fits(g)) return ASUCA_ERR_UNSUPPORTED;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!open_ws_ok(g, ws, ws_bytes)) return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    return g->d.prec == ASUCA_FP64 ? run_open_prepare<double>(g, st, first != 0, (char *)ws, s)
                                   : run_open_prepare<float>(g, st, first != 0, (char *)ws, s);
}

asuca_status asuca_open_stage(asuca_grid *g, asuca_state *st, const void *tend, double dt, int stage, void *ws,
                              size_t ws_bytes, double *budgets, void *cuda_stream) {
    if (!g || !state_ok(g, st) || stage < 0 || stage > 2 || !std::isfinite(dt) || dt < 0.0) return ASUCA_ERR_ARG;
    if (!open_fits(g)) return ASUCA_ERR_UNSUPPORTED;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!open_ws_ok(g, ws, ws_bytes)) return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    return g->d.prec == ASUCA_FP64 ? run_open_stage<double>(g, st, tend, dt, stage, (char *)ws, budgets, s)
                                   : run_open_stage<float>(g, st, tend, dt, stage, (char *)ws, budgets, s);
}

asuca_status asuca_halo_pack(asuca_grid *g, const void *ws, size_t ws_bytes, int buffer, void *send,
                             void *cuda_stream) {
    if (!g || !send || buffer < 0 || buffer > 2) return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!open_ws_ok(g, ws, ws_bytes)) return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    char *w = (char *)const_cast<void *>(ws);
    return g->d.prec == ASUCA_FP64 ? run_open_halo<double>(g, w, buffer, true, nullptr, nullptr, 0.0, send, s)
                                   : run_open_halo<float>(g, w, buffer, true, nullptr, nullptr, 0.0, send, s);
}

asuca_status asuca_halo_unpack(asuca_grid *g, void *ws, size_t ws_bytes, int buffer, const void *recv,
                               const void *bnd1, double tratio, void *cuda_stream) {
    if (!g || !recv || buffer < 0 || buffer > 2 || !std::isfinite(tratio)) return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (!open_ws_ok(g, ws, ws_bytes)) return ASUCA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    return g->d.prec == ASUCA_FP64
               ? run_open_halo<double>(g, (char *)ws, buffer, false, recv, bnd1, tratio, nullptr, s)
               : run_open_halo<float>(g, (char *)ws, buffer, false, recv, bnd1, tratio, nullptr, s);
}

asuca_status asuca_step_open(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps,
                             const void *bnd0, const void *bnd1, double tratio, void *ws, size_t ws_bytes,
                             double *budgets, void *cuda_stream) {
    if (!g || !state_ok(g, st) || nsteps < 0 || !std::isfinite(dt) || dt < 0.0 || !bnd0 || !std::isfinite(tratio))
        return ASUCA_ERR_ARG;
    if (!open_fits(g)) return ASUCA_ERR_UNSUPPORTED;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    if (nsteps == 0 && !budgets) return ASUCA_OK;
    if (!open_ws_ok(g, ws, ws_bytes)) return ASUCA_ERR_WORKSPACE;
    return g->d.prec == ASUCA_FP64
               ? run_step_open<double>(g, st, tend, dt, nsteps, bnd0, bnd1, tratio, (char *)ws, budgets, s)
               : run_step_open<float>(g, st, tend, dt, nsteps, bnd0, bnd1, tratio, (char *)ws, budgets, s);
}

asuca_status asuca_profile_enable(asuca_grid *g, int on) {
    if (!g) return ASUCA_ERR_ARG;
    g->prof_on = on != 0;
    g->prof_used = 0;
    return ASUCA_OK;
}

asuca_status asuca_stencil7(const void *in, void *out, int nx, int ny, int nz, int layout, int prec, double c,
                            void *cuda_stream) {
    if (!in || !out || in == out || nx < 2 || ny < 2 || nz < 1 || (layout != 0 && layout != 1) ||
        (prec != ASUCA_FP64 && prec != ASUCA_FP32_MIXED) || !std::isfinite(c))
        return ASUCA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const cudaError_t e = prec == ASUCA_FP64
                              ? launch_stencil7<double>((const double *)in, (double *)out, nx, ny, nz, layout, c, s)
                              : launch_stencil7<float>((const float *)in, (float *)out, nx, ny, nz, layout, (float)c, s);
    return cuda_status(e);
}

asuca_status asuca_debug_damping_cells(int nx, int ny, int nz, int width, int ntop, unsigned *ijk, size_t n) {
    if (nx < 1 || ny < 1 || nz < 1 || width < 0 || width > ASUCA_DAMP_MAX_WIDTH || 2 * width > std::min(nx, ny) ||
        ntop < 0 || ntop > nz || (double)nx * ny * nz >= 4294967296.0)
        return ASUCA_ERR_ARG;
    const DampZone z = damping_zone(nx, ny, nz, width, ntop);
    if (!ijk || n != (size_t)z.total) return ASUCA_ERR_ARG;
    for (unsigned u = 0; u < z.total; u++)
        damping_cell(u, (unsigned)width, (unsigned)nx, (unsigned)ny, (unsigned)nz, (unsigned)ntop, z.frame, z.nlow,
                     z.plane, ijk[3 * (size_t)u], ijk[3 * (size_t)u + 1], ijk[3 * (size_t)u + 2]);
    return ASUCA_OK;
}

size_t asuca_damping_zone_cells(int nx, int ny, int nz, int width, int ntop) {
    if (nx < 1 || ny < 1 || nz < 1 || width < 0 || width > ASUCA_DAMP_MAX_WIDTH || 2 * width > std::min(nx, ny) ||
        ntop < 0 || ntop > nz || (double)nx * ny * nz >= 4294967296.0)
        return 0;
    return damping_zone(nx, ny, nz, width, ntop).total;
}

asuca_status asuca_damping(asuca_grid *g, asuca_state *st, const void *ref, const void *bnd0, const void *bnd1,
                           double mtratio, double tratio, double dt, const asuca_damping_desc *desc,
                           void *cuda_stream) {
    if (!g || !st || !st->rho || !st->rhotheta || (g->d.ntracers && !st->rhoq) || !ref || !bnd0 || !bnd1 || !desc)
        return ASUCA_ERR_ARG;
    const int nx = g->d.nx, ny = g->d.ny, nz = g->d.nz;
    const asuca_damping_desc &dd = *desc;
    if (dd.width < 0 || dd.width > ASUCA_DAMP_MAX_WIDTH || 2 * dd.width > std::min(nx, ny) || dd.ntop < 0 ||
        dd.ntop > nz || !std::isfinite(dd.nu_lat) || dd.nu_lat < 0.0 || !std::isfinite(dd.nu_top) ||
        dd.nu_top < 0.0 || !std::isfinite(dt) || dt < 0.0 || !std::isfinite(mtratio) || !std::isfinite(tratio))
        return ASUCA_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ASUCA_ERR_CUDA;
    if (dev != g->device) return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (g->d.prec == ASUCA_FP64) {
        double *y[MAXF];
        field_ptrs<double>(g, st->rho, st->rhotheta, st->rhoq, y);
        e = launch_damping<double>(y, g->F, (const double *)ref, (const double *)bnd0, (const double *)bnd1, nx, ny,
                                   nz, dd.width, dd.ntop, dd.nu_lat, dd.nu_top, mtratio, tratio, dt, g->nsm, s);
    } else {
        float *y[MAXF];
        field_ptrs<float>(g, st->rho, st->rhotheta, st->rhoq, y);
        e = launch_damping<float>(y, g->F, (const float *)ref, (const float *)bnd0, (const float *)bnd1, nx, ny,
                                  nz, dd.width, dd.ntop, dd.nu_lat, dd.nu_top, mtratio, tratio, dt, g->nsm, s);
    }
    return cuda_status(e);
}

size_t asuca_acoustic_workspace_bytes(const asuca_grid *g) {
    if (!g) return 0;
    const size_t s = g->d.prec == ASUCA_FP64 ? sizeof(double) : sizeof(float);
    const size_t plane = (size_t)g->plane;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return 3 * al(plane * g->d.nz * s) + al(plane * (g->d.nz + 1) * s);
}

}  // extern "C"

namespace {
// the per-level coefficients and the factorisation of one stage (length tau)
template <typename T>
void acoustic_tables(const asuca_grid *g, const asuca_acoustic_desc &a, double tau, AcousticParams<T> &p) {
    const int nz = g->d.nz;
    double Bd[MAXNZ];
    for (int k = 0; k < nz; k++) {
        const double r0 = a.rho0c[k], dz = g->dz[k];
        p.gx[k] = (T)(tau * a.cs2 * r0 / g->d.dx);
        p.gy[k] = (T)(tau * a.cs2 * r0 / g->d.dy);
        p.cr[k] = (T)(tau / r0);
        p.cw[k] = (T)((1.0 - a.beta) / dz);
        Bd[k] = tau * a.beta / (r0 * dz);
        p.B[k] = (T)Bd[k];
    }
    double cprev = 0.0;
    for (int f = 0; f <= nz; f++) {
        p.cq[f] = p.A[f] = p.lo[f] = p.inv[f] = p.cp[f] = T(0);
        if (f < 1 || f > nz - 1) continue;
        const double dzc = 0.5 * (g->dz[f - 1] + g->dz[f]);
        const double G = tau * a.cs2 * a.rho0f[f] / dzc;
        const double A = G * a.beta;
        const double lower = f >= 2 ? -A * Bd[f - 1] : 0.0;
        const double diag = 1.0 + A * (Bd[f] + Bd[f - 1]);
        const double upper = f <= nz - 2 ? -A * Bd[f] : 0.0;
        const double inv = 1.0 / (diag - lower * cprev);
        cprev = upper * inv;
        p.cq[f] = (T)(G * (1.0 - a.beta));
        p.A[f] = (T)A;
        p.lo[f] = (T)lower;
        p.inv[f] = (T)inv;
        p.cp[f] = (T)cprev;
    }
}

// ---- acoustic short steps nested in the RK3 stages --------------------------

// short steps of RK stage q (weights 1/3, 1/2, 1) when a long step has ns
int hevi_short_steps(int ns, int q) {
    const double frac = q == 0 ? 1.0 / 3.0 : (q == 1 ? 0.5 : 1.0);
    const int n = (int)std::floor(frac * ns + 0.5);
    return n < 1 ? 1 : n;
}

struct HeviLayout {
    size_t Sn, Ua, Va, Wa, Sa, Mu, Mv, Mw, Us, Vs, Ws, Ss, total;
};

// the step workspace, then the acoustic arrays: s^n, a stage's integration
// (Ua, Va, Wa, Sa), its mean mass fluxes (Mu, Mv, Mw) and the short steps'
// stage-1 values (Us, Vs, Ws, Ss)
HeviLayout hevi_layout(const asuca_grid *g) {
    HeviLayout L;
    const size_t es = elem_size(g), C = (size_t)g->cells * es, CW = ((size_t)g->cells + (size_t)g->plane) * es;
    size_t off = step_layout(g).total;
    size_t *slot[12] = {&L.Sn, &L.Ua, &L.Va, &L.Wa, &L.Sa, &L.Mu, &L.Mv, &L.Mw, &L.Us, &L.Vs, &L.Ws, &L.Ss};
    const bool wface[12] = {false, false, false, true, false, false, false, true, false, false, true, false};
    for (int q = 0; q < 12; q++) {
        *slot[q] = off;
        off = align_up(off + (wface[q] ? CW : C));
    }
    L.total = off;
    return L;
}

// The work before each RK stage of a step with nested short steps: stage q
// integrates the acoustic system from t^n (the caller's momenta, s^n from the
// density) over its weight times dt in hevi_short_steps(ns, q) short steps,
// accumulating the mean mass fluxes the scalar stage then advects with; stage
// 3 integrates the caller's momenta in place (the new momentum state).
template <typename T>
struct HeviPre {
    static constexpr bool none = false;
    asuca_grid *g;
    asuca_state *st;
    asuca_acoustic_desc a;
    int ns;
    double dt;
    cudaStream_t s;
    char *ws;
    T *s_final;
    HeviLayout L;

    T *at(size_t off) const { return (T *)(ws + off); }

    cudaError_t operator()(int, int stg, StageParams<T> &sp) {
        if (stg < 0)
            return timed(g, ASUCA_KERNEL_ACOUSTIC, s, [&] {
                return launch_hevi_init<T>((const T *)st->rho, a.rho0c, at(L.Sn), g->d.nx, g->d.ny, g->d.nz, s);
            });
        const double w = stg == 0 ? dt / 3.0 : (stg == 1 ? dt / 2.0 : dt);
        const int nq = hevi_short_steps(ns, stg);
        const double h = w / nq;
        T *U0 = (T *)const_cast<void *>(st->mu), *V0 = (T *)const_cast<void *>(st->mv),
          *W0 = (T *)const_cast<void *>(st->mw);
        T *Uq = stg < 2 ? at(L.Ua) : U0, *Vq = stg < 2 ? at(L.Va) : V0, *Wq = stg < 2 ? at(L.Wa) : W0;
        T *Sq = (stg == 2 && s_final) ? s_final : at(L.Sa);
        AcousticParams<T> p[2];
        for (int q = 0; q < 2; q++) {
            std::memset(&p[q], 0, sizeof(p[q]));
            p[q].Us = at(L.Us);
            p[q].Vs = at(L.Vs);
            p[q].Ws = at(L.Ws);
            p[q].Ss = at(L.Ss);
            p[q].Uo = Uq;
            p[q].Vo = Vq;
            p[q].Wo = Wq;
            p[q].So = Sq;
            p[q].nx = g->d.nx;
            p[q].ny = g->d.ny;
            p[q].nz = g->d.nz;
            p[q].plane = (unsigned)g->plane;
            p[q].rdx = (T)(1.0 / g->d.dx);
            p[q].rdy = (T)(1.0 / g->d.dy);
            acoustic_tables<T>(g, a, q == 0 ? 0.5 * h : h, p[q]);
        }
        p[1].Mu = at(L.Mu);
        p[1].Mv = at(L.Mv);
        p[1].Mw = at(L.Mw);
        p[1].wacc = (T)(1.0 / nq);
        p[1].wlo = (T)((1.0 - a.beta) / nq);
        p[1].whi = (T)(a.beta / nq);
        for (int m = 0; m < nq; m++) {
            for (int q = 0; q < 2; q++) {
                p[q].U = m == 0 ? U0 : Uq;
                p[q].V = m == 0 ? V0 : Vq;
                p[q].W = m == 0 ? W0 : Wq;
                p[q].S = m == 0 ? at(L.Sn) : Sq;
            }
            p[1].acc_init = m == 0;
            for (int q = 0; q < 2; q++) {
                const cudaError_t e =
                    timed(g, ASUCA_KERNEL_ACOUSTIC, s, [&] { return launch_acoustic_stage<T>(p[q], q + 1, s); });
                if (e != cudaSuccess) return e;
            }
        }
        sp.mu = at(L.Mu);
        sp.mv = at(L.Mv);
        sp.mw = at(L.Mw);
        return cudaSuccess;
    }
};

template <typename T>
cudaError_t run_acoustic(const asuca_grid *g, void *U, void *V, void *W, void *S, const asuca_acoustic_desc &a,
                         double h, int nshort, char *ws, cudaStream_t s) {
    const size_t plane = (size_t)g->plane;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t fb = al(plane * g->d.nz * sizeof(T));
    AcousticParams<T> p[2];
    for (int q = 0; q < 2; q++) {
        std::memset(&p[q], 0, sizeof(p[q]));
        p[q].U = (T *)U;
        p[q].V = (T *)V;
        p[q].W = (T *)W;
        p[q].S = (T *)S;
        p[q].Uo = (T *)U;
        p[q].Vo = (T *)V;
        p[q].Wo = (T *)W;
        p[q].So = (T *)S;
        p[q].Us = (T *)ws;
        p[q].Vs = (T *)(ws + fb);
        p[q].Ss = (T *)(ws + 2 * fb);
        p[q].Ws = (T *)(ws + 3 * fb);
        p[q].nx = g->d.nx;
        p[q].ny = g->d.ny;
        p[q].nz = g->d.nz;
        p[q].plane = (unsigned)plane;
        p[q].rdx = (T)(1.0 / g->d.dx);
        p[q].rdy = (T)(1.0 / g->d.dy);
        acoustic_tables<T>(g, a, q == 0 ? 0.5 * h : h, p[q]);
    }
    for (int n = 0; n < nshort; n++)
        for (int q = 0; q < 2; q++) {
            const cudaError_t e = launch_acoustic_stage<T>(p[q], q + 1, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}
}  // namespace

extern "C" {

asuca_status asuca_acoustic_steps(asuca_grid *g, void *U, void *V, void *W, void *S, const asuca_acoustic_desc *desc,
                                  double dtau, int nshort, void *workspace, size_t workspace_bytes,
                                  void *cuda_stream) {
    if (!g || !U || !V || !W || !S || !desc || !desc->rho0c || !desc->rho0f || !std::isfinite(dtau) || dtau < 0.0 ||
        nshort < 0 || !std::isfinite(desc->cs2) || desc->cs2 <= 0.0 || !(desc->beta >= 0.5 && desc->beta <= 1.0))
        return ASUCA_ERR_ARG;
    const int nz = g->d.nz;
    for (int k = 0; k < nz; k++)
        if (!(desc->rho0c[k] > 0.0) || !std::isfinite(desc->rho0c[k])) return ASUCA_ERR_ARG;
    for (int f = 1; f < nz; f++)
        if (!(desc->rho0f[f] > 0.0) || !std::isfinite(desc->rho0f[f])) return ASUCA_ERR_ARG;
    if (!workspace || workspace_bytes < asuca_acoustic_workspace_bytes(g) || ((uintptr_t)workspace & 255))
        return ASUCA_ERR_WORKSPACE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ASUCA_ERR_CUDA;
    if (dev != g->device) return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    if (nshort == 0) return ASUCA_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const cudaError_t e = g->d.prec == ASUCA_FP64
                              ? run_acoustic<double>(g, U, V, W, S, *desc, dtau, nshort, (char *)workspace, s)
                              : run_acoustic<float>(g, U, V, W, S, *desc, dtau, nshort, (char *)workspace, s);
    return cuda_status(e);
}

size_t asuca_hevi_workspace_bytes(const asuca_grid *g) { return g ? hevi_layout(g).total : 0; }

asuca_status asuca_step_hevi(asuca_grid *g, asuca_state *st, const void *tend, double dt, int nsteps,
                             const asuca_acoustic_desc *desc, int nshort, void *s_final, void *workspace,
                             size_t workspace_bytes, double *budgets, void *cuda_stream) {
    if (!g || !state_ok(g, st) || nsteps < 0 || !std::isfinite(dt) || dt < 0.0 || nshort < 1 || !desc ||
        !desc->rho0c || !desc->rho0f || !std::isfinite(desc->cs2) || desc->cs2 <= 0.0 ||
        !(desc->beta >= 0.5 && desc->beta <= 1.0))
        return ASUCA_ERR_ARG;
    const int nz = g->d.nz;
    for (int k = 0; k < nz; k++)
        if (!(desc->rho0c[k] > 0.0) || !std::isfinite(desc->rho0c[k])) return ASUCA_ERR_ARG;
    for (int f = 1; f < nz; f++)
        if (!(desc->rho0f[f] > 0.0) || !std::isfinite(desc->rho0f[f])) return ASUCA_ERR_ARG;
    asuca_status prev = take_status(g);
    if (prev != ASUCA_OK) return prev;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g->last_stream = s;
    if (nsteps == 0 && !budgets) return ASUCA_OK;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < hevi_layout(g).total)
        return ASUCA_ERR_WORKSPACE;
    char *ws = (char *)workspace;
    if (g->d.prec == ASUCA_FP64) {
        HeviPre<double> pre{g, st, *desc, nshort, dt, s, ws, (double *)s_final, hevi_layout(g)};
        return run_step<double, HeviPre<double>>(g, st, tend, dt, nsteps, ws, budgets, s, true, pre);
    }
    HeviPre<float> pre{g, st, *desc, nshort, dt, s, ws, (float *)s_final, hevi_layout(g)};
    return run_step<float, HeviPre<float>>(g, st, tend, dt, nsteps, ws, budgets, s, true, pre);
}

asuca_status asuca_profile_read(asuca_grid *g, double *ms, int *launches, int nkinds) {
    if (!g || !ms || !launches || nkinds <= 0) return ASUCA_ERR_ARG;
    for (int k = 0; k < nkinds; k++) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    if (g->prof_used > 0 && cudaEventSynchronize(g->prof_ev[2 * g->prof_used - 1]) != cudaSuccess)
        return ASUCA_ERR_CUDA;
    for (int q = 0; q < g->prof_used; q++) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g->prof_ev[2 * q], g->prof_ev[2 * q + 1]) != cudaSuccess)
            return ASUCA_ERR_CUDA;
        const int k = g->prof_kind[q];
        if (k >= 0 && k < nkinds) {
            ms[k] += t;
            launches[k] += 1;
        }
    }
    g->prof_used = 0;
    return ASUCA_OK;
}

}  // extern "C"
