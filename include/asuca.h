/* libasuca -- C ABI of the GB300-native ASUCA-style time step.
 *
 * The computation is the structured-grid weather step the Hybrid Fortran
 * paper ports to GPUs (arXiv 1710.08616): a finite-volume scheme on a
 * rectangular grid advanced by Wicker-Skamarock RK3 (Sec. 1.1 "ASUCA on
 * GPU"), parallel over the horizontal I/J columns with the K column marched
 * in one thread (Sec. 1.1, Sec. 1.3 "Memory Layout"), followed by per-column
 * physics applied at column granularity (Sec. 1.2 "Parallelization
 * Granularity"; Fig. 1 and 2).  The paper prints no operator, so the
 * operators are the textbook ones named here:
 *   - prognostic fields rho, rho*theta, rho*q_1..N in flux form on an
 *     Arakawa-C grid, periodic in i and j, rigid lids (zero flux) in k;
 *   - face values from the Koren limiter (or the unlimited kappa = 1/3
 *     scheme, or first-order upwind) on the side the face mass flux comes
 *     from (M = 0 counts as M >= 0), vertical ghost levels copying the
 *     boundary cell;
 *   - RK3 stages Y* = Yn + dt/3 R(Yn), Y** = Yn + dt/2 R(Y*),
 *     Yn+1 = Yn + dt R(Y**), R = -div(M phi_face) + tendency;
 *   - then, per column: implicit theta relaxation to 300 + 0.004 z K,
 *     top-down implicit sedimentation of one tracer, and implicit vertical
 *     diffusion of theta and every q by a Thomas solve whose factorisation
 *     is shared by all fields (FP64 in both precisions);
 *   - FP64 budgets: total mass, rho*theta, each tracer, precipitation.
 *
 * Memory and streams belong to the caller.  Every device pointer is
 * caller-owned device memory; the library never allocates device memory
 * (it allocates a few bytes of pinned host memory per grid for its status
 * word).  Every call is asynchronous on the given CUDA stream (NULL = the
 * legacy default stream).  Argument errors are returned synchronously;
 * errors found on the device (non-finite budgets, a barrier that timed out)
 * are written to the grid's status word and returned by the next call on
 * that grid or by asuca_get_status().
 *
 * Field layout: every 3D field is [nz][ny][nx] with i fastest and no
 * padding ("IJK" order of Sec. 1.3).  rhoq holds the N tracer fields back
 * to back ([N][nz][ny][nx]).  mu[k][j][i] is the mass flux through face
 * i+1/2, mv[k][j][i] through face j+1/2, and mw ([nz+1][ny][nx]) through the
 * face below cell k; mw[0] and mw[nz] are the lids and are never read.
 * The element type of every field is double for ASUCA_FP64 and float for
 * ASUCA_FP32_MIXED.
 */
#ifndef ASUCA_H
#define ASUCA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASUCA_MAX_TRACERS 8
#define ASUCA_MAX_NZ 128

typedef enum {
    ASUCA_OK = 0,
    ASUCA_ERR_ARG = 1,          /* invalid argument (returned synchronously) */
    ASUCA_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    ASUCA_ERR_WORKSPACE = 3,    /* workspace missing, misaligned or too small */
    ASUCA_ERR_NONFINITE = 4,    /* a budget sum was NaN or infinite */
    ASUCA_ERR_TIMEOUT = 5,      /* a device-wide barrier gave up waiting */
    ASUCA_ERR_UNSUPPORTED = 6,  /* sizes beyond the compiled limits */
    ASUCA_ERR_BOUNDS = 7        /* a kernel index fell outside its buffer (recorded only by the
                                   bounds-check build, see asuca_bounds_checked) */
} asuca_status;

typedef enum {
    ASUCA_FP64 = 0,             /* every operation in double */
    ASUCA_FP32_MIXED = 1        /* float fields and stencils; double Thomas solve and sums */
} asuca_precision;

typedef enum {
    ASUCA_LIM_KOREN = 0,        /* psi(r) = max(0, min(2r, (1 + 2r)/3, 2)) */
    ASUCA_LIM_LINEAR = 1,       /* unlimited kappa = 1/3 upwind-biased face value */
    ASUCA_LIM_UPWIND1 = 2       /* first-order upwind */
} asuca_limiter;

typedef enum {
    ASUCA_OP_STEP = 0,
    ASUCA_OP_ADJOINT = 1,
    ASUCA_OP_ENSEMBLE = 2
} asuca_op;

typedef struct {
    int nx, ny, nz;             /* nx, ny >= 4; 3 <= nz <= ASUCA_MAX_NZ */
    int ntracers;               /* 0 .. ASUCA_MAX_TRACERS */
    double dx, dy;              /* horizontal spacing (m), > 0 */
    const double *dz;           /* host array of nz layer depths (m), > 0; copied */
    double tau_theta;           /* theta relaxation time (s); 0 disables it */
    double k0, k_h;             /* K(z) = k0 exp(-z / k_h) (m^2/s); k0 = 0 disables diffusion */
    double v_sed;               /* fall speed (m/s); 0 disables sedimentation */
    int sed_tracer;             /* index of the sedimenting tracer; -1 = none */
    asuca_limiter lim;
    asuca_precision prec;
} asuca_grid_desc;

typedef struct asuca_grid asuca_grid;   /* opaque, host side */

typedef struct {
    void *rho, *rhotheta, *rhoq;        /* updated in place */
    const void *mu, *mv, *mw;           /* steady mass fluxes */
} asuca_state;

/* Create a grid: validates the description, copies dz, precomputes level
 * tables.  *out receives the grid; free it with asuca_free_grid.
 * ASUCA_ERR_ARG for nx, ny < 4, nz < 3, non-positive or non-finite spacings
 * or constants, an out-of-range tracer, limiter or precision;
 * ASUCA_ERR_UNSUPPORTED beyond the compiled limits: N > ASUCA_MAX_TRACERS,
 * nz > ASUCA_MAX_NZ, or a field (nx * ny * (nz + 1) elements, or its padded
 * stage copy (nx + 8 rounded up to 8) * (ny + 4) * nz) of 2^32 elements or
 * more, since the kernels index within a field with 32-bit offsets. */
asuca_status asuca_init_grid(const asuca_grid_desc *desc, asuca_grid **out);
asuca_status asuca_free_grid(asuca_grid *grid);

/* Bytes of device workspace op needs (256-byte aligned pointer required).
 * ASUCA_OP_STEP: two stage states plus the column-solve scratch (and, with
 * the fused column pass of ASUCA_TUNE_FUSED_COLUMN, its (F + 2) nz ny nx
 * doubles), per-column precipitation and budget partials.  ASUCA_OP_ADJOINT: param = nsteps with
 * checkpoints every 10 steps (asuca_adjoint_workspace_bytes takes any
 * interval).  Returns 0 for an invalid grid or op. */
size_t asuca_workspace_bytes(const asuca_grid *grid, int op, int param);

/* Advance the state by nsteps RK3 steps, each followed by the column physics
 * (Sec. 1.1 RK3 long step; Sec. 1.2 column processes).  tendencies, if not
 * NULL, are 1+N fields ([1+N][nz][ny][nx], rho*theta then the tracers) of
 * constant forcing added in every stage.  budgets_dev, if not NULL, receives
 * N+3 doubles on the device: total mass, total rho*theta, each tracer's
 * total (all sum(field * dz * dx * dy)) after the last step, and the
 * precipitation accumulated over these nsteps.  nsteps = 0 only computes
 * the budgets. */
asuca_status asuca_step(asuca_grid *grid, asuca_state *state, const void *tendencies, double dt,
                        int nsteps, void *workspace, size_t workspace_bytes, double *budgets_dev,
                        void *cuda_stream);

/* Workspace of asuca_adjoint_step: the step workspace, ceil(nsteps / K)
 * checkpoints, one segment of K recorded steps (stage states, limiter
 * branches, the face values of every stage and the column pass's
 * factorisation and solution), two such segments when there are several
 * (see asuca_adjoint_step), four adjoint fields and the column-transpose
 * scratch. */
size_t asuca_adjoint_workspace_bytes(const asuca_grid *grid, int nsteps, int checkpoint_every);

/* Adjoint (vector-Jacobian product) of nsteps calls of asuca_step's time
 * step, the gradient engine of a 4D-Var-style assimilation: given
 * lambda_final = dJ/dY_final ([F][nz][ny][nx], F = 2 + N fields in the
 * order rho, rho*theta, rho*q), it returns grad_initial = dJ/dY_initial
 * ([F][nz][ny][nx]) and the gradients with respect to the mass fluxes
 * (grad_mu, grad_mv [nz][ny][nx], grad_mw [nz+1][ny][nx]; the lid entries
 * of grad_mw are zero), all treated as independent inputs.  The forward
 * trajectory is recomputed from `initial` (not modified): states are kept
 * every checkpoint_every steps, and each segment is recomputed once more
 * while recording the stage states and the limiter branch of every face,
 * then reversed step by step (column transpose, then the three stage
 * transposes).  Tendencies enter the trajectory but are not differentiated.
 * Element types follow the grid's precision; the column transpose uses
 * double for its tridiagonal solves in both precisions. */
asuca_status asuca_adjoint_step(asuca_grid *grid, const asuca_state *initial, const void *tendencies, double dt,
                                int nsteps, int checkpoint_every, const void *lambda_final, void *grad_initial,
                                void *grad_mu, void *grad_mv, void *grad_mw, void *workspace,
                                size_t workspace_bytes, void *cuda_stream);

/* Bytes of the checkpoint buffer of asuca_forward_checkpointed:
 * ceil(nsteps / checkpoint_every) states of F fields, each rounded up to
 * 256 bytes.  0 for nsteps = 0 or an invalid argument. */
size_t asuca_checkpoint_bytes(const asuca_grid *grid, int nsteps, int checkpoint_every);

/* The forward half of checkpointed differentiation: advances `state` by
 * nsteps exactly as asuca_step does (same kernels, bit-identical result and
 * budgets) and keeps the state before steps 0, K, 2K, ... (K =
 * checkpoint_every) in `checkpoints` (device, 256-byte aligned, at least
 * asuca_checkpoint_bytes; block c holds the F fields [F][nz][ny][nx] of
 * step c K).  A later asuca_adjoint_from_checkpoints then recomputes only
 * within segments, so the reverse pass does not repeat the forward run.
 * The workspace is asuca_step's.  ASUCA_ERR_ARG for a missing or short
 * checkpoint buffer. */
asuca_status asuca_forward_checkpointed(asuca_grid *grid, asuca_state *state, const void *tendencies, double dt,
                                        int nsteps, int checkpoint_every, void *checkpoints,
                                        size_t checkpoint_bytes, void *workspace, size_t workspace_bytes,
                                        double *budgets_dev, void *cuda_stream);

/* The reverse half: the same result as asuca_adjoint_step (bit for bit),
 * starting from the checkpoints an asuca_forward_checkpointed call with the
 * same grid, fluxes, tendencies, dt, nsteps and checkpoint_every kept.
 * Only fluxes->mu, mv, mw are read.  Each segment is recomputed once while
 * recording stage states and limiter branches, then reversed.  The
 * workspace is asuca_adjoint_workspace_bytes(grid, nsteps, K) bytes
 * (its checkpoint area is left unused). */
asuca_status asuca_adjoint_from_checkpoints(asuca_grid *grid, const void *checkpoints, const asuca_state *fluxes,
                                            const void *tendencies, double dt, int nsteps, int checkpoint_every,
                                            const void *lambda_final, void *grad_initial, void *grad_mu,
                                            void *grad_mv, void *grad_mw, void *workspace, size_t workspace_bytes,
                                            void *cuda_stream);

/* Both adjoint entries recompute segment c - 1 on a stream of the grid's own
 * (made by asuca_init_grid) while cuda_stream reverses segment c; that
 * stream waits for the work cuda_stream holds when the call begins, and
 * cuda_stream waits for all of it before the call's last operation, so the
 * call orders on cuda_stream like any other (also inside a stream capture).
 * Calls on one grid must not run concurrently. */

/* ---- ensemble -------------------------------------------------------------
 * Members are grids with the same nz, number of tracers, precision and
 * limiter and any horizontal size; they are advanced together by one
 * persistent cooperative kernel per call (three stage phases, the second and
 * third carrying the top-down half of the column pass, and one
 * back-substitution phase per step, each phase a flattened list of (member, tile) or (member,
 * column) work items, separated by device-wide barriers whose waits give up
 * after about one second and report ASUCA_ERR_TIMEOUT).  Members never share
 * a tile, so every member's result equals asuca_step on that member alone.
 * On a non-default stream that is not already being captured, the launch
 * sequence of a call (parameter upload, resets, the persistent kernel, the
 * per-member budget kernels) is captured once into a CUDA graph, cached by
 * its arguments (up to four), and replayed by later calls with the same
 * arguments. */
size_t asuca_ensemble_workspace_bytes(asuca_grid *const *grids, int nmembers);

/* states[m] and dts[m] belong to grids[m]; budgets_dev, if not NULL, receives
 * nmembers x (N + 3) doubles, member-major, as for asuca_step. */
asuca_status asuca_ensemble_step(asuca_grid *const *grids, asuca_state *states, const double *dts, int nmembers,
                                 int nsteps, void *workspace, size_t workspace_bytes, double *budgets_dev,
                                 void *cuda_stream);

/* ---- tuning knobs (set by the autotuner) --------------------------------- */
typedef enum {
    ASUCA_TUNE_COL_BLOCKS_PER_SM = 0,   /* resident column-kernel blocks per SM (1..16); sizes the column scratch */
    ASUCA_TUNE_BARRIER_EXTRA = 1,       /* test hook: the ensemble barrier waits for this many extra CTAs (0) */
    ASUCA_TUNE_STAGE_TILE_ROWS = 2,     /* stage tile 32 x rows: 4, 8 (default) or 16 for FP32; 8 for FP64 */
    ASUCA_TUNE_ENSEMBLE_TILE_ROWS = 3,  /* ensemble tile 32 x rows: 4 or 8 (default) for FP32; 8 for FP64 */
    ASUCA_TUNE_STEP_MODE = 4            /* asuca_step: 0 one launch per stage and column pass; 1 one persistent
                                           dataflow launch per 16 steps (tasks wait on per-tile counters, so the
                                           FP64 column work overlaps the stencil stages); sizes the workspace */,
    ASUCA_TUNE_FUSED_COLUMN = 5         /* asuca_step with step mode 0 and diffusion on: 1 (default) carries the
                                           top-down half of the column pass in the stage kernels, marching
                                           downward: the second stage computes the FP64 factorisation from the
                                           density after the step, the third the relaxation, sedimentation and
                                           elimination sweep (the nested acoustic step, whose mass fluxes change
                                           per stage, keeps the whole top-down half in the third stage), then a
                                           bottom-up back-substitution kernel; 0 runs the stages and the column
                                           pass as separate launches.  Results are bit-identical; 1 adds
                                           (F + 2) nz ny nx doubles of scratch to the workspace */
} asuca_tune_key;
asuca_status asuca_set_tuning(asuca_grid *grid, int key, int value);
int asuca_get_tuning(const asuca_grid *grid, int key);

/* Synchronise the stream of the last call on this grid, return and clear
 * the device status word (ASUCA_OK when no device error was recorded). */
asuca_status asuca_get_status(asuca_grid *grid);
const char *asuca_status_string(asuca_status s);

/* 1 when this library is the bounds-check build (compiled with
 * ASUCA_BOUNDS_CHECK), else 0.  In that build the step's kernels (the stage
 * kernels, the branch-recording stage, the column hooks of the stages, the
 * column passes, also inside the ensemble kernel) test each global-memory
 * index, and each offset into the stage's shared-memory ring, against its
 * buffer's extent before the access; an index outside the buffer records
 * ASUCA_ERR_BOUNDS in the device status word (asuca_get_status) and the
 * access is redirected to the buffer's first element, so the kernel neither
 * traps nor touches memory outside the buffer.  The results of a call that
 * recorded ASUCA_ERR_BOUNDS are meaningless.  Built on request
 * (paper_1710_08616_gb300.build.build(bounds_check=True)) as libasuca_bc.so;
 * it is slower and meant for tests on small cases. */
int asuca_bounds_checked(void);

/* ---- sub-steps, exported for per-kernel parity tests ------------------ */

/* One RK stage: out = base + cdt * R(in), with M taken from in.  in, base
 * and out may alias only as in == base (a forward-Euler stage). */
asuca_status asuca_debug_stage(asuca_grid *grid, const asuca_state *in, const asuca_state *base,
                               asuca_state *out, const void *tendencies, double cdt,
                               void *cuda_stream);

/* The column pass alone (relaxation, sedimentation, diffusion) at step dt.
 * precip_col_dev ([ny][nx] doubles) is incremented by each column's
 * precipitation (dt * P_bottom * dx * dy). */
asuca_status asuca_debug_column(asuca_grid *grid, asuca_state *state, double dt,
                                double *precip_col_dev, void *workspace, size_t workspace_bytes,
                                void *cuda_stream);

/* nsteps forward steps from `initial` (not modified) that write the limiter
 * branch of every face of every RK stage to branches_dev, laid out
 * [nsteps][3][F-1][nz][ny][nx], one byte per cell and field with 2 bits per
 * direction (bits 0-1 face i+1/2, 2-3 face j+1/2, 4-5 face k+1/2; 0 zero,
 * 1 "2r", 2 "kappa=1/3", 3 "cap 2").  Used to tell whether a perturbed
 * trajectory crosses a limiter kink.  Workspace: asuca_adjoint_workspace_bytes(grid, 1, 1). */
asuca_status asuca_debug_record_branches(asuca_grid *grid, const asuca_state *initial, const void *tendencies,
                                         double dt, int nsteps, unsigned char *branches_dev, void *workspace,
                                         size_t workspace_bytes, void *cuda_stream);

/* Host-only test hook: the task order of the dataflow step kernel for
 * nphases phases (4 per step, at most 64) on nrows tile rows; out receives
 * nphases * nrows entries (phase << 12) | row. */
asuca_status asuca_debug_dataflow_order(int nphases, int nrows, unsigned *out);

/* Test hook for the arithmetic helpers of the column solve (device arrays of
 * n values; any output may be NULL): widen[i] = in_f[i] as double, narrow[i]
 * = in_d[i] rounded to float (nearest-even), both computed on the integer
 * pipe from the IEEE-754 bit fields; rcp[i] = 1 / in_d[i] from a float
 * reciprocal seed and one third-order correction (within an ulp; |in_d| in
 * the float normal range). */
asuca_status asuca_debug_numerics(const float *in_f, const double *in_d, int n, double *widen,
                                  float *narrow, double *rcp, void *cuda_stream);

/* ---- column pass without a workspace ------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory, e.g. a host model whose memory pool is fixed
 * at start-up, or a caller in the middle of capturing a stream, where
 * cudaMalloc is not allowed.  It runs the same column pass as
 * asuca_debug_column (relaxation, sedimentation, implicit vertical
 * diffusion with the FP64 Thomas solve) on the caller's state and adds each
 * column's precipitation to precip_col_dev ([ny][nx] doubles), but it takes
 * no workspace: the solve's scratch is a 16 MiB array compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.  It allocates nothing: no cudaMalloc, cudaFree or allocating
 * library call.
 *   - The scratch is looked up (cudaGetSymbolAddress) on the first call on
 *     each device, with that device current; make that first call before
 *     any stream capture.  The grid's device must be the current device.
 *   - The launch uses as many 128-column blocks as fit in the array
 *     (nz * (F + 1) * 128 * 8 bytes each; at least eleven within the compiled
 *     limits of nz and tracers); a size whose single block would not fit is
 *     rejected with ASUCA_ERR_UNSUPPORTED.
 *   - All calls on a device share the array and it keeps the last call's
 *     contents (every value is written before it is read, nothing needs to
 *     start at zero).  Calls that overlap on the GPU (on different streams
 *     without ordering) race on it and give wrong results. */
asuca_status asuca_column_noalloc(asuca_grid *grid, asuca_state *state, double dt,
                                  double *precip_col_dev, void *cuda_stream);

/* ---- storage-order experiment ------------------------------------------
 * One explicit 7-point diffusion step, the kernel of the reduced weather
 * application of Sec. 4 ("Productivity- and Performance Results"), run with
 * the same thread mapping on two storage orders, to measure the effect Sec. 1.3
 * ("Memory Layout") reports (KIJ order 7.7x slower than IJK on GPU):
 *   out = in + c (in(i-1) + in(i+1) + in(j-1) + in(j+1) + in(k-1) + in(k+1) - 6 in),
 * periodic in i and j, zero flux through the lids (ghost levels copy the
 * boundary cell).  layout 0 (IJK): element (i, j, k) at (k ny + j) nx + i;
 * layout 1 (KIJ): at (j nx + i) nz + k.  in and out are caller-owned device
 * arrays of nx ny nz elements of the precision's type (double for ASUCA_FP64,
 * float for ASUCA_FP32_MIXED) and must not overlap.  Asynchronous on the
 * stream; ASUCA_ERR_ARG for null or equal pointers, nx, ny < 2, nz < 1, or an
 * unknown layout or precision. */
asuca_status asuca_stencil7(const void *in, void *out, int nx, int ny, int nz, int layout, int prec, double c,
                            void *cuda_stream);

/* ---- lateral and upper damping -----------------------------------------
 * Relaxation of the prognostic fields toward boundary data in a damping zone,
 * the kernel Sec. 2.1 ("Parallel Loop Abstraction") takes from the dynamical
 * core: the damping target is the reference state plus the boundary
 * perturbation interpolated in time between two boundary datasets,
 *   ptb_damp = mtratio (ref + bnd0) + tratio (ref + bnd1) - ref,
 *   target   = ref + ptb_damp,
 * (mtratio = 1 - tratio for an interpolation at the fraction tratio of the
 * boundary interval), and every field relaxes toward it implicitly:
 *   y <- (y + a target) / (1 + a),   a = dt nu(i, j, k),
 *   nu = max(nu_lat w_lat, nu_top w_top),
 *   w_lat = ((width - d) / width)^2 for d < width, d = min(i, nx-1-i, j, ny-1-j),
 *   w_top = ((k - (nz - ntop) + 1) / ntop)^2 on the top ntop levels,
 * both zero elsewhere.  Cells outside the zone are not read or written.
 * The paper prints the target formula only; the relaxation form and the
 * quadratic profiles are this library's choice.
 *   - state: the grid's fields (rho, rho theta, rho q; mu, mv, mw unused),
 *     updated in place; ref, bnd0, bnd1: caller-owned device arrays of
 *     [F][nz][ny][nx] values in the grid's precision, F = 2 + N in the order
 *     rho, rho theta, tracers (conserved variables, like the state).
 *   - 0 <= width <= ASUCA_DAMP_MAX_WIDTH, 2 width <= min(nx, ny);
 *     0 <= ntop <= nz; nu_lat, nu_top, dt >= 0 and finite; mtratio, tratio
 *     finite.  Otherwise (or a null pointer) ASUCA_ERR_ARG.
 *   - Asynchronous on the stream; the grid's device must be current. */
#define ASUCA_DAMP_MAX_WIDTH 64
typedef struct {
    int width;       /* lateral zone: cells fewer than `width` cells from an i or j edge */
    int ntop;        /* upper zone: the top ntop levels */
    double nu_lat;   /* damping rate (1/s) at the outermost cells */
    double nu_top;   /* damping rate (1/s) at the top level */
} asuca_damping_desc;

asuca_status asuca_damping(asuca_grid *grid, asuca_state *state, const void *ref, const void *bnd0,
                           const void *bnd1, double mtratio, double tratio, double dt,
                           const asuca_damping_desc *desc, void *cuda_stream);

/* Host-only views of the zone asuca_damping touches (no device work): the
 * number of zone cells (0 for arguments asuca_damping would reject), and the
 * kernel's enumeration of them.  ijk: caller-owned host array of 3 n
 * unsigned values, (i, j, k) of the zone's cells in the order the kernel's
 * flat index visits them; n must equal the zone's cell count, else
 * ASUCA_ERR_ARG. */
size_t asuca_damping_zone_cells(int nx, int ny, int nz, int width, int ntop);
asuca_status asuca_debug_damping_cells(int nx, int ny, int nz, int width, int ntop, unsigned *ijk, size_t n);

/* ---- HEVI acoustic short steps ------------------------------------------
 * Sound and gravity waves advanced in short steps by a two-stage Runge-Kutta
 * scheme, horizontally explicit and vertically implicit (Sec. 1.1, "ASUCA on
 * GPU"), for the linear acoustic-gravity system about a resting, horizontally
 * uniform base state rho0(z):
 *   dU/dt = -c^2 rho0_k (s_{i+1} - s_i)/dx,  dV/dt = -c^2 rho0_k (s_{j+1} - s_j)/dy,
 *   dW_f/dt = -c^2 rho0f_f (s_f - s_{f-1})/dzc_f,  dzc_f = (dz_{f-1} + dz_f)/2,
 *   rho0_k ds/dt = -[(U_{i+1/2} - U_{i-1/2})/dx + (V_{j+1/2} - V_{j-1/2})/dy + (W_{k+1} - W_k)/dz_k],
 * s = rho'/rho0 (for rho0 = rho_s exp(-g z / c^2) the W equation is
 * dW/dt = -dp'/dz - g rho').  A short step of length dtau: stage 1 over
 * dtau/2, U* = U - (dtau/2) G(s), then W*, s* from the implicit vertical
 * system with the horizontal divergence of U*, V*; stage 2 over dtau from the
 * same start, U+ = U - dtau G(s*), then W+, s+ implicit with the divergence
 * of U*, V*.  The implicit system weights the new and old vertical terms by
 * beta and 1 - beta (beta = 1/2: Crank-Nicolson; larger: damped).  The paper
 * names the scheme only; these equations are this library's reading.
 *   - U, V, S: [nz][ny][nx] (U at the faces i+1/2, V at j+1/2, S at the
 *     centres); W: [nz+1][ny][nx] (W[k] the face below cell k; W[0] and W[nz]
 *     are rigid lids, never read or written).  Device arrays of the grid's
 *     precision, updated in place; the grid's dx, dy, dz.
 *   - desc: rho0c (nz values) and rho0f (nz + 1, entries 1..nz-1 used), host
 *     arrays, > 0; cs2 > 0 the squared sound speed; 1/2 <= beta <= 1.
 *   - The FP64 path computes in double; the FP32 path in float, with the
 *     column systems' factorisation computed in double on the host.
 *   - workspace: asuca_acoustic_workspace_bytes(grid) bytes, 256-byte
 *     aligned, else ASUCA_ERR_WORKSPACE.  dtau >= 0, nshort >= 0, else (or a
 *     null pointer) ASUCA_ERR_ARG.  Two launches per short step, asynchronous
 *     on the stream. */
typedef struct {
    const double *rho0c;   /* nz base densities at the level centres */
    const double *rho0f;   /* nz + 1 base densities at the faces */
    double cs2;            /* squared sound speed (m^2/s^2) */
    double beta;           /* implicit weight */
} asuca_acoustic_desc;

size_t asuca_acoustic_workspace_bytes(const asuca_grid *grid);
asuca_status asuca_acoustic_steps(asuca_grid *grid, void *U, void *V, void *W, void *S,
                                  const asuca_acoustic_desc *desc, double dtau, int nshort, void *workspace,
                                  size_t workspace_bytes, void *cuda_stream);

/* ---- open lateral boundaries: limited-area domains, decomposed domains --
 * The periodic step's lateral wrap replaced by ghost cells: the edge cells'
 * lateral neighbours are two ghost columns (rows) per side, written from
 * outside the stage kernels, either from boundary data (a limited-area
 * domain: the boundary datasets of the damping kernel, Sec. 2.1 "Parallel
 * Loop Abstraction") or by a halo exchange between the blocks of a
 * horizontally decomposed domain (Sec. 1.1 "ASUCA on GPU": horizontal blocks
 * with halo communication; Sec. 2.2 "Device Data Region": halo updates every
 * time step).  The face reconstruction is the periodic step's, reading a ghost
 * wherever its four-cell stencil leaves the domain; the density needs no
 * ghost (its flux is M).  The stencil is a cross, so the ghost corners are
 * never read.
 *   - state: the block's or domain's fields as for asuca_step, but mu and mv
 *     are the open domain's face fluxes: mu [nz][ny][nx+1], entry i the face
 *     i-1/2 of cell i (i = nx: the east face of the last cell); mv
 *     [nz][ny+1][nx], entry j the face j-1/2; mw as for asuca_step.
 *   - Halo layout (received strips, boundary data, send buffers): four
 *     strips one after another, W and E ([F-1][nz][2][ny] each), then S and
 *     N ([F-1][nz][2][nx] each), for the F-1 quantities phi = rho phi / rho
 *     (theta, then the mixing ratios).  As ghosts, strip W holds the cells
 *     i = c-2, E i = nx+c, S j = c-2, N j = ny+c (c = 0, 1); as packed by
 *     asuca_halo_pack, strip W holds the block's cells i = c, E i = nx-2+c,
 *     S j = c, N j = ny-2+c, so a block's received W strip is its west
 *     neighbour's packed E strip, and so on.  asuca_halo_count gives the
 *     values of one such array, 2 (2 nx + 2 ny) nz (F-1).
 *   - workspace: asuca_open_workspace_bytes(grid) bytes, 256-byte aligned,
 *     else ASUCA_ERR_WORKSPACE; it holds the three padded stage inputs
 *     (buffer 0: phi^n, 1: phi*, 2: phi**), whose ghosts the calls below
 *     fill and read.  Halo and boundary arrays are caller-owned device arrays
 *     in the grid's precision.
 *   - One step is: asuca_open_prepare (buffer 0 from the state); fill buffer
 *     0's ghosts; asuca_open_stage 0; fill buffer 1's ghosts; stage 1; fill
 *     buffer 2's ghosts; stage 2 (the third stage, the column pass and, if
 *     budgets_dev is set, this block's budgets as for asuca_step, the
 *     precipitation summed since the last prepare with first_of_call set).
 *     Ghosts are filled with asuca_halo_unpack, from received strips (a
 *     decomposed domain: pack, exchange, unpack) or from boundary data.
 *     asuca_step_open runs whole steps of a limited-area domain, the
 *     boundary data held for the call.
 *   - Asynchronous on the stream; null pointers, a stage or buffer outside
 *     0..2, or a non-finite dt or tratio give ASUCA_ERR_ARG; a grid whose
 *     open face-flux arrays do not fit 32-bit offsets ASUCA_ERR_UNSUPPORTED. */
size_t asuca_open_workspace_bytes(const asuca_grid *grid);
size_t asuca_halo_count(const asuca_grid *grid);
/* buffer 0's interior = phi of the state; first_of_call != 0 also restarts
 * the precipitation sum of the budgets */
asuca_status asuca_open_prepare(asuca_grid *grid, const asuca_state *state, int first_of_call, void *workspace,
                                size_t workspace_bytes, void *cuda_stream);
/* RK stage `stage` (0, 1, 2: weights dt/3, dt/2, dt) from buffer `stage`
 * (ghosts filled); stages 0 and 1 write the interior of buffer stage+1,
 * stage 2 writes the state and runs the column pass */
asuca_status asuca_open_stage(asuca_grid *grid, asuca_state *state, const void *tendencies, double dt, int stage,
                              void *workspace, size_t workspace_bytes, double *budgets_dev, void *cuda_stream);
/* send: halo-layout array filled with the block's edge strips of buffer `buffer` */
asuca_status asuca_halo_pack(asuca_grid *grid, const void *workspace, size_t workspace_bytes, int buffer,
                             void *send, void *cuda_stream);
/* ghosts of buffer `buffer` = recv (bnd1 NULL), else (1 - tratio) recv + tratio bnd1 (two
 * boundary datasets interpolated in time) */
asuca_status asuca_halo_unpack(asuca_grid *grid, void *workspace, size_t workspace_bytes, int buffer,
                               const void *recv, const void *bnd1, double tratio, void *cuda_stream);
/* nsteps steps of a limited-area domain whose ghosts are (1 - tratio) bnd0 + tratio bnd1
 * (bnd1 may be NULL: bnd0 alone) in every stage */
asuca_status asuca_step_open(asuca_grid *grid, asuca_state *state, const void *tendencies, double dt, int nsteps,
                             const void *bnd0, const void *bnd1, double tratio, void *workspace,
                             size_t workspace_bytes, double *budgets_dev, void *cuda_stream);

/* ---- acoustic short steps nested in the RK3 long step -------------------
 * The two halves of the dynamical core together (Sec. 1.1 "ASUCA on GPU":
 * the long step by RK3, sound and gravity waves by the HEVI short steps):
 * the momenta are prognostic and the scalars are advected by them.  Wicker-
 * Skamarock splitting: RK stage q (weight c_q = 1/3, 1/2, 1) integrates the
 * acoustic system of asuca_acoustic_steps from t^n over c_q dt in
 * n_q = max(1, round(c_q nshort)) short steps of c_q dt / n_q, starting from
 * the momenta at t^n and s^n = rho^n / rho0c - 1 (the acoustic density
 * perturbation of the advected density), and the scalar stage
 * Y^(q) = Y^n + c_q dt R(Y^(q-1)) advects with the short steps' mean
 * effective mass fluxes (1/n_q) sum (U*, V*, (1 - beta) W + beta W'), the
 * fluxes whose divergence the acoustic density equation applies, so that the
 * advected density equals rho0c (1 + s) of the integration to rounding.  The
 * third stage's integration is the new momentum state.  Then the column pass
 * and budgets as asuca_step.  The coupling of the acoustic system to the
 * scalars beyond the density (a buoyancy from theta) is not modelled: the
 * base state is resting and horizontally uniform.
 *   - state: as for asuca_step, but mu, mv, mw are the prognostic momenta
 *     U, V ([nz][ny][nx], faces i+1/2, j+1/2) and W ([nz+1][ny][nx], the face
 *     below cell k; the lids are never read or written), updated in place.
 *   - desc: the acoustic base state and constants as for asuca_acoustic_steps;
 *     nshort >= 1 short steps per long step.
 *   - s_final: NULL, or a device array [nz][ny][nx] that receives s of the
 *     last step's third-stage integration.
 *   - workspace: asuca_hevi_workspace_bytes(grid) bytes, 256-byte aligned,
 *     else ASUCA_ERR_WORKSPACE.  Argument errors as asuca_step and
 *     asuca_acoustic_steps.  Asynchronous on the stream. */
size_t asuca_hevi_workspace_bytes(const asuca_grid *grid);
asuca_status asuca_step_hevi(asuca_grid *grid, asuca_state *state, const void *tendencies, double dt, int nsteps,
                             const asuca_acoustic_desc *desc, int nshort, void *s_final, void *workspace,
                             size_t workspace_bytes, double *budgets_dev, void *cuda_stream);

/* ---- per-kernel timing ------------------------------------------------- */

typedef enum {
    ASUCA_KERNEL_STAGE = 0,     /* one RK stage sweep */
    ASUCA_KERNEL_COLUMN = 1,    /* column physics + Thomas solve (+ budget partials) */
    ASUCA_KERNEL_REDUCE = 2,    /* final budget reduction */
    ASUCA_KERNEL_ADJ_STAGE = 3, /* transpose of one RK stage */
    ASUCA_KERNEL_ADJ_COLUMN = 4,/* transpose of the column pass */
    ASUCA_KERNEL_ENSEMBLE = 5,  /* persistent ensemble kernel (all steps of a call) */
    ASUCA_KERNEL_DATAFLOW = 6,  /* persistent dataflow step kernel (up to 16 steps) */
    ASUCA_KERNEL_STAGE_COLUMN = 7, /* third stage fused with the top-down column pass, or with its
                                      elimination sweep (its bottom-up half is counted as
                                      ASUCA_KERNEL_COLUMN) */
    ASUCA_KERNEL_ACOUSTIC = 8,  /* a stage of an acoustic short step nested in a long step (and the
                                   density perturbation it starts from) */
    ASUCA_KERNEL_STAGE_FACTOR = 9, /* second stage carrying the FP64 factorisation of the column pass */
    ASUCA_KERNEL_KINDS = 10
} asuca_kernel_kind;

/* When on, every kernel launch of later calls on this grid is bracketed by
 * two CUDA events on the call's stream (host-side event objects, created on
 * demand; no device memory).  Turning it on or off discards pending marks. */
asuca_status asuca_profile_enable(asuca_grid *grid, int on);

/* Wait for the last recorded event, then report per kernel kind the summed
 * event-measured duration (ms[kind]) and launch count since the last read;
 * clears the marks.  nkinds entries are written. */
asuca_status asuca_profile_read(asuca_grid *grid, double *ms, int *launches, int nkinds);

#ifdef __cplusplus
}
#endif
#endif
