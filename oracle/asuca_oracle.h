/* FP64 CPU oracle of the ASUCA-style step -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header or constant table with
 * the CUDA library; the two meet only through the seeded inputs of the
 * generator package.
 *
 * Field layout: the prognostic state Y is one array [F][nz][ny][nx] with
 * F = 2 + ntr fields in the order rho, rho*theta, rho*q_1 .. rho*q_ntr;
 * i is fastest.  mu[k][j][i] is the mass flux through face i+1/2,
 * mv[k][j][i] through face j+1/2, mw[k][j][i] (k = 0..nz) through the face
 * below cell k.  Tendencies, when given, are [F-1][nz][ny][nx] for
 * rho*theta and the tracers.
 */
#ifndef ASUCA_ORACLE_H
#define ASUCA_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz, ntr;
    double dx, dy;
    const double *dz;          /* nz layer depths */
    double tau;                /* theta relaxation time scale (s); 0 = off */
    double k0, kh;             /* K(z) = k0 exp(-z / kh); k0 = 0 = off */
    double vsed;               /* sedimentation speed (m/s); 0 = off */
    int sed;                   /* index of the sedimenting tracer; -1 = none */
    int lim;                   /* 0 Koren, 1 linear (kappa = 1/3), 2 first-order upwind */
} orc_grid;

/* limiter increment L(d0, d1); branch receives 0 zero, 1 "2r", 2 "kappa=1/3", 3 "cap 2" */
double orc_limiter(double d0, double d1, int lim, int *branch);
/* face value from the four cells around face i+1/2 (values at i-1, i, i+1, i+2) */
double orc_face(double pm1, double p0, double p1, double p2, double m, int lim, int *branch);

void orc_rhs(const orc_grid *g, const double *Y, const double *mu, const double *mv,
             const double *mw, const double *tend, double *R, unsigned char *branch);
void orc_euler(const orc_grid *g, const double *Y, const double *mu, const double *mv,
               const double *mw, const double *tend, double dt, double *out);
void orc_rk3(const orc_grid *g, double *Y, const double *mu, const double *mv,
             const double *mw, const double *tend, double dt);
void orc_column(const orc_grid *g, double *Y, double dt, double *precip_col);
void orc_thomas(int n, const double *a, const double *b, const double *c, const double *d,
                double *x);
void orc_budgets(const orc_grid *g, const double *Y, double precip, double *out);
void orc_step(const orc_grid *g, double *Y, const double *mu, const double *mv,
              const double *mw, const double *tend, double dt, int nsteps, double *budgets);
int orc_step_window(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                    const double *mw, const double *tend, double dt, int nsteps,
                    int i0, int j0, int w, int h, double *out);
/* tangent-linear and adjoint (limiter branches frozen at the forward values) */
void orc_rhs_tl(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                const double *mw, const double *dY, const double *dmu, const double *dmv,
                const double *dmw, double *dR);
void orc_rhs_adj(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                 const double *mw, const double *lamR, double *lamY, double *gmu, double *gmv,
                 double *gmw);
void orc_column_tl(const orc_grid *g, const double *Y3, const double *dY3, double dt, double *dOut);
void orc_column_adj(const orc_grid *g, const double *Y3, double *lam, double dt);
void orc_step_tl(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                 const double *mw, const double *tend, double dt, int nsteps, const double *dY0,
                 const double *dmu, const double *dmv, const double *dmw, double *dYn);
void orc_step_adj(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                  const double *mw, const double *tend, double dt, int nsteps,
                  const double *lam_final, double *lam0, double *gmu, double *gmv, double *gmw);
/* the same with the branch of every face fixed by the caller */
void orc_step_tl_br(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                    const double *mw, const double *tend, double dt, int nsteps, const double *dY0,
                    const double *dmu, const double *dmv, const double *dmw,
                    const unsigned char *traj_br, double *dYn);
void orc_step_adj_br(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                     const double *mw, const double *tend, double dt, int nsteps,
                     const double *lam_final, const unsigned char *traj_br, double *lam0,
                     double *gmu, double *gmv, double *gmw);
void orc_trajectory_branches(const orc_grid *g, const double *Y0, const double *mu,
                             const double *mv, const double *mw, const double *tend, double dt,
                             int nsteps, unsigned char *out);
/* Open (non-periodic) lateral boundaries: a limited-area domain or one block
 * of a decomposed domain.  ghost holds phi (fields 1..F-1) of the two ghost
 * columns/rows per side in the halo layout (strips W: i = c-2, E: i = nx+c,
 * S: j = c-2, N: j = ny+c, c = 0, 1; each [F-1][nz][2][len], len = ny, ny,
 * nx, nx); mu_x [nz][ny][nx+1] and mv_x [nz][ny+1][nx] hold the mass flux of
 * every face, index i (j) being face i-1/2 (j-1/2).  The ghosts are held for
 * the call. */
void orc_rhs_open(const orc_grid *g, const double *Y, const double *mu_x, const double *mv_x,
                  const double *mw, const double *tend, const double *ghost, double *R);
void orc_step_open(const orc_grid *g, double *Y, const double *mu_x, const double *mv_x, const double *mw,
                   const double *tend, const double *ghost, double dt, int nsteps, double *budgets);
/* One explicit step of 7-point diffusion (the reduced weather application's
 * kernel, Sec. 4): out = in + c (sum of the six neighbours - 6 in), periodic in
 * i and j, zero flux through both lids (ghost levels copy the boundary cell);
 * fields [nz][ny][nx]. */
void orc_stencil7(int nx, int ny, int nz, double c, const double *in, double *out);
/* Lateral and upper damping toward boundary data (Sec. 2.1, the damping
 * kernel): for each listed cell (i, j, k) and field f,
 *   ptb = mtratio (ref + b0) + tratio (ref + b1) - ref,  target = ref + ptb,
 *   y <- (y + a target) / (1 + a),  a = dt max(nu_lat w_lat, nu_top w_top),
 * w_lat = ((width - d) / width)^2 for d = min(i, nx-1-i, j, ny-1-j) < width,
 * w_top = ((k - (nz - ntop) + 1) / ntop)^2 for k >= nz - ntop, else 0.
 * ijk == NULL: every cell of the domain, arrays [F][nz][ny][nx] (ncell is
 * ignored); else ijk holds ncell (i, j, k) triples and the arrays are
 * [F][ncell], one column of values per listed cell. */
void orc_damping(int nx, int ny, int nz, int F, int width, int ntop, double nu_lat, double nu_top,
                 double mtratio, double tratio, double dt, long long ncell, const int *ijk, double *y,
                 const double *ref, const double *b0, const double *b1);
/* nshort HEVI short steps of the linear acoustic-gravity system (Sec. 1.1), in
 * place: U, V, S [nz][ny][nx] (U at faces i+1/2, V at j+1/2, S = rho'/rho0 at
 * the centres), W [nz+1][ny][nx] (face below cell k; W[0] and W[nz] are rigid
 * lids, never read, left as they are).  rho0c[nz], rho0f[nz+1] base density at
 * centres and faces, cs2 the squared sound speed, beta the implicit weight. */
void orc_acoustic(int nx, int ny, int nz, double dx, double dy, const double *dz, const double *rho0c,
                  const double *rho0f, double cs2, double beta, double h, int nshort, double *U, double *V,
                  double *W, double *S);
/* Short steps of RK stage q (0, 1, 2: weights 1/3, 1/2, 1) when a long step
 * has ns: max(1, round(weight ns)). */
int orc_hevi_short_steps(int ns, int q);
/* nsteps long steps with the acoustic short steps nested in every RK3 stage
 * (Wicker-Skamarock splitting): U, V [nz][ny][nx] and W [nz+1][ny][nx] are
 * the prognostic momenta (mass fluxes), updated in place; RK stage q
 * integrates them with orc_acoustic from t^n over its weight times dt, in
 * orc_hevi_short_steps(ns, q) short steps from s^n = rho^n / rho0c - 1, and
 * advects the scalars with the short steps' mean effective mass fluxes
 * (U*, V*, (1 - beta) W + beta W'); stage 3's integration is the new
 * momentum state (and s_final [nz][ny][nx], if set).  Then the column pass;
 * budgets as orc_step.  stage_rho, if set, receives the density of the first
 * two RK stages of the last step ([2][nz][ny][nx]). */
void orc_step_hevi(const orc_grid *g, double *Y, double *U, double *V, double *W, const double *tend,
                   const double *rho0c, const double *rho0f, double cs2, double beta, int ns, double dt,
                   int nsteps, double *s_final, double *budgets, double *stage_rho);
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
