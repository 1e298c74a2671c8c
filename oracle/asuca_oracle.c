/* FP64 CPU oracle of the ASUCA-style step -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow and written to be checked by eye against the scheme:
 *   - finite-volume flux form on a rectangular 2 km grid, time-stepped by the
 *     third-order Runge-Kutta scheme of Wicker and Skamarock (Sec. 1.1,
 *     "ASUCA on GPU"); the stage weights are 1/3, 1/2, 1;
 *   - horizontal (i, j) work is parallel, the K column is marched
 *     sequentially (Sec. 1.1 and Sec. 1.3, "Memory Layout");
 *   - physics is a per-column process applied once per long step
 *     (Sec. 1.2, "Parallelization Granularity"; Fig. 1 and 2).
 * The paper prints none of the operators below.  Each one is the textbook
 * scheme the specification names, in the reading stated beside it:
 *   - Koren limiter psi(r) = max(0, min(2r, (1 + 2r)/3, 2)) in
 *     division-free form with sign tests;
 *   - upwind side chosen by the sign of the face mass flux (M = 0 counts as
 *     M >= 0); vertical ghosts copy the boundary cell; both lids carry zero
 *     flux; the lateral boundaries are periodic;
 *   - implicit theta relaxation, top-down implicit sedimentation, implicit
 *     vertical diffusion by the Thomas algorithm (Lie splitting, in that
 *     order, after the three RK stages).
 * No closed form gives the full nonlinear Koren step on a large grid; it is
 * pinned through its parts and the invariants the test suite checks
 * (conservation, constant preservation, the Courant-1 shift, the linear
 * Fourier-mode closed form, Thomas vs dense LU, sedimentation closure,
 * relaxation fixed point), and the suite's mutation check plants slips in
 * copies of this file to show that each one fails a pin.
 *
 * Build: cc -O2 -fno-fast-math -ffp-contract=off [-fopenmp] -shared -fPIC.
 * OpenMP only splits independent cells or columns; every sum runs serially
 * in a fixed order, so results do not depend on the thread count.
 */
#include "asuca_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* reference theta profile of the relaxation term: 300 K + 4 K/km */
#define THETA_REF0 300.0
#define THETA_REF_LAPSE 0.004

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* ---------------------------------------------------------------- limiter */

double orc_limiter(double d0, double d1, int lim, int *branch) {
    int br;
    double L;
    if (lim == 2) {                       /* first-order upwind */
        br = 0;
        L = 0.0;
    } else if (lim == 1) {                /* unlimited kappa = 1/3 */
        br = 2;
        L = (d0 + 2.0 * d1) / 3.0;
    } else {
        /* Koren: zero unless d0 and d1 are both > 0 or both < 0 (sign
         * tests, not the product, so nothing underflows) */
        int same = (d0 > 0.0 && d1 > 0.0) || (d0 < 0.0 && d1 < 0.0);
        if (!same) {
            br = 0;
            L = 0.0;
        } else {
            double a0 = fabs(d0), a1 = fabs(d1);
            double t1 = 2.0 * a1;                 /* "2r" */
            double t2 = (a0 + 2.0 * a1) / 3.0;    /* kappa = 1/3 */
            double t3 = 2.0 * a0;                 /* cap at 2 */
            double m = t1;
            br = 1;
            if (t2 < m) { m = t2; br = 2; }       /* ties keep the earlier branch */
            if (t3 < m) { m = t3; br = 3; }
            L = d0 > 0.0 ? m : -m;
        }
    }
    if (branch) *branch = br;
    return L;
}

double orc_face(double pm1, double p0, double p1, double p2, double m, int lim, int *branch) {
    if (m >= 0.0) {
        double d0 = p0 - pm1, d1 = p1 - p0;
        return p0 + 0.5 * orc_limiter(d0, d1, lim, branch);
    } else {
        double d0 = p1 - p2, d1 = p0 - p1;
        return p1 + 0.5 * orc_limiter(d0, d1, lim, branch);
    }
}

/* ------------------------------------------------------------ patches
 * A patch is a rectangle of columns held in its own [F][nz][ph][pw] array.
 * The whole domain is the periodic patch; a window patch is not periodic and
 * is only evaluated where the stencil stays inside it. */
typedef struct {
    int pw, ph;     /* patch width (i) and height (j) */
    int gi0, gj0;   /* global index of local (0, 0) */
    int per;        /* 1: local indices wrap (whole periodic domain) */
} patch;

static double pval(const orc_grid *g, const patch *p, const double *Y, int f, int k, int lj, int li) {
    if (p->per) {
        li = wrap(li, p->pw);
        lj = wrap(lj, p->ph);
    }
    (void)g;
    return Y[(((size_t)f * g->nz + k) * p->ph + lj) * p->pw + li];
}

/* phi = (rho phi) / rho; the density field itself has phi = 1 */
static double phi_at(const orc_grid *g, const patch *p, const double *Y, int f, int k, int lj, int li) {
    return pval(g, p, Y, f, k, lj, li) / pval(g, p, Y, 0, k, lj, li);
}

static size_t gidx(const orc_grid *g, int k, int gj, int gi) {
    return ((size_t)k * g->ny + wrap(gj, g->ny)) * g->nx + wrap(gi, g->nx);
}

/* flux through face i+1/2 (dir 0), j+1/2 (dir 1) or k+1/2 (dir 2) of local cell (li, lj, k) */
static double face_flux(const orc_grid *g, const patch *p, const double *Y, int f, int dir,
                        int k, int lj, int li, const double *mu, const double *mv,
                        const double *mw, int *branch) {
    int gi = p->gi0 + li, gj = p->gj0 + lj;
    double m;
    if (branch) *branch = 0;
    if (dir == 0) {
        m = mu[gidx(g, k, gj, gi)];
        if (f == 0) return m;
        return m * orc_face(phi_at(g, p, Y, f, k, lj, li - 1), phi_at(g, p, Y, f, k, lj, li),
                            phi_at(g, p, Y, f, k, lj, li + 1), phi_at(g, p, Y, f, k, lj, li + 2),
                            m, g->lim, branch);
    } else if (dir == 1) {
        m = mv[gidx(g, k, gj, gi)];
        if (f == 0) return m;
        return m * orc_face(phi_at(g, p, Y, f, k, lj - 1, li), phi_at(g, p, Y, f, k, lj, li),
                            phi_at(g, p, Y, f, k, lj + 1, li), phi_at(g, p, Y, f, k, lj + 2, li),
                            m, g->lim, branch);
    } else {
        int nz = g->nz;
        if (k < 0 || k >= nz - 1) return 0.0;    /* rigid lids: no flux */
        m = mw[gidx(g, k + 1, gj, gi)];
        if (f == 0) return m;
        /* ghost levels copy the boundary cell */
        int km1 = k - 1 < 0 ? 0 : k - 1;
        int kp2 = k + 2 > nz - 1 ? nz - 1 : k + 2;
        return m * orc_face(phi_at(g, p, Y, f, km1, lj, li), phi_at(g, p, Y, f, k, lj, li),
                            phi_at(g, p, Y, f, k + 1, lj, li), phi_at(g, p, Y, f, kp2, lj, li),
                            m, g->lim, branch);
    }
}

/* R = -[dX/dx + dY/dy + dZ/dz] + tendency on local cells [li0,li1) x [lj0,lj1) */
static void rhs_patch(const orc_grid *g, const patch *p, const double *Y, const double *mu,
                      const double *mv, const double *mw, const double *tend, int li0,
                      int li1, int lj0, int lj1, double *R, unsigned char *branch) {
    const int F = 2 + g->ntr, nz = g->nz;
    const size_t pc = (size_t)nz * p->ph * p->pw;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int lj = lj0; lj < lj1; lj++) {
        for (int f = 0; f < F; f++) {
            for (int k = 0; k < nz; k++) {
                for (int li = li0; li < li1; li++) {
                    int bx, by, bz;
                    double xp = face_flux(g, p, Y, f, 0, k, lj, li, mu, mv, mw, &bx);
                    double xm = face_flux(g, p, Y, f, 0, k, lj, li - 1, mu, mv, mw, NULL);
                    double yp = face_flux(g, p, Y, f, 1, k, lj, li, mu, mv, mw, &by);
                    double ym = face_flux(g, p, Y, f, 1, k, lj - 1, li, mu, mv, mw, NULL);
                    double zp = face_flux(g, p, Y, f, 2, k, lj, li, mu, mv, mw, &bz);
                    double zm = face_flux(g, p, Y, f, 2, k - 1, lj, li, mu, mv, mw, NULL);
                    double r = -((xp - xm) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k]);
                    if (tend && f > 0) {
                        int gi = p->gi0 + li, gj = p->gj0 + lj;
                        r += tend[(size_t)(f - 1) * nz * g->ny * g->nx + gidx(g, k, gj, gi)];
                    }
                    size_t o = (((size_t)f * nz + k) * p->ph + lj) * p->pw + li;
                    R[o] = r;
                    if (branch) {
                        /* one byte per face: 2 bits per direction (i, j, k) */
                        branch[o] = (unsigned char)(bx | (by << 2) | (bz << 4));
                    }
                }
            }
        }
    }
    (void)pc;
}

void orc_rhs(const orc_grid *g, const double *Y, const double *mu, const double *mv,
             const double *mw, const double *tend, double *R, unsigned char *branch) {
    patch p = {g->nx, g->ny, 0, 0, 1};
    rhs_patch(g, &p, Y, mu, mv, mw, tend, 0, g->nx, 0, g->ny, R, branch);
}

void orc_euler(const orc_grid *g, const double *Y, const double *mu, const double *mv,
               const double *mw, const double *tend, double dt, double *out) {
    size_t n = (size_t)(2 + g->ntr) * g->nz * g->ny * g->nx;
    double *R = (double *)malloc(n * sizeof(double));
    orc_rhs(g, Y, mu, mv, mw, tend, R, NULL);
    for (size_t q = 0; q < n; q++) out[q] = Y[q] + dt * R[q];
    free(R);
}

/* Wicker-Skamarock RK3 on a patch region: Y* = Yn + dt/3 R(Yn),
 * Y** = Yn + dt/2 R(Y*), Yn+1 = Yn + dt R(Y**).  Each stage is evaluated on
 * the region shrunk by `shrink` columns on every side (0 for the periodic
 * domain, 2 per stage for a window patch). */
static void rk3_patch(const orc_grid *g, const patch *p, double *Y, const double *mu,
                      const double *mv, const double *mw, const double *tend, double dt,
                      int margin, int shrink) {
    size_t n = (size_t)(2 + g->ntr) * g->nz * p->ph * p->pw;
    double *Yn = (double *)malloc(n * sizeof(double));
    double *Ys = (double *)malloc(n * sizeof(double));
    double *R = (double *)malloc(n * sizeof(double));
    memcpy(Yn, Y, n * sizeof(double));
    memcpy(Ys, Y, n * sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    const int F = 2 + g->ntr, nz = g->nz;
    for (int s = 0; s < 3; s++) {
        int m = margin + shrink * (s + 1);
        int li0 = m, li1 = p->pw - m, lj0 = m, lj1 = p->ph - m;
        rhs_patch(g, p, Ys, mu, mv, mw, tend, li0, li1, lj0, lj1, R, NULL);
        double *dst = (s == 2) ? Y : Ys;
        for (int f = 0; f < F; f++)
            for (int k = 0; k < nz; k++)
                for (int lj = lj0; lj < lj1; lj++)
                    for (int li = li0; li < li1; li++) {
                        size_t o = (((size_t)f * nz + k) * p->ph + lj) * p->pw + li;
                        dst[o] = Yn[o] + c[s] * R[o];
                    }
    }
    free(Yn);
    free(Ys);
    free(R);
}

void orc_rk3(const orc_grid *g, double *Y, const double *mu, const double *mv,
             const double *mw, const double *tend, double dt) {
    patch p = {g->nx, g->ny, 0, 0, 1};
    rk3_patch(g, &p, Y, mu, mv, mw, tend, dt, 0, 0);
}

/* ------------------------------------------------------------ column physics */

void orc_thomas(int n, const double *a, const double *b, const double *c, const double *d,
                double *x) {
    /* textbook Thomas algorithm: forward elimination upward, back substitution downward */
    double *cp = (double *)malloc((size_t)n * sizeof(double));
    double *dp = (double *)malloc((size_t)n * sizeof(double));
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int k = 1; k < n; k++) {
        double den = b[k] - a[k] * cp[k - 1];
        cp[k] = c[k] / den;
        dp[k] = (d[k] - a[k] * dp[k - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int k = n - 2; k >= 0; k--) x[k] = dp[k] - cp[k] * x[k + 1];
    free(cp);
    free(dp);
}

static void level_heights(const orc_grid *g, double *zf, double *zc) {
    zf[0] = 0.0;
    for (int k = 0; k < g->nz; k++) zf[k + 1] = zf[k] + g->dz[k];
    for (int k = 0; k < g->nz; k++) zc[k] = zf[k] + 0.5 * g->dz[k];
}

/* physics of one column whose values sit at stride `cs` apart in k and
 * `fs` apart between fields; precip receives dt * P_bottom * dx * dy */
static void column_one(const orc_grid *g, double *Y, size_t fs, size_t cs, double dt,
                       const double *zf, const double *zc, double *precip) {
    const int nz = g->nz, F = 2 + g->ntr;
    /* (i) implicit relaxation of theta towards theta_ref(z) */
    if (g->tau > 0.0) {
        double r = dt / g->tau;
        for (int k = 0; k < nz; k++) {
            double rho = Y[k * cs];
            double th = Y[fs + k * cs] / rho;
            th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + r);
            Y[fs + k * cs] = rho * th;
        }
    }
    /* (ii) top-down implicit sedimentation of one tracer:
     * (rho q)_k <- ((rho q)_k dz_k + dt P_{k+1/2}) / (dz_k + dt v), P_{k-1/2} = v (rho q)_k */
    if (g->vsed > 0.0 && g->sed >= 0 && g->sed < g->ntr) {
        double *q = Y + (size_t)(2 + g->sed) * fs;
        double P = 0.0;
        for (int k = nz - 1; k >= 0; k--) {
            double dz = g->dz[k];
            q[k * cs] = (q[k * cs] * dz + dt * P) / (dz + dt * g->vsed);
            P = g->vsed * q[k * cs];
        }
        *precip += dt * P * g->dx * g->dy;
    }
    /* (iii) implicit vertical diffusion of every phi = (rho phi) / rho, phi != rho:
     * a_k = -g_{k-1/2}, c_k = -g_{k+1/2}, b_k = rho_k dz_k + g_{k-1/2} + g_{k+1/2},
     * d_k = dz_k (rho phi)_k, with g_{k+1/2} = dt rho_{k+1/2} K_{k+1/2} / dzc_{k+1/2}
     * and g = 0 at both lids. */
    if (g->k0 > 0.0 && nz >= 2) {
        double *a = (double *)malloc((size_t)nz * sizeof(double));
        double *b = (double *)malloc((size_t)nz * sizeof(double));
        double *c = (double *)malloc((size_t)nz * sizeof(double));
        double *d = (double *)malloc((size_t)nz * sizeof(double));
        double *x = (double *)malloc((size_t)nz * sizeof(double));
        double *gf = (double *)malloc((size_t)(nz + 1) * sizeof(double));
        gf[0] = 0.0;
        gf[nz] = 0.0;
        for (int k = 0; k < nz - 1; k++) {
            double rhof = 0.5 * (Y[k * cs] + Y[(k + 1) * cs]);
            double K = g->k0 * exp(-zf[k + 1] / g->kh);
            double dzc = zc[k + 1] - zc[k];
            gf[k + 1] = dt * rhof * K / dzc;
        }
        for (int k = 0; k < nz; k++) {
            a[k] = -gf[k];
            c[k] = -gf[k + 1];
            b[k] = Y[k * cs] * g->dz[k] + gf[k] + gf[k + 1];
        }
        for (int f = 1; f < F; f++) {
            for (int k = 0; k < nz; k++) d[k] = g->dz[k] * Y[f * fs + k * cs];
            orc_thomas(nz, a, b, c, d, x);
            for (int k = 0; k < nz; k++) Y[f * fs + k * cs] = Y[k * cs] * x[k];
        }
        free(a); free(b); free(c); free(d); free(x); free(gf);
    }
}

static void column_patch(const orc_grid *g, const patch *p, double *Y, double dt, int li0,
                         int li1, int lj0, int lj1, double *precip_col) {
    const int nz = g->nz;
    double *zf = (double *)malloc((size_t)(nz + 1) * sizeof(double));
    double *zc = (double *)malloc((size_t)nz * sizeof(double));
    level_heights(g, zf, zc);
    size_t cs = (size_t)p->ph * p->pw, fs = (size_t)nz * cs;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int lj = lj0; lj < lj1; lj++)
        for (int li = li0; li < li1; li++) {
            double pr = 0.0;
            column_one(g, Y + (size_t)lj * p->pw + li, fs, cs, dt, zf, zc, &pr);
            if (precip_col) precip_col[(size_t)lj * p->pw + li] += pr;
        }
    free(zf);
    free(zc);
}

void orc_column(const orc_grid *g, double *Y, double dt, double *precip_col) {
    patch p = {g->nx, g->ny, 0, 0, 1};
    column_patch(g, &p, Y, dt, 0, g->nx, 0, g->ny, precip_col);
}

/* ------------------------------------------------------------ budgets */

/* Compensated summation (Neumaier, 1974): the running sum s and the rounding
 * errors c of its additions, recovered exactly by Fast2Sum ordered by
 * magnitude.  The result is within about 2 ulp of the exact sum of the terms
 * for any count, where a plain running sum drifts by up to n ulp (a budget
 * sums tens of millions of cells). */
typedef struct { double s, c; } csum;
static void csum_add(csum *a, double x) {
    const double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double csum_value(const csum *a) { return a->s + a->c; }

void orc_budgets(const orc_grid *g, const double *Y, double precip, double *out) {
    const int F = 2 + g->ntr, nz = g->nz;
    const size_t cs = (size_t)g->ny * g->nx, fs = (size_t)nz * cs;
    for (int f = 0; f < F; f++) {
        csum s = {0.0, 0.0};
        /* sum over cells of f dV, dV = dz_k dx dy; fixed order: k innermost, then i, then j */
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                for (int k = 0; k < nz; k++)
                    csum_add(&s, Y[f * fs + k * cs + (size_t)j * g->nx + i] * g->dz[k] * g->dx * g->dy);
        out[f] = csum_value(&s);
    }
    out[F] = precip;
}

/* ------------------------------------------------------------ the step */

void orc_step(const orc_grid *g, double *Y, const double *mu, const double *mv,
              const double *mw, const double *tend, double dt, int nsteps, double *budgets) {
    size_t ncol = (size_t)g->ny * g->nx;
    double *pc = (double *)calloc(ncol, sizeof(double));
    for (int s = 0; s < nsteps; s++) {
        orc_rk3(g, Y, mu, mv, mw, tend, dt);
        orc_column(g, Y, dt, pc);
    }
    if (budgets) {
        csum tot = {0.0, 0.0};
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) csum_add(&tot, pc[(size_t)j * g->nx + i]);
        orc_budgets(g, Y, csum_value(&tot), budgets);
    }
    free(pc);
}

/* nsteps full steps evaluated only on the dependency cone of the window
 * [i0, i0+w) x [j0, j0+h) (periodic global indices).  Each step reaches 6
 * columns out (three stages of a 2-wide stencil), so the working patch is
 * 6*nsteps wider on each side.  out is [F][nz][h][w].  Returns 0 on success. */
int orc_step_window(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                    const double *mw, const double *tend, double dt, int nsteps,
                    int i0, int j0, int w, int h, double *out) {
    if (w <= 0 || h <= 0 || nsteps < 0) return 1;
    const int F = 2 + g->ntr, nz = g->nz, r = 6 * nsteps;
    patch p = {w + 2 * r, h + 2 * r, i0 - r, j0 - r, 0};
    size_t n = (size_t)F * nz * p.ph * p.pw;
    double *P = (double *)malloc(n * sizeof(double));
    if (!P) return 2;
    for (int f = 0; f < F; f++)
        for (int k = 0; k < nz; k++)
            for (int lj = 0; lj < p.ph; lj++)
                for (int li = 0; li < p.pw; li++)
                    P[(((size_t)f * nz + k) * p.ph + lj) * p.pw + li] =
                        Y[(size_t)f * nz * g->ny * g->nx + gidx(g, k, p.gj0 + lj, p.gi0 + li)];
    for (int s = 0; s < nsteps; s++) {
        int margin = 6 * s;
        rk3_patch(g, &p, P, mu, mv, mw, tend, dt, margin, 2);
        int m = margin + 6;
        column_patch(g, &p, P, dt, m, p.pw - m, m, p.ph - m, NULL);
    }
    for (int f = 0; f < F; f++)
        for (int k = 0; k < nz; k++)
            for (int lj = 0; lj < h; lj++)
                for (int li = 0; li < w; li++)
                    out[(((size_t)f * nz + k) * h + lj) * w + li] =
                        P[(((size_t)f * nz + k) * p.ph + lj + r) * p.pw + li + r];
    free(P);
    return 0;
}

/* ====================================================================
 * Tangent-linear and adjoint of the discrete step (FP64, plain).
 *
 * Differentiated map: Y^{n+1} = Col(Y3), Y3 from the three RK stages of
 * Y^n with mass fluxes M = (mu, mv, mw) treated as independent inputs (the
 * vertical flux is not re-derived from continuity); tendencies are constant.
 * Limiter branches are frozen at the values the forward pass takes: with a
 * fixed branch the limiter increment is linear, L = a d0 + b d1 with
 * (a, b) = (0,0) zero, (0,2) "2r", (1/3,2/3) "kappa=1/3", (2,0) "cap 2".
 * ==================================================================== */

static void branch_ab(int br, double *a, double *b) {
    switch (br) {
        case 1: *a = 0.0; *b = 2.0; break;
        case 2: *a = 1.0 / 3.0; *b = 2.0 / 3.0; break;
        case 3: *a = 2.0; *b = 0.0; break;
        default: *a = 0.0; *b = 0.0; break;
    }
}

/* d face / d (pm1, p0, p1, p2) for the branch taken at this face, or for the
 * branch `forced` (0..3) when it is not negative */
static void face_coefs(double pm1, double p0, double p1, double p2, double m, int lim, int forced, double c[4]) {
    int br;
    (void)orc_face(pm1, p0, p1, p2, m, lim, &br);
    if (forced >= 0) br = forced;
    double a, b;
    branch_ab(br, &a, &b);
    if (m >= 0.0) {   /* face = p0 + (a (p0 - pm1) + b (p1 - p0)) / 2 */
        c[0] = -0.5 * a; c[1] = 1.0 + 0.5 * a - 0.5 * b; c[2] = 0.5 * b; c[3] = 0.0;
    } else {          /* face = p1 + (a (p1 - p2) + b (p0 - p1)) / 2 */
        c[0] = 0.0; c[1] = 0.5 * b; c[2] = 1.0 + 0.5 * a - 0.5 * b; c[3] = -0.5 * a;
    }
}

/* cell indices (global, periodic in i/j, clamped in k) of the 4-cell stencil of
 * face "a+1/2" of cell a = (i, j, k) in direction dir */
static void face_stencil(const orc_grid *g, int dir, int k, int j, int i, size_t idx[4], int kk[4]) {
    for (int q = 0; q < 4; q++) {
        int o = q - 1;
        int ii = i, jj = j, kq = k;
        if (dir == 0) ii = i + o;
        else if (dir == 1) jj = j + o;
        else {
            kq = k + o;
            if (kq < 0) kq = 0;
            if (kq > g->nz - 1) kq = g->nz - 1;
        }
        kk[q] = kq;
        idx[q] = gidx(g, kq, jj, ii);
    }
}

static size_t mface_index(const orc_grid *g, int dir, int k, int j, int i) {
    return dir == 2 ? gidx(g, k + 1, j, i) : gidx(g, k, j, i);
}

static const double *mface_array(int dir, const double *mu, const double *mv, const double *mw) {
    return dir == 0 ? mu : (dir == 1 ? mv : mw);
}

static double rdelta(const orc_grid *g, int dir, int k) {
    return dir == 0 ? 1.0 / g->dx : (dir == 1 ? 1.0 / g->dy : 1.0 / g->dz[k]);
}

/* dR = d/dY R(Y; M)[dY] + d/dM R(Y; M)[dM]  (dM may be NULL) */
void orc_rhs_tl_br(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                   const double *mw, const double *dY, const double *dmu, const double *dmv,
                   const double *dmw, const unsigned char *br, double *dR) {
    const int F = 2 + g->ntr, nz = g->nz;
    const size_t C = (size_t)nz * g->ny * g->nx;
    memset(dR, 0, (size_t)F * C * sizeof(double));
    for (int dir = 0; dir < 3; dir++) {
        const double *M = mface_array(dir, mu, mv, mw);
        const double *dM = dmu ? mface_array(dir, dmu, dmv, dmw) : NULL;
        for (int k = 0; k < nz; k++) {
            if (dir == 2 && k >= nz - 1) continue;          /* lids carry no flux */
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    const size_t fm = mface_index(g, dir, k, j, i);
                    const double m = M[fm], dm = dM ? dM[fm] : 0.0;
                    size_t a = gidx(g, k, j, i);
                    size_t b = dir == 0 ? gidx(g, k, j, i + 1) : (dir == 1 ? gidx(g, k, j + 1, i) : gidx(g, k + 1, j, i));
                    const int kb = dir == 2 ? k + 1 : k;
                    size_t st[4];
                    int kk[4];
                    face_stencil(g, dir, k, j, i, st, kk);
                    for (int f = 0; f < F; f++) {
                        double dF;
                        if (f == 0) {
                            dF = dm;
                        } else {
                            double ph[4], dph[4], c[4];
                            for (int q = 0; q < 4; q++) {
                                double rho = Y[st[q]], rp = Y[(size_t)f * C + st[q]];
                                ph[q] = rp / rho;
                                dph[q] = (dY[(size_t)f * C + st[q]] - ph[q] * dY[st[q]]) / rho;
                            }
                            face_coefs(ph[0], ph[1], ph[2], ph[3], m, g->lim,
                                       br ? (br[(size_t)f * C + a] >> (2 * dir)) & 3 : -1, c);
                            double face = orc_face(ph[0], ph[1], ph[2], ph[3], m, g->lim, NULL);
                            double dface = c[0] * dph[0] + c[1] * dph[1] + c[2] * dph[2] + c[3] * dph[3];
                            dF = dm * face + m * dface;
                        }
                        dR[(size_t)f * C + a] -= dF * rdelta(g, dir, k);
                        dR[(size_t)f * C + b] += dF * rdelta(g, dir, kb);
                    }
                }
        }
    }
}

void orc_rhs_tl(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                const double *mw, const double *dY, const double *dmu, const double *dmv,
                const double *dmw, double *dR) {
    orc_rhs_tl_br(g, Y, mu, mv, mw, dY, dmu, dmv, dmw, NULL, dR);
}

/* lamY += (dR/dY)^T mu,  gM += (dR/dM)^T mu   (gM arrays may be NULL); br, when
 * given, holds the branch of every face (the layout orc_rhs writes) */
void orc_rhs_adj_br(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                    const double *mw, const double *lamR, const unsigned char *br, double *lamY,
                    double *gmu, double *gmv, double *gmw) {
    const int F = 2 + g->ntr, nz = g->nz;
    const size_t C = (size_t)nz * g->ny * g->nx;
    for (int dir = 0; dir < 3; dir++) {
        const double *M = mface_array(dir, mu, mv, mw);
        double *gM = gmu ? (dir == 0 ? gmu : (dir == 1 ? gmv : gmw)) : NULL;
        for (int k = 0; k < nz; k++) {
            if (dir == 2 && k >= nz - 1) continue;
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    const size_t fm = mface_index(g, dir, k, j, i);
                    const double m = M[fm];
                    size_t a = gidx(g, k, j, i);
                    size_t b = dir == 0 ? gidx(g, k, j, i + 1) : (dir == 1 ? gidx(g, k, j + 1, i) : gidx(g, k + 1, j, i));
                    const int kb = dir == 2 ? k + 1 : k;
                    size_t st[4];
                    int kk[4];
                    face_stencil(g, dir, k, j, i, st, kk);
                    for (int f = 0; f < F; f++) {
                        /* adjoint of the flux through this face */
                        const double lF = lamR[(size_t)f * C + b] * rdelta(g, dir, kb) -
                                          lamR[(size_t)f * C + a] * rdelta(g, dir, k);
                        if (f == 0) {
                            if (gM) gM[fm] += lF;
                            continue;
                        }
                        double ph[4], c[4];
                        for (int q = 0; q < 4; q++) ph[q] = Y[(size_t)f * C + st[q]] / Y[st[q]];
                        face_coefs(ph[0], ph[1], ph[2], ph[3], m, g->lim,
                                   br ? (br[(size_t)f * C + a] >> (2 * dir)) & 3 : -1, c);
                        double face = orc_face(ph[0], ph[1], ph[2], ph[3], m, g->lim, NULL);
                        if (gM) gM[fm] += lF * face;
                        for (int q = 0; q < 4; q++) {
                            const double lph = lF * m * c[q];         /* adjoint of phi at stencil cell q */
                            const double rho = Y[st[q]];
                            lamY[(size_t)f * C + st[q]] += lph / rho;
                            lamY[st[q]] -= lph * ph[q] / rho;
                        }
                    }
                }
        }
    }
}

void orc_rhs_adj(const orc_grid *g, const double *Y, const double *mu, const double *mv,
                 const double *mw, const double *lamR, double *lamY, double *gmu, double *gmv,
                 double *gmw) {
    orc_rhs_adj_br(g, Y, mu, mv, mw, lamR, NULL, lamY, gmu, gmv, gmw);
}

/* forward column pass of one column, keeping the intermediates the
 * derivatives need: Ya (after relaxation), Yb (after sedimentation),
 * phi[f][k] (diffusion solution, f >= 1) and the face weights gf[k] */
typedef struct {
    double *Ya, *Yb, *phi, *gf, *kcf;
} colwork;

static void col_forward(const orc_grid *g, const double *Y3, double dt, const double *zf,
                        const double *zc, colwork *w) {
    const int nz = g->nz, F = 2 + g->ntr;
    /* Y3, Ya, Yb are [F][nz] for one column */
    memcpy(w->Ya, Y3, (size_t)F * nz * sizeof(double));
    if (g->tau > 0.0) {
        double r = dt / g->tau;
        for (int k = 0; k < nz; k++) {
            double rho = w->Ya[k];
            double th = w->Ya[nz + k] / rho;
            th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + r);
            w->Ya[nz + k] = rho * th;
        }
    }
    memcpy(w->Yb, w->Ya, (size_t)F * nz * sizeof(double));
    if (g->vsed > 0.0 && g->sed >= 0 && g->sed < g->ntr) {
        double *q = w->Yb + (size_t)(2 + g->sed) * nz;
        double P = 0.0;
        for (int k = nz - 1; k >= 0; k--) {
            q[k] = (q[k] * g->dz[k] + dt * P) / (g->dz[k] + dt * g->vsed);
            P = g->vsed * q[k];
        }
    }
    for (int k = 0; k <= nz; k++) { w->gf[k] = 0.0; w->kcf[k] = 0.0; }
    if (g->k0 > 0.0 && nz >= 2) {
        for (int k = 0; k < nz - 1; k++) {
            double K = g->k0 * exp(-zf[k + 1] / g->kh);
            w->kcf[k + 1] = 0.5 * dt * K / (zc[k + 1] - zc[k]);    /* d g_{k+1/2} / d rho_k */
            w->gf[k + 1] = dt * 0.5 * (w->Yb[k] + w->Yb[k + 1]) * K / (zc[k + 1] - zc[k]);
        }
        double *a = (double *)malloc((size_t)nz * sizeof(double));
        double *b = (double *)malloc((size_t)nz * sizeof(double));
        double *c = (double *)malloc((size_t)nz * sizeof(double));
        double *d = (double *)malloc((size_t)nz * sizeof(double));
        for (int k = 0; k < nz; k++) {
            a[k] = -w->gf[k];
            c[k] = -w->gf[k + 1];
            b[k] = w->Yb[k] * g->dz[k] + w->gf[k] + w->gf[k + 1];
        }
        for (int f = 1; f < F; f++) {
            for (int k = 0; k < nz; k++) d[k] = g->dz[k] * w->Yb[(size_t)f * nz + k];
            orc_thomas(nz, a, b, c, d, w->phi + (size_t)f * nz);
        }
        free(a); free(b); free(c); free(d);
    }
}

static void col_matrix(const orc_grid *g, const colwork *w, double *a, double *b, double *c) {
    for (int k = 0; k < g->nz; k++) {
        a[k] = -w->gf[k];
        c[k] = -w->gf[k + 1];
        b[k] = w->Yb[k] * g->dz[k] + w->gf[k] + w->gf[k + 1];
    }
}

/* tangent of the column pass of one column: dY3 -> dOut ([F][nz]) */
static void col_tl(const orc_grid *g, const double *Y3, const double *dY3, double dt,
                   const double *zf, const double *zc, colwork *w, double *dOut) {
    const int nz = g->nz, F = 2 + g->ntr;
    col_forward(g, Y3, dt, zf, zc, w);
    double *dA = (double *)malloc((size_t)F * nz * sizeof(double));
    memcpy(dA, dY3, (size_t)F * nz * sizeof(double));
    if (g->tau > 0.0) {   /* rho theta_a = (rho theta + r rho theta_ref) / (1 + r) */
        double r = dt / g->tau;
        for (int k = 0; k < nz; k++)
            dA[nz + k] = (dY3[nz + k] + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k]) * dY3[k]) / (1.0 + r);
    }
    if (g->vsed > 0.0 && g->sed >= 0 && g->sed < g->ntr) {
        double *dq = dA + (size_t)(2 + g->sed) * nz;
        double dP = 0.0;
        for (int k = nz - 1; k >= 0; k--) {
            dq[k] = (dq[k] * g->dz[k] + dt * dP) / (g->dz[k] + dt * g->vsed);
            dP = g->vsed * dq[k];
        }
    }
    memcpy(dOut, dA, (size_t)F * nz * sizeof(double));
    if (g->k0 > 0.0 && nz >= 2) {
        /* u = rho phi, A(rho) phi = dz x  =>  A dphi = dz dx - dA phi,  du = drho phi + rho dphi */
        double *a = (double *)malloc((size_t)nz * sizeof(double));
        double *b = (double *)malloc((size_t)nz * sizeof(double));
        double *c = (double *)malloc((size_t)nz * sizeof(double));
        double *d = (double *)malloc((size_t)nz * sizeof(double));
        double *x = (double *)malloc((size_t)nz * sizeof(double));
        col_matrix(g, w, a, b, c);
        const double *drho = dA;
        for (int f = 1; f < F; f++) {
            const double *ph = w->phi + (size_t)f * nz;
            for (int k = 0; k < nz; k++) {
                /* (dA phi)_k = drho_k dz_k phi_k + sum over faces of dg (phi_k - phi_other) */
                double dAp = drho[k] * g->dz[k] * ph[k];
                if (k > 0) dAp += w->kcf[k] * (drho[k - 1] + drho[k]) * (ph[k] - ph[k - 1]);
                if (k < nz - 1) dAp += w->kcf[k + 1] * (drho[k] + drho[k + 1]) * (ph[k] - ph[k + 1]);
                d[k] = g->dz[k] * dA[(size_t)f * nz + k] - dAp;
            }
            orc_thomas(nz, a, b, c, d, x);
            for (int k = 0; k < nz; k++) dOut[(size_t)f * nz + k] = drho[k] * ph[k] + w->Yb[k] * x[k];
        }
        free(a); free(b); free(c); free(d); free(x);
    }
    free(dA);
}

/* adjoint of the column pass of one column: lam ([F][nz]) in: adjoint of
 * the output; out: adjoint of Y3 */
static void col_adj(const orc_grid *g, const double *Y3, double *lam, double dt, const double *zf,
                    const double *zc, colwork *w) {
    const int nz = g->nz, F = 2 + g->ntr;
    col_forward(g, Y3, dt, zf, zc, w);
    if (g->k0 > 0.0 && nz >= 2) {
        double *a = (double *)malloc((size_t)nz * sizeof(double));
        double *b = (double *)malloc((size_t)nz * sizeof(double));
        double *c = (double *)malloc((size_t)nz * sizeof(double));
        double *d = (double *)malloc((size_t)nz * sizeof(double));
        double *psi = (double *)malloc((size_t)nz * sizeof(double));
        col_matrix(g, w, a, b, c);   /* A is symmetric: A^T = A */
        for (int f = 1; f < F; f++) {
            const double *ph = w->phi + (size_t)f * nz;
            double *lu = lam + (size_t)f * nz;
            for (int k = 0; k < nz; k++) d[k] = w->Yb[k] * lu[k];
            orc_thomas(nz, a, b, c, d, psi);
            for (int k = 0; k < nz; k++) {
                double lr = lu[k] * ph[k] - g->dz[k] * psi[k] * ph[k];
                if (k > 0) lr -= w->kcf[k] * (psi[k] - psi[k - 1]) * (ph[k] - ph[k - 1]);
                if (k < nz - 1) lr -= w->kcf[k + 1] * (psi[k] - psi[k + 1]) * (ph[k] - ph[k + 1]);
                lam[k] += lr;
            }
            for (int k = 0; k < nz; k++) lu[k] = g->dz[k] * psi[k];
        }
        free(a); free(b); free(c); free(d); free(psi);
    }
    if (g->vsed > 0.0 && g->sed >= 0 && g->sed < g->ntr) {
        /* q'_k = (q_k dz_k + dt v q'_{k+1}) w_k, w_k = 1/(dz_k + dt v): the adjoint runs bottom-up */
        double *lq = lam + (size_t)(2 + g->sed) * nz;
        double nu_prev = 0.0;
        for (int k = 0; k < nz; k++) {
            double nu = lq[k];
            if (k > 0) nu += dt * g->vsed / (g->dz[k - 1] + dt * g->vsed) * nu_prev;
            nu_prev = nu;
            lq[k] = nu * g->dz[k] / (g->dz[k] + dt * g->vsed);
        }
    }
    if (g->tau > 0.0) {
        double r = dt / g->tau;
        for (int k = 0; k < nz; k++) {
            double lt = lam[nz + k];
            lam[k] += lt * r * (THETA_REF0 + THETA_REF_LAPSE * zc[k]) / (1.0 + r);
            lam[nz + k] = lt / (1.0 + r);
        }
    }
}

static void col_alloc(const orc_grid *g, colwork *w) {
    size_t n = (size_t)(2 + g->ntr) * g->nz;
    w->Ya = (double *)calloc(n, sizeof(double));
    w->Yb = (double *)calloc(n, sizeof(double));
    w->phi = (double *)calloc(n, sizeof(double));
    w->gf = (double *)calloc((size_t)g->nz + 1, sizeof(double));
    w->kcf = (double *)calloc((size_t)g->nz + 1, sizeof(double));
}

static void col_free(colwork *w) {
    free(w->Ya); free(w->Yb); free(w->phi); free(w->gf); free(w->kcf);
}

static void gather_col(const orc_grid *g, const double *Y, int j, int i, double *out) {
    const size_t C = (size_t)g->nz * g->ny * g->nx;
    for (int f = 0; f < 2 + g->ntr; f++)
        for (int k = 0; k < g->nz; k++) out[(size_t)f * g->nz + k] = Y[(size_t)f * C + gidx(g, k, j, i)];
}

static void scatter_col(const orc_grid *g, double *Y, int j, int i, const double *in) {
    const size_t C = (size_t)g->nz * g->ny * g->nx;
    for (int f = 0; f < 2 + g->ntr; f++)
        for (int k = 0; k < g->nz; k++) Y[(size_t)f * C + gidx(g, k, j, i)] = in[(size_t)f * g->nz + k];
}

void orc_column_tl(const orc_grid *g, const double *Y3, const double *dY3, double dt, double *dOut) {
    const int nz = g->nz, F = 2 + g->ntr;
    double *zf = (double *)malloc((size_t)(nz + 1) * sizeof(double));
    double *zc = (double *)malloc((size_t)nz * sizeof(double));
    level_heights(g, zf, zc);
    colwork w;
    col_alloc(g, &w);
    double *y = (double *)malloc((size_t)F * nz * sizeof(double));
    double *dy = (double *)malloc((size_t)F * nz * sizeof(double));
    double *o = (double *)malloc((size_t)F * nz * sizeof(double));
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            gather_col(g, Y3, j, i, y);
            gather_col(g, dY3, j, i, dy);
            col_tl(g, y, dy, dt, zf, zc, &w, o);
            scatter_col(g, dOut, j, i, o);
        }
    free(y); free(dy); free(o); col_free(&w); free(zf); free(zc);
}

void orc_column_adj(const orc_grid *g, const double *Y3, double *lam, double dt) {
    const int nz = g->nz, F = 2 + g->ntr;
    double *zf = (double *)malloc((size_t)(nz + 1) * sizeof(double));
    double *zc = (double *)malloc((size_t)nz * sizeof(double));
    level_heights(g, zf, zc);
    colwork w;
    col_alloc(g, &w);
    double *y = (double *)malloc((size_t)F * nz * sizeof(double));
    double *l = (double *)malloc((size_t)F * nz * sizeof(double));
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            gather_col(g, Y3, j, i, y);
            gather_col(g, lam, j, i, l);
            col_adj(g, y, l, dt, zf, zc, &w);
            scatter_col(g, lam, j, i, l);
        }
    free(y); free(l); col_free(&w); free(zf); free(zc);
}

/* states of one forward step: Yn (input), Y1, Y2 (stage states), Y3 (before the column pass) */
static void step_states(const orc_grid *g, const double *Yn, const double *mu, const double *mv,
                        const double *mw, const double *tend, double dt, double *Y1, double *Y2,
                        double *Y3, double *Ynext) {
    const size_t n = (size_t)(2 + g->ntr) * g->nz * g->ny * g->nx;
    double *R = (double *)malloc(n * sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    double *outs[3] = {Y1, Y2, Y3};
    const double *in = Yn;
    for (int s = 0; s < 3; s++) {
        orc_rhs(g, in, mu, mv, mw, tend, R, NULL);
        for (size_t q = 0; q < n; q++) outs[s][q] = Yn[q] + c[s] * R[q];
        in = outs[s];
    }
    memcpy(Ynext, Y3, n * sizeof(double));
    orc_column(g, Ynext, dt, NULL);
    free(R);
}

/* tangent of nsteps steps: (dY0, dM) -> dYn; traj_br, when given, fixes the
 * branch of every face of every stage ([nsteps][3][F][nz][ny][nx] bytes) */
void orc_step_tl_br(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                    const double *mw, const double *tend, double dt, int nsteps, const double *dY0,
                    const double *dmu, const double *dmv, const double *dmw,
                    const unsigned char *traj_br, double *dYn) {
    const size_t n = (size_t)(2 + g->ntr) * g->nz * g->ny * g->nx;
    double *Y = (double *)malloc(n * sizeof(double));
    double *Y1 = (double *)malloc(n * sizeof(double));
    double *Y2 = (double *)malloc(n * sizeof(double));
    double *Y3 = (double *)malloc(n * sizeof(double));
    double *Yx = (double *)malloc(n * sizeof(double));
    double *dY = (double *)malloc(n * sizeof(double));
    double *dS = (double *)malloc(n * sizeof(double));
    double *dR = (double *)malloc(n * sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    memcpy(Y, Y0, n * sizeof(double));
    memcpy(dY, dY0, n * sizeof(double));
    for (int s = 0; s < nsteps; s++) {
        step_states(g, Y, mu, mv, mw, tend, dt, Y1, Y2, Y3, Yx);
        const double *st[3] = {Y, Y1, Y2};
        memcpy(dS, dY, n * sizeof(double));              /* tangent of the stage input */
        for (int q = 0; q < 3; q++) {
            orc_rhs_tl_br(g, st[q], mu, mv, mw, dS, dmu, dmv, dmw,
                          traj_br ? traj_br + ((size_t)s * 3 + q) * n : NULL, dR);
            for (size_t e = 0; e < n; e++) dS[e] = dY[e] + c[q] * dR[e];
        }
        orc_column_tl(g, Y3, dS, dt, dY);
        memcpy(Y, Yx, n * sizeof(double));
    }
    memcpy(dYn, dY, n * sizeof(double));
    free(Y); free(Y1); free(Y2); free(Y3); free(Yx); free(dY); free(dS); free(dR);
}

void orc_step_tl(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                 const double *mw, const double *tend, double dt, int nsteps, const double *dY0,
                 const double *dmu, const double *dmv, const double *dmw, double *dYn) {
    orc_step_tl_br(g, Y0, mu, mv, mw, tend, dt, nsteps, dY0, dmu, dmv, dmw, NULL, dYn);
}

/* adjoint of nsteps steps: lam_final -> lam0 (adjoint of Y0), g_mu/g_mv/g_mw
 * (adjoint of the mass fluxes; overwritten).  The whole trajectory is kept.
 * traj_br as for orc_step_tl_br. */
void orc_step_adj_br(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                     const double *mw, const double *tend, double dt, int nsteps,
                     const double *lam_final, const unsigned char *traj_br, double *lam0,
                     double *gmu, double *gmv, double *gmw) {
    const size_t C = (size_t)g->nz * g->ny * g->nx;
    const size_t n = (size_t)(2 + g->ntr) * C;
    const size_t nw = (size_t)(g->nz + 1) * g->ny * g->nx;
    double *traj = (double *)malloc((size_t)(nsteps + 1) * 3 * n * sizeof(double) + 1);
    /* per step s: [Y^s, Y1, Y2] at traj + 3 n s, Y3 kept at the next slot's ... */
    double *Y3s = (double *)malloc((size_t)(nsteps > 0 ? nsteps : 1) * n * sizeof(double));
    memcpy(traj, Y0, n * sizeof(double));
    for (int s = 0; s < nsteps; s++) {
        double *Ys = traj + (size_t)3 * n * s;
        step_states(g, Ys, mu, mv, mw, tend, dt, Ys + n, Ys + 2 * n, Y3s + (size_t)s * n,
                    traj + (size_t)3 * n * (s + 1));
    }
    memset(gmu, 0, C * sizeof(double));
    memset(gmv, 0, C * sizeof(double));
    memset(gmw, 0, nw * sizeof(double));
    double *lam = (double *)malloc(n * sizeof(double));
    double *l2 = (double *)malloc(n * sizeof(double));
    double *l1 = (double *)malloc(n * sizeof(double));
    double *mu_r = (double *)malloc(n * sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    memcpy(lam, lam_final, n * sizeof(double));
    for (int s = nsteps - 1; s >= 0; s--) {
        const double *Ys = traj + (size_t)3 * n * s;
        orc_column_adj(g, Y3s + (size_t)s * n, lam, dt);          /* lam: adjoint of Y3 */
        /* Y3 = Yn + c3 R(Y2) */
        for (size_t e = 0; e < n; e++) { mu_r[e] = c[2] * lam[e]; l2[e] = 0.0; }
        const unsigned char *b3 = traj_br ? traj_br + ((size_t)s * 3 + 2) * n : NULL;
        const unsigned char *b2 = traj_br ? traj_br + ((size_t)s * 3 + 1) * n : NULL;
        const unsigned char *b1 = traj_br ? traj_br + ((size_t)s * 3 + 0) * n : NULL;
        orc_rhs_adj_br(g, Ys + 2 * n, mu, mv, mw, mu_r, b3, l2, gmu, gmv, gmw);
        /* Y2 = Yn + c2 R(Y1) */
        for (size_t e = 0; e < n; e++) { mu_r[e] = c[1] * l2[e]; l1[e] = 0.0; }
        orc_rhs_adj_br(g, Ys + n, mu, mv, mw, mu_r, b2, l1, gmu, gmv, gmw);
        /* Y1 = Yn + c1 R(Yn) */
        for (size_t e = 0; e < n; e++) { lam[e] += l2[e] + l1[e]; mu_r[e] = c[0] * l1[e]; }
        orc_rhs_adj_br(g, Ys, mu, mv, mw, mu_r, b1, lam, gmu, gmv, gmw);
    }
    memcpy(lam0, lam, n * sizeof(double));
    free(traj); free(Y3s); free(lam); free(l2); free(l1); free(mu_r);
}

void orc_step_adj(const orc_grid *g, const double *Y0, const double *mu, const double *mv,
                  const double *mw, const double *tend, double dt, int nsteps,
                  const double *lam_final, double *lam0, double *gmu, double *gmv, double *gmw) {
    orc_step_adj_br(g, Y0, mu, mv, mw, tend, dt, nsteps, lam_final, NULL, lam0, gmu, gmv, gmw);
}

/* limiter branches of every face of every stage of nsteps steps:
 * out[(step * 3 + stage) * F * C + f * C + cell] (2 bits per direction) */
void orc_trajectory_branches(const orc_grid *g, const double *Y0, const double *mu,
                             const double *mv, const double *mw, const double *tend, double dt,
                             int nsteps, unsigned char *out) {
    const size_t n = (size_t)(2 + g->ntr) * g->nz * g->ny * g->nx;
    double *Y = (double *)malloc(n * sizeof(double));
    double *S = (double *)malloc(n * sizeof(double));
    double *R = (double *)malloc(n * sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    memcpy(Y, Y0, n * sizeof(double));
    for (int s = 0; s < nsteps; s++) {
        const double *in = Y;
        for (int q = 0; q < 3; q++) {
            orc_rhs(g, in, mu, mv, mw, tend, R, out + ((size_t)s * 3 + q) * n);
            for (size_t e = 0; e < n; e++) S[e] = Y[e] + c[q] * R[e];
            if (q < 2) {
                double *t = (double *)malloc(n * sizeof(double));
                memcpy(t, S, n * sizeof(double));
                if (in != Y) free((void *)in);
                in = t;
            }
        }
        if (in != Y) free((void *)in);
        orc_column(g, S, dt, NULL);
        memcpy(Y, S, n * sizeof(double));
    }
    free(Y); free(S); free(R);
}

/* ---- open (non-periodic) lateral boundaries -------------------------------
 * A domain whose edge cells have no periodic neighbours: a limited-area
 * domain fed by boundary data (the boundary datasets of the damping kernel,
 * Sec. 2.1), or one block of a horizontally decomposed domain (Sec. 1.1:
 * horizontal blocks exchanging halos).  The lateral neighbours outside the
 * domain are two ghost columns (rows) per side whose phi values, for fields
 * 1 .. F-1, are given in the halo layout: four strips one after another,
 *   W: phi at i = c - 2,   E: phi at i = nx + c   (c = 0, 1; every j)
 *   S: phi at j = c - 2,   N: phi at j = ny + c   (c = 0, 1; every i)
 * each [F-1][nz][2][len], len = ny for W and E, nx for S and N.  The
 * density needs no ghost: its flux is M itself.  Every face of the domain,
 * the outer ones included, has its own mass flux:
 *   mu_x[k][j][i], i = 0 .. nx: face i - 1/2 of cell i  ([nz][ny][nx+1]);
 *   mv_x[k][j][i], j = 0 .. ny: face j - 1/2 of cell j  ([nz][ny+1][nx]);
 *   mw as in the periodic domain.
 * The faces are the periodic domain's Koren reconstruction, reading a ghost
 * wherever the four-cell stencil leaves the domain; the ghosts are held for
 * the whole call.  Vertical faces are unchanged. */

static size_t halo_index(const orc_grid *g, int strip, int f1, int k, int c, int pos) {
    const size_t T = (size_t)(1 + g->ntr), nz = (size_t)g->nz;
    const size_t sw = T * nz * 2 * (size_t)g->ny, ss = T * nz * 2 * (size_t)g->nx;
    const size_t base = strip == 0 ? 0 : (strip == 1 ? sw : (strip == 2 ? 2 * sw : 2 * sw + ss));
    const size_t len = strip < 2 ? (size_t)g->ny : (size_t)g->nx;
    return base + (((size_t)f1 * nz + k) * 2 + c) * len + pos;
}

/* phi of field f >= 1 at (k, j, i), i in [-2, nx+1] or j in [-2, ny+1] (not both outside) */
static double phi_open(const orc_grid *g, const double *Y, const double *ghost, int f, int k, int j, int i) {
    if (i < 0) return ghost[halo_index(g, 0, f - 1, k, i + 2, j)];
    if (i >= g->nx) return ghost[halo_index(g, 1, f - 1, k, i - g->nx, j)];
    if (j < 0) return ghost[halo_index(g, 2, f - 1, k, j + 2, i)];
    if (j >= g->ny) return ghost[halo_index(g, 3, f - 1, k, j - g->ny, i)];
    const size_t C = (size_t)g->nz * g->ny * g->nx, o = ((size_t)k * g->ny + j) * g->nx + i;
    return Y[(size_t)f * C + o] / Y[o];
}

/* flux through face i+1/2 (dir 0, i = -1 .. nx-1), j+1/2 (dir 1, j = -1 .. ny-1)
 * or k+1/2 (dir 2) of cell (i, j, k) */
static double flux_open(const orc_grid *g, const double *Y, const double *ghost, const double *mu_x,
                        const double *mv_x, const double *mw, int f, int dir, int k, int j, int i) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    double m;
    if (dir == 0) {
        m = mu_x[((size_t)k * ny + j) * (nx + 1) + (i + 1)];
        if (f == 0) return m;
        return m * orc_face(phi_open(g, Y, ghost, f, k, j, i - 1), phi_open(g, Y, ghost, f, k, j, i),
                            phi_open(g, Y, ghost, f, k, j, i + 1), phi_open(g, Y, ghost, f, k, j, i + 2),
                            m, g->lim, NULL);
    } else if (dir == 1) {
        m = mv_x[((size_t)k * (ny + 1) + (j + 1)) * nx + i];
        if (f == 0) return m;
        return m * orc_face(phi_open(g, Y, ghost, f, k, j - 1, i), phi_open(g, Y, ghost, f, k, j, i),
                            phi_open(g, Y, ghost, f, k, j + 1, i), phi_open(g, Y, ghost, f, k, j + 2, i),
                            m, g->lim, NULL);
    }
    if (k < 0 || k >= nz - 1) return 0.0;    /* rigid lids: no flux */
    m = mw[((size_t)(k + 1) * ny + j) * nx + i];
    if (f == 0) return m;
    const int km1 = k - 1 < 0 ? 0 : k - 1, kp2 = k + 2 > nz - 1 ? nz - 1 : k + 2;
    return m * orc_face(phi_open(g, Y, ghost, f, km1, j, i), phi_open(g, Y, ghost, f, k, j, i),
                        phi_open(g, Y, ghost, f, k + 1, j, i), phi_open(g, Y, ghost, f, kp2, j, i),
                        m, g->lim, NULL);
}

void orc_rhs_open(const orc_grid *g, const double *Y, const double *mu_x, const double *mv_x,
                  const double *mw, const double *tend, const double *ghost, double *R) {
    const int F = 2 + g->ntr, nz = g->nz, ny = g->ny, nx = g->nx;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < ny; j++)
        for (int f = 0; f < F; f++)
            for (int k = 0; k < nz; k++)
                for (int i = 0; i < nx; i++) {
                    double xp = flux_open(g, Y, ghost, mu_x, mv_x, mw, f, 0, k, j, i);
                    double xm = flux_open(g, Y, ghost, mu_x, mv_x, mw, f, 0, k, j, i - 1);
                    double yp = flux_open(g, Y, ghost, mu_x, mv_x, mw, f, 1, k, j, i);
                    double ym = flux_open(g, Y, ghost, mu_x, mv_x, mw, f, 1, k, j - 1, i);
                    double zp = flux_open(g, Y, ghost, mu_x, mv_x, mw, f, 2, k, j, i);
                    double zm = flux_open(g, Y, ghost, mu_x, mv_x, mw, f, 2, k - 1, j, i);
                    double r = -((xp - xm) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k]);
                    const size_t o = (((size_t)f * nz + k) * ny + j) * nx + i;
                    if (tend && f > 0) r += tend[o - (size_t)nz * ny * nx];
                    R[o] = r;
                }
}

/* nsteps steps of the open domain: the three RK stages with the ghosts held,
 * then the column pass and, if budgets is set, the budgets as orc_step
 * (the mass budget then changes by the mass that crossed the outer faces). */
void orc_step_open(const orc_grid *g, double *Y, const double *mu_x, const double *mv_x, const double *mw,
                   const double *tend, const double *ghost, double dt, int nsteps, double *budgets) {
    const size_t n = (size_t)(2 + g->ntr) * g->nz * g->ny * g->nx;
    double *Yn = (double *)malloc(n * sizeof(double));
    double *Ys = (double *)malloc(n * sizeof(double));
    double *R = (double *)malloc(n * sizeof(double));
    double *pc = (double *)calloc((size_t)g->ny * g->nx, sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    for (int s = 0; s < nsteps; s++) {
        memcpy(Yn, Y, n * sizeof(double));
        const double *in = Yn;
        for (int q = 0; q < 3; q++) {
            orc_rhs_open(g, in, mu_x, mv_x, mw, tend, ghost, R);
            double *dst = q == 2 ? Y : Ys;
            for (size_t e = 0; e < n; e++) dst[e] = Yn[e] + c[q] * R[e];
            in = Ys;
        }
        orc_column(g, Y, dt, pc);
    }
    if (budgets) {
        csum tot = {0.0, 0.0};
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) csum_add(&tot, pc[(size_t)j * g->nx + i]);
        orc_budgets(g, Y, csum_value(&tot), budgets);
    }
    free(Yn);
    free(Ys);
    free(R);
    free(pc);
}

/* ---- 7-point diffusion stencil (Sec. 4, reduced weather application) ---------
 * The paper names the kernel but prints no formula; the reading is the
 * textbook explicit diffusion step with one diffusion number c for all three
 * directions: out = in + c (in(i-1) + in(i+1) + in(j-1) + in(j+1) + in(k-1)
 * + in(k+1) - 6 in), periodic in i and j, and zero flux through the lids
 * (the ghost level copies the boundary cell, so its difference vanishes). */
void orc_stencil7(int nx, int ny, int nz, double c, const double *in, double *out) {
    const long long plane = (long long)nx * ny;
#ifdef _OPENMP
#pragma omp parallel for
#endif
    for (int k = 0; k < nz; k++) {
        const int kd = k > 0 ? k - 1 : 0, ku = k < nz - 1 ? k + 1 : nz - 1;
        for (int j = 0; j < ny; j++) {
            const int jd = wrap(j - 1, ny), ju = wrap(j + 1, ny);
            for (int i = 0; i < nx; i++) {
                const int id = wrap(i - 1, nx), iu = wrap(i + 1, nx);
                const double v = in[k * plane + (long long)j * nx + i];
                const double sum = in[k * plane + (long long)j * nx + id] + in[k * plane + (long long)j * nx + iu] +
                                   in[k * plane + (long long)jd * nx + i] + in[k * plane + (long long)ju * nx + i] +
                                   in[kd * plane + (long long)j * nx + i] + in[ku * plane + (long long)j * nx + i];
                out[k * plane + (long long)j * nx + i] = v + c * (sum - 6.0 * v);
            }
        }
    }
}

/* ---- lateral and upper damping (Sec. 2.1, the damping kernel) --------------
 * The paper's kernel forms the damping target: the reference state plus the
 * boundary perturbation, weighted between two boundary datasets by mtratio
 * and tratio.  It prints no damping operator; the reading is an implicit
 * (backward Euler) Rayleigh relaxation toward that target,
 * dy/dt = -nu (y - target), with a rate that grows quadratically toward the
 * lateral edges over `width` cells and toward the model top over ntop levels,
 * the larger of the two where the zones overlap. */
static double damping_rate(int nx, int ny, int nz, int width, int ntop, double nu_lat, double nu_top, int i, int j,
                           int k) {
    int d = i;
    if (nx - 1 - i < d) d = nx - 1 - i;
    if (j < d) d = j;
    if (ny - 1 - j < d) d = ny - 1 - j;
    double lat = 0.0, top = 0.0;
    if (d < width) {
        const double x = (double)(width - d) / width;
        lat = nu_lat * (x * x);
    }
    if (ntop > 0 && k >= nz - ntop) {
        const double x = (double)(k - (nz - ntop) + 1) / ntop;
        top = nu_top * (x * x);
    }
    return lat > top ? lat : top;
}

void orc_damping(int nx, int ny, int nz, int F, int width, int ntop, double nu_lat, double nu_top,
                 double mtratio, double tratio, double dt, long long ncell, const int *ijk, double *y,
                 const double *ref, const double *b0, const double *b1) {
    const long long n = ijk ? ncell : (long long)nx * ny * nz;
#ifdef _OPENMP
#pragma omp parallel for
#endif
    for (long long c = 0; c < n; c++) {
        int i, j, k;
        if (ijk) {
            i = ijk[3 * c];
            j = ijk[3 * c + 1];
            k = ijk[3 * c + 2];
        } else {
            i = (int)(c % nx);
            j = (int)((c / nx) % ny);
            k = (int)(c / ((long long)nx * ny));
        }
        const double a = dt * damping_rate(nx, ny, nz, width, ntop, nu_lat, nu_top, i, j, k);
        for (int f = 0; f < F; f++) {
            const long long q = (long long)f * n + c;
            const double ptb = mtratio * (ref[q] + b0[q]) + tratio * (ref[q] + b1[q]) - ref[q];
            const double target = ref[q] + ptb;
            y[q] = (y[q] + a * target) / (1.0 + a);
        }
    }
}

/* ---- HEVI acoustic short steps (Sec. 1.1: sound and gravity waves in a
 * second-order Runge-Kutta scheme, horizontally explicit, vertically implicit)
 * The paper names the scheme only.  The reading: the linear acoustic-gravity
 * system about a resting, horizontally uniform base state rho0(z), written
 * for the momenta U, V (faces i+1/2, j+1/2), W (faces k-1/2, rigid lids) and
 * s = rho'/rho0 at the centres,
 *   dU/dt = -c^2 rho0_k (s_{i+1} - s_i) / dx,   dV/dt likewise in j,
 *   dW_f/dt = -c^2 rho0f_f (s_f - s_{f-1}) / dzc_f,   dzc_f = (dz_{f-1} + dz_f) / 2,
 *   rho0_k ds/dt = -[(U_{i+1/2} - U_{i-1/2})/dx + (V_{j+1/2} - V_{j-1/2})/dy + (W_{k+1} - W_k)/dz_k],
 * (for rho0 = rho_s exp(-g z / c^2) the W equation is dW/dt = -dp'/dz - g rho').
 * A short step of length h is two stages from the same start (U, V, W, s):
 *   stage 1 (tau = h/2): U* = U - tau G_x(s); (W*, s*) implicit with Dh(U*, V*);
 *   stage 2 (tau = h):   U+ = U - tau G_x(s*); (W+, s+) implicit with Dh(U*, V*);
 * the implicit part weights the new and old vertical terms by beta, 1 - beta:
 *   W'_f = W_f - tau c^2 rho0f_f [beta (s'_f - s'_{f-1}) + (1-beta)(s_f - s_{f-1})] / dzc_f
 *   rho0_k s'_k = rho0_k s_k - tau [Dh_k + (beta (W'_{k+1} - W'_k) + (1-beta)(W_{k+1} - W_k)) / dz_k]
 * Here the two implicit equations are solved together as written: with the
 * unknowns interleaved (s'_0, W'_1, s'_1, ..., W'_{nz-1}, s'_{nz-1}) the
 * system is tridiagonal, solved by plain Gaussian elimination. */
static void acoustic_column(int nz, const double *dz, const double *rho0c, const double *rho0f, double cs2,
                            double beta, double tau, const double *Dh, const double *W, const double *s,
                            double *Wn, double *sn, double *lo, double *di, double *up, double *rhs) {
    /* row 2k: the s'_k equation, row 2f-1: the W'_f equation */
    const int n = 2 * nz - 1;
    for (int k = 0; k < nz; k++) {
        const int r = 2 * k;
        const double Wk = k > 0 ? W[k] : 0.0, Wk1 = k < nz - 1 ? W[k + 1] : 0.0;
        /* rho0 s' + tau beta (W'_{k+1} - W'_k)/dz = rho0 s - tau Dh - tau (1-beta)(W_{k+1} - W_k)/dz */
        di[r] = rho0c[k];
        lo[r] = k > 0 ? -tau * beta / dz[k] : 0.0;
        up[r] = k < nz - 1 ? tau * beta / dz[k] : 0.0;
        rhs[r] = rho0c[k] * s[k] - tau * Dh[k] - tau * (1.0 - beta) * (Wk1 - Wk) / dz[k];
    }
    for (int f = 1; f < nz; f++) {
        const int r = 2 * f - 1;
        const double dzc = 0.5 * (dz[f - 1] + dz[f]);
        const double g = tau * cs2 * rho0f[f] / dzc;
        /* W'_f + g beta (s'_f - s'_{f-1}) = W_f - g (1-beta)(s_f - s_{f-1}) */
        di[r] = 1.0;
        lo[r] = -g * beta;
        up[r] = g * beta;
        rhs[r] = W[f] - g * (1.0 - beta) * (s[f] - s[f - 1]);
    }
    /* forward elimination, no pivoting, then back substitution */
    for (int r = 1; r < n; r++) {
        const double m = lo[r] / di[r - 1];
        di[r] -= m * up[r - 1];
        rhs[r] -= m * rhs[r - 1];
    }
    double x = rhs[n - 1] / di[n - 1];
    sn[nz - 1] = x;
    for (int r = n - 2; r >= 0; r--) {
        x = (rhs[r] - up[r] * x) / di[r];
        if (r % 2 == 0) sn[r / 2] = x;
        else Wn[(r + 1) / 2] = x;
    }
    Wn[0] = 0.0;
    Wn[nz] = 0.0;
}

/* nshort HEVI short steps of length h, in place (fields as in the header).
 * When Mu is set, each short step also adds wgt times the mass fluxes its
 * density equation applies, (U*, V*, (1 - beta) W + beta W') on every face
 * (W' the new vertical momentum, interior faces only), to Mu, Mv, Mw. */
static void acoustic_run(int nx, int ny, int nz, double dx, double dy, const double *dz, const double *rho0c,
                         const double *rho0f, double cs2, double beta, double h, int nshort, double *U, double *V,
                         double *W, double *S, double *Mu, double *Mv, double *Mw, double wgt) {
    const long long plane = (long long)nx * ny, n = plane * nz;
    double *Us = (double *)malloc(n * sizeof(double)), *Vs = (double *)malloc(n * sizeof(double));
    double *Ss = (double *)malloc(n * sizeof(double));
    double *Up = (double *)malloc(n * sizeof(double)), *Vp = (double *)malloc(n * sizeof(double));
    for (int step = 0; step < nshort; step++) {
        for (int stage = 0; stage < 2; stage++) {
            const double tau = stage == 0 ? 0.5 * h : h;
            const double *se = stage == 0 ? S : Ss;        /* s that drives the horizontal momenta */
            double *Uo = stage == 0 ? Us : Up, *Vo = stage == 0 ? Vs : Vp;
            for (int k = 0; k < nz; k++)
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        const long long c = k * plane + (long long)j * nx + i;
                        const long long e = k * plane + (long long)j * nx + wrap(i + 1, nx);
                        const long long no = k * plane + (long long)wrap(j + 1, ny) * nx + i;
                        Uo[c] = U[c] - tau * cs2 * rho0c[k] * (se[e] - se[c]) / dx;
                        Vo[c] = V[c] - tau * cs2 * rho0c[k] * (se[no] - se[c]) / dy;
                    }
#ifdef _OPENMP
#pragma omp parallel
#endif
            {
                /* per column: Dh nz, Wc nz+1, sc nz, Wn nz+1, sn nz, and the four rows of
                 * the interleaved system, 2 nz - 1 each (2 nz allotted): 13 nz + 2 doubles */
                double *col = (double *)malloc((size_t)(13 * nz + 2) * sizeof(double));
                double *Dh = col, *Wc = Dh + nz, *sc = Wc + nz + 1, *Wn = sc + nz, *sn = Wn + nz + 1;
                double *lo = sn + nz, *di = lo + 2 * nz, *up = di + 2 * nz, *rhs = up + 2 * nz;
#ifdef _OPENMP
#pragma omp for
#endif
                for (long long q = 0; q < plane; q++) {
                    const int j = (int)(q / nx), i = (int)(q % nx);
                    const long long w = (long long)j * nx + wrap(i - 1, nx), so = (long long)wrap(j - 1, ny) * nx + i;
                    for (int k = 0; k < nz; k++) {
                        const long long c = k * plane + q;
                        Dh[k] = (Us[c] - Us[k * plane + w]) / dx + (Vs[c] - Vs[k * plane + so]) / dy;
                        sc[k] = S[c];
                    }
                    for (int f = 0; f <= nz; f++) Wc[f] = W[f * plane + q];
                    acoustic_column(nz, dz, rho0c, rho0f, cs2, beta, tau, Dh, Wc, sc, Wn, sn, lo, di, up, rhs);
                    if (stage == 0) {
                        for (int k = 0; k < nz; k++) Ss[k * plane + q] = sn[k];
                    } else {
                        if (Mu) {
                            for (int k = 0; k < nz; k++) {
                                Mu[k * plane + q] += wgt * Us[k * plane + q];
                                Mv[k * plane + q] += wgt * Vs[k * plane + q];
                            }
                            for (int f = 1; f < nz; f++)
                                Mw[f * plane + q] += wgt * ((1.0 - beta) * Wc[f] + beta * Wn[f]);
                        }
                        for (int k = 0; k < nz; k++) S[k * plane + q] = sn[k];
                        for (int f = 1; f < nz; f++) W[f * plane + q] = Wn[f];
                    }
                }
                free(col);
            }
        }
        memcpy(U, Up, n * sizeof(double));
        memcpy(V, Vp, n * sizeof(double));
    }
    free(Us); free(Vs); free(Ss); free(Up); free(Vp);
}

void orc_acoustic(int nx, int ny, int nz, double dx, double dy, const double *dz, const double *rho0c,
                  const double *rho0f, double cs2, double beta, double h, int nshort, double *U, double *V,
                  double *W, double *S) {
    acoustic_run(nx, ny, nz, dx, dy, dz, rho0c, rho0f, cs2, beta, h, nshort, U, V, W, S, NULL, NULL, NULL, 0.0);
}

/* short steps of RK stage q (weights 1/3, 1/2, 1) for ns short steps per long step */
int orc_hevi_short_steps(int ns, int q) {
    const double frac = q == 0 ? 1.0 / 3.0 : (q == 1 ? 0.5 : 1.0);
    const int n = (int)floor(frac * ns + 0.5);
    return n < 1 ? 1 : n;
}

/* ---- HEVI short steps nested in the RK3 long step (Sec. 1.1) --------------
 * The momenta U, V, W (the mass fluxes of the C grid) are prognostic and
 * evolve by the linear acoustic-gravity system of orc_acoustic; the scalar
 * fields are advected by them.  Wicker-Skamarock splitting: RK stage q
 * (weight c_q = 1/3, 1/2, 1) integrates the fast system from t^n over c_q dt
 * in n_q short steps (orc_hevi_short_steps) from (U, V, W)^n and
 * s^n = rho^n / rho0 - 1, and its scalar update Y^(q) = Y^n + c_q dt R(Y^(q-1))
 * advects with the short steps' mean effective mass fluxes
 *   Mbar = (1 / n_q) sum_m (U*_m, V*_m, (1 - beta) W_m + beta W_(m+1)),
 * the fluxes whose divergence the acoustic density equation applies, so the
 * advected density stays rho0 (1 + s) of the acoustic integration.  The third
 * stage's integration gives (U, V, W)^{n+1} (and s_final, if set).  Then the
 * column pass.  Fields: U, V [nz][ny][nx], W [nz+1][ny][nx] (lids kept). */
void orc_step_hevi(const orc_grid *g, double *Y, double *U, double *V, double *W, const double *tend,
                   const double *rho0c, const double *rho0f, double cs2, double beta, int ns, double dt,
                   int nsteps, double *s_final, double *budgets, double *stage_rho) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const size_t plane = (size_t)nx * ny, C = plane * nz, n = (size_t)(2 + g->ntr) * C, CW = C + plane;
    double *Yn = (double *)malloc(n * sizeof(double)), *Ys = (double *)malloc(n * sizeof(double));
    double *R = (double *)malloc(n * sizeof(double));
    double *pc = (double *)calloc(plane, sizeof(double));
    double *Sn = (double *)malloc(C * sizeof(double)), *Sa = (double *)malloc(C * sizeof(double));
    double *Ua = (double *)malloc(C * sizeof(double)), *Va = (double *)malloc(C * sizeof(double));
    double *Wa = (double *)malloc(CW * sizeof(double));
    double *Mu = (double *)malloc(C * sizeof(double)), *Mv = (double *)malloc(C * sizeof(double));
    double *Mw = (double *)malloc(CW * sizeof(double));
    const double c[3] = {dt / 3.0, dt / 2.0, dt};
    for (int step = 0; step < nsteps; step++) {
        memcpy(Yn, Y, n * sizeof(double));
        for (int k = 0; k < nz; k++)
            for (size_t q = 0; q < plane; q++) Sn[k * plane + q] = Y[k * plane + q] / rho0c[k] - 1.0;
        const double *in = Yn;
        for (int q = 0; q < 3; q++) {
            const int nq = orc_hevi_short_steps(ns, q);
            memcpy(Ua, U, C * sizeof(double));
            memcpy(Va, V, C * sizeof(double));
            memcpy(Wa, W, CW * sizeof(double));
            memcpy(Sa, Sn, C * sizeof(double));
            memset(Mu, 0, C * sizeof(double));
            memset(Mv, 0, C * sizeof(double));
            memset(Mw, 0, CW * sizeof(double));
            acoustic_run(nx, ny, nz, g->dx, g->dy, g->dz, rho0c, rho0f, cs2, beta, c[q] / nq, nq, Ua, Va, Wa, Sa,
                         Mu, Mv, Mw, 1.0 / nq);
            orc_rhs(g, in, Mu, Mv, Mw, tend, R, NULL);
            double *dst = q == 2 ? Y : Ys;
            for (size_t e = 0; e < n; e++) dst[e] = Yn[e] + c[q] * R[e];
            if (stage_rho && q < 2) memcpy(stage_rho + q * C, Ys, C * sizeof(double));
            in = Ys;
        }
        memcpy(U, Ua, C * sizeof(double));
        memcpy(V, Va, C * sizeof(double));
        memcpy(W, Wa, CW * sizeof(double));
        if (s_final) memcpy(s_final, Sa, C * sizeof(double));
        orc_column(g, Y, dt, pc);
    }
    if (budgets) {
        csum tot = {0.0, 0.0};
        for (size_t q = 0; q < plane; q++) csum_add(&tot, pc[q]);
        orc_budgets(g, Y, csum_value(&tot), budgets);
    }
    free(Yn); free(Ys); free(R); free(pc); free(Sn); free(Sa); free(Ua); free(Va); free(Wa);
    free(Mu); free(Mv); free(Mw);
}
