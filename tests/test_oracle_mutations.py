"""Mutation check of the oracle's pins.

Each entry below plants one plausible slip in a copy of the oracle's C source
(a sign, an index, a weight, a transposed coefficient, a dropped factor), the
copy is compiled with the oracle's own flags, and the CPU pin suites run
against it in a child process (the oracle module loads the copy through
ORACLE_LIBRARY).  Every mutant must make at least one pin fail; an
unmutated copy, built and loaded the same way, must pass them all.  A slip
that no pin notices would be a slip the oracle could carry into every GPU
parity test unseen.

Each slip is a literal text substitution that must match the source exactly
once, so an edit of the oracle that moves a line fails here loudly instead of
silently testing nothing.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "asuca_oracle.c")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py", "tests/test_oracle_open.py",
             "tests/test_oracle_hevi.py"]

# the RK3 stage weights, as written in each step of the oracle, and a slip of them
W3 = "const double c[3] = {dt / 3.0, dt / 2.0, dt};"
W2 = "const double c[3] = {dt / 2.0, dt / 2.0, dt};"

# (name, original text, slip): Koren limiter and upwind face
MUTANTS = [
    ("koren kappa weights swapped",
     "double t2 = (a0 + 2.0 * a1) / 3.0;", "double t2 = (2.0 * a0 + a1) / 3.0;"),
    ("koren 2r term on the wrong difference",
     "double t1 = 2.0 * a1;", "double t1 = 2.0 * a0;"),
    ("koren cap at 1 instead of 2",
     "double t3 = 2.0 * a0;", "double t3 = a0;"),
    ("koren sign of the increment",
     "L = d0 > 0.0 ? m : -m;", "L = d0 > 0.0 ? -m : m;"),
    ("koren limits only rising slopes",
     "int same = (d0 > 0.0 && d1 > 0.0) || (d0 < 0.0 && d1 < 0.0);", "int same = (d0 > 0.0 && d1 > 0.0);"),
    ("upwind tie M = 0 taken from the right",
     "if (m >= 0.0) {\n        double d0 = p0 - pm1, d1 = p1 - p0;",
     "if (m > 0.0) {\n        double d0 = p0 - pm1, d1 = p1 - p0;"),
    ("negative-flow differences reversed",
     "double d0 = p1 - p2, d1 = p0 - p1;", "double d0 = p2 - p1, d1 = p1 - p0;"),
    ("half of the limited increment dropped",
     "return p0 + 0.5 * orc_limiter(d0, d1, lim, branch);", "return p0 + orc_limiter(d0, d1, lim, branch);"),
    # flux form and divergence
    ("i flux difference reversed",
     "double r = -((xp - xm) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k]);\n"
     "                    if (tend && f > 0) {",
     "double r = -((xm - xp) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k]);\n"
     "                    if (tend && f > 0) {"),
    ("j divergence divided by dx",
     "double r = -((xp - xm) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k]);\n"
     "                    if (tend && f > 0) {",
     "double r = -((xp - xm) / g->dx + (yp - ym) / g->dx + (zp - zm) / g->dz[k]);\n"
     "                    if (tend && f > 0) {"),
    ("k divergence divided by the level below's dz",
     "double r = -((xp - xm) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k]);\n"
     "                    if (tend && f > 0) {",
     "double r = -((xp - xm) / g->dx + (yp - ym) / g->dy + (zp - zm) / g->dz[k > 0 ? k - 1 : 0]);\n"
     "                    if (tend && f > 0) {"),
    ("j faces carry the i mass flux",
     "m = mv[gidx(g, k, gj, gi)];", "m = mu[gidx(g, k, gj, gi)];"),
    ("vertical mass flux one level low",
     "m = mw[gidx(g, k + 1, gj, gi)];", "m = mw[gidx(g, k, gj, gi)];"),
    ("top ghost mirrors instead of copying",
     "int kp2 = k + 2 > nz - 1 ? nz - 1 : k + 2;", "int kp2 = k + 2 > nz - 1 ? nz - 2 : k + 2;"),
    # RK3
    ("first RK weight 1/2",
     "const double c[3] = {dt / 3.0, dt / 2.0, dt};\n    const int F = 2 + g->ntr, nz = g->nz;",
     "const double c[3] = {dt / 2.0, dt / 2.0, dt};\n    const int F = 2 + g->ntr, nz = g->nz;"),
    ("RK stages start from the previous stage",
     "dst[o] = Yn[o] + c[s] * R[o];", "dst[o] = Ys[o] + c[s] * R[o];"),
    # column physics
    ("Thomas elimination with the upper coefficient",
     "dp[k] = (d[k] - a[k] * dp[k - 1]) / den;", "dp[k] = (d[k] - c[k] * dp[k - 1]) / den;"),
    ("Thomas back substitution sign",
     "x[k] = dp[k] - cp[k] * x[k + 1];", "x[k] = dp[k] + cp[k] * x[k + 1];"),
    ("face density not averaged",
     "double rhof = 0.5 * (Y[k * cs] + Y[(k + 1) * cs]);", "double rhof = Y[k * cs];"),
    ("diffusion diagonal misses the lower face",
     "b[k] = Y[k * cs] * g->dz[k] + gf[k] + gf[k + 1];", "b[k] = Y[k * cs] * g->dz[k] + gf[k + 1];"),
    ("diffusivity taken at the cell centre",
     "double K = g->k0 * exp(-zf[k + 1] / g->kh);\n            double dzc",
     "double K = g->k0 * exp(-zc[k] / g->kh);\n            double dzc"),
    ("sedimentation flux halved",
     "P = g->vsed * q[k * cs];", "P = 0.5 * g->vsed * q[k * cs];"),
    ("sedimentation denominator without dt",
     "q[k * cs] = (q[k * cs] * dz + dt * P) / (dz + dt * g->vsed);",
     "q[k * cs] = (q[k * cs] * dz + dt * P) / (dz + g->vsed);"),
    ("precipitation without dt",
     "*precip += dt * P * g->dx * g->dy;", "*precip += P * g->dx * g->dy;"),
    ("relaxation target at the face height",
     "th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + r);\n            Y[fs + k * cs]",
     "th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zf[k])) / (1.0 + r);\n            Y[fs + k * cs]"),
    ("relaxation implicit factor doubled",
     "th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + r);\n            Y[fs + k * cs]",
     "th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + 2.0 * r);\n            Y[fs + k * cs]"),
    # budgets and the window
    ("budget without the layer depth",
     "Y[f * fs + k * cs + (size_t)j * g->nx + i] * g->dz[k] * g->dx * g->dy",
     "Y[f * fs + k * cs + (size_t)j * g->nx + i] * g->dx * g->dy"),
    ("compensation term of the wrong order",
     "if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;", "if (fabs(a->s) >= fabs(x)) a->c += (x - t) + a->s;"),
    ("window cone too narrow",
     "const int F = 2 + g->ntr, nz = g->nz, r = 6 * nsteps;", "const int F = 2 + g->ntr, nz = g->nz, r = 4 * nsteps;"),
    # tangent-linear and adjoint
    ("frozen kappa branch weights swapped",
     "case 2: *a = 1.0 / 3.0; *b = 2.0 / 3.0; break;", "case 2: *a = 2.0 / 3.0; *b = 1.0 / 3.0; break;"),
    ("adjoint of phi = u / rho: density term sign",
     "lamY[st[q]] -= lph * ph[q] / rho;", "lamY[st[q]] += lph * ph[q] / rho;"),
    ("adjoint flux difference at the wrong level",
     "const double lF = lamR[(size_t)f * C + b] * rdelta(g, dir, kb) -",
     "const double lF = lamR[(size_t)f * C + b] * rdelta(g, dir, k) -"),
    ("column tangent drops the density perturbation",
     "dOut[(size_t)f * nz + k] = drho[k] * ph[k] + w->Yb[k] * x[k];",
     "dOut[(size_t)f * nz + k] = w->Yb[k] * x[k];"),
    ("sedimentation adjoint with the wrong layer",
     "if (k > 0) nu += dt * g->vsed / (g->dz[k - 1] + dt * g->vsed) * nu_prev;",
     "if (k > 0) nu += dt * g->vsed / (g->dz[k] + dt * g->vsed) * nu_prev;"),
    # open boundaries
    ("east ghosts read from the west strip",
     "if (i >= g->nx) return ghost[halo_index(g, 1, f - 1, k, i - g->nx, j)];",
     "if (i >= g->nx) return ghost[halo_index(g, 0, f - 1, k, i - g->nx, j)];"),
    ("open j faces with the level pitch of the cells",
     "m = mv_x[((size_t)k * (ny + 1) + (j + 1)) * nx + i];", "m = mv_x[((size_t)k * ny + (j + 1)) * nx + i];"),
    # 7-point stencil, damping
    ("7-point stencil wraps through the lids",
     "ku = k < nz - 1 ? k + 1 : nz - 1;", "ku = k < nz - 1 ? k + 1 : 0;"),
    ("7-point stencil centre weight of a 2-D Laplacian",
     "v + c * (sum - 6.0 * v)", "v + c * (sum - 4.0 * v)"),
    ("damping target with the boundary datasets swapped",
     "mtratio * (ref[q] + b0[q]) + tratio * (ref[q] + b1[q]) - ref[q]",
     "mtratio * (ref[q] + b1[q]) + tratio * (ref[q] + b0[q]) - ref[q]"),
    ("damping ramp reversed",
     "const double x = (double)(width - d) / width;", "const double x = (double)d / width;"),
    ("damping explicit instead of implicit",
     "y[q] = (y[q] + a * target) / (1.0 + a);", "y[q] = y[q] + a * (target - y[q]);"),
    # acoustic short steps and their nesting
    ("acoustic first stage of full length",
     "const double tau = stage == 0 ? 0.5 * h : h;", "const double tau = h;"),
    ("acoustic vertical spacing of the upper level only",
     "const double dzc = 0.5 * (dz[f - 1] + dz[f]);\n        const double g = tau",
     "const double dzc = dz[f];\n        const double g = tau"),
    ("acoustic off-centring weights swapped",
     "rhs[r] = W[f] - g * (1.0 - beta) * (s[f] - s[f - 1]);", "rhs[r] = W[f] - g * beta * (s[f] - s[f - 1]);"),
    ("acoustic pressure gradient sign in i",
     "Uo[c] = U[c] - tau * cs2 * rho0c[k] * (se[e] - se[c]) / dx;",
     "Uo[c] = U[c] - tau * cs2 * rho0c[k] * (se[c] - se[e]) / dx;"),
    ("short steps per stage truncated",
     "const int n = (int)floor(frac * ns + 0.5);", "const int n = (int)floor(frac * ns);"),
    ("mean vertical flux from the new momentum only",
     "Mw[f * plane + q] += wgt * ((1.0 - beta) * Wc[f] + beta * Wn[f]);", "Mw[f * plane + q] += wgt * Wn[f];"),
    ("mean i flux of the stage-2 momentum",
     "Mu[k * plane + q] += wgt * Us[k * plane + q];", "Mu[k * plane + q] += wgt * Up[k * plane + q];"),
    ("every stage integrates over the whole long step",
     "c[q] / nq, nq, Ua", "dt / nq, nq, Ua"),
    ("acoustic j gradient divided by dx",
     "Vo[c] = V[c] - tau * cs2 * rho0c[k] * (se[no] - se[c]) / dy;",
     "Vo[c] = V[c] - tau * cs2 * rho0c[k] * (se[no] - se[c]) / dx;"),
    ("acoustic i divergence divided by dy",
     "Dh[k] = (Us[c] - Us[k * plane + w]) / dx + (Vs[c] - Vs[k * plane + so]) / dy;",
     "Dh[k] = (Us[c] - Us[k * plane + w]) / dy + (Vs[c] - Vs[k * plane + so]) / dy;"),
    ("acoustic lower coefficient with the level below's dz",
     "lo[r] = k > 0 ? -tau * beta / dz[k] : 0.0;", "lo[r] = k > 0 ? -tau * beta / dz[k - 1] : 0.0;"),
    ("acoustic face density taken at the centre",
     "const double g = tau * cs2 * rho0f[f] / dzc;", "const double g = tau * cs2 * rho0c[f] / dzc;"),
    # more of the step, the damping and the derivatives
    ("forcing read with i and j swapped",
     "r += tend[(size_t)(f - 1) * nz * g->ny * g->nx + gidx(g, k, gj, gi)];",
     "r += tend[(size_t)(f - 1) * nz * g->ny * g->nx + gidx(g, k, gi, gj)];"),
    ("column physics before the dynamics",
     "        orc_rk3(g, Y, mu, mv, mw, tend, dt);\n        orc_column(g, Y, dt, pc);",
     "        orc_column(g, Y, dt, pc);\n        orc_rk3(g, Y, mu, mv, mw, tend, dt);"),
    ("linear scheme weights swapped",
     "L = (d0 + 2.0 * d1) / 3.0;", "L = (2.0 * d0 + d1) / 3.0;"),
    ("open domain reads rho phi as phi",
     "return Y[(size_t)f * C + o] / Y[o];", "return Y[(size_t)f * C + o];"),
    ("precipitation left out of the budget",
     "        orc_budgets(g, Y, csum_value(&tot), budgets);\n    }\n    free(pc);\n}",
     "        orc_budgets(g, Y, 0.0, budgets);\n    }\n    free(pc);\n}"),
    ("7-point stencil wraps j by nx",
     "ju = wrap(j + 1, ny);", "ju = wrap(j + 1, nx);"),
    ("damping top zone one level short",
     "if (ntop > 0 && k >= nz - ntop) {", "if (ntop > 0 && k > nz - ntop) {"),
    ("damping top ramp linear",
     "top = nu_top * (x * x);", "top = nu_top * x;"),
    ("tangent of phi = u / rho: density term sign",
     "dph[q] = (dY[(size_t)f * C + st[q]] - ph[q] * dY[st[q]]) / rho;",
     "dph[q] = (dY[(size_t)f * C + st[q]] + ph[q] * dY[st[q]]) / rho;"),
    ("relaxation adjoint without the implicit factor",
     "lam[nz + k] = lt / (1.0 + r);", "lam[nz + k] = lt;"),
    ("column tangent's diffusion derivative doubled",
     "w->kcf[k + 1] = 0.5 * dt * K / (zc[k + 1] - zc[k]);", "w->kcf[k + 1] = dt * K / (zc[k + 1] - zc[k]);"),
    ("column adjoint's diffusion term sign",
     "if (k > 0) lr -= w->kcf[k] * (psi[k] - psi[k - 1]) * (ph[k] - ph[k - 1]);",
     "if (k > 0) lr += w->kcf[k] * (psi[k] - psi[k - 1]) * (ph[k] - ph[k - 1]);"),
    ("step adjoint drops the path through stage 1",
     "lam[e] += l2[e] + l1[e];", "lam[e] += l2[e];"),
    ("step tangent builds each stage on the previous one",
     "dS[e] = dY[e] + c[q] * dR[e];", "dS[e] = dS[e] + c[q] * dR[e];"),
    ("tangent drops the mass-flux perturbation",
     "dF = dm * face + m * dface;", "dF = m * dface;"),
    ("west ghost columns in reverse order",
     "halo_index(g, 0, f - 1, k, i + 2, j)", "halo_index(g, 0, f - 1, k, -1 - i, j)"),
    ("north ghosts read from the south strip",
     "if (j >= g->ny) return ghost[halo_index(g, 3, f - 1, k, j - g->ny, i)];",
     "if (j >= g->ny) return ghost[halo_index(g, 2, f - 1, k, j - g->ny, i)];"),
    ("open vertical mass flux one level low",
     "m = mw[((size_t)(k + 1) * ny + j) * nx + i];", "m = mw[((size_t)k * ny + j) * nx + i];"),
    ("7-point stencil's lower neighbour taken from above",
     "in[kd * plane + (long long)j * nx + i] + in[ku * plane + (long long)j * nx + i];",
     "in[ku * plane + (long long)j * nx + i] + in[ku * plane + (long long)j * nx + i];"),
    ("damping zone ignores the j edges",
     "if (j < d) d = j;", "if (j < 0) d = j;"),
    ("damping overlap takes the smaller rate",
     "return lat > top ? lat : top;", "return lat > top ? top : lat;"),
    ("acoustic elimination with the lower coefficient",
     "di[r] -= m * up[r - 1];", "di[r] -= m * lo[r - 1];"),
    ("acoustic second stage driven by the starting s",
     "const double *se = stage == 0 ? S : Ss;", "const double *se = S;"),
    ("nested step's s without the -1",
     "Y[k * plane + q] / rho0c[k] - 1.0;", "Y[k * plane + q] / rho0c[k];"),
    # the RK weights and budgets of the other steps, forcing in the window and
    # the open domain, the precipitation sum, the remaining index slips
    ("stage states of the derivatives: first weight 1/2",
     W3 + "\n    double *outs[3]", W2 + "\n    double *outs[3]"),
    ("tangent-linear step: first weight 1/2",
     W3 + "\n    memcpy(Y, Y0, n * sizeof(double));\n    memcpy(dY",
     W2 + "\n    memcpy(Y, Y0, n * sizeof(double));\n    memcpy(dY"),
    ("adjoint step: first weight 1/2",
     W3 + "\n    memcpy(lam, lam_final", W2 + "\n    memcpy(lam, lam_final"),
    ("branch trajectory: first weight 1/2",
     W3 + "\n    memcpy(Y, Y0, n * sizeof(double));\n    for (int s = 0; s < nsteps; s++) {\n        const double *in = Y;",
     W2 + "\n    memcpy(Y, Y0, n * sizeof(double));\n    for (int s = 0; s < nsteps; s++) {\n        const double *in = Y;"),
    ("open step: first weight 1/2",
     W3 + "\n    for (int s = 0; s < nsteps; s++) {\n        memcpy(Yn, Y",
     W2 + "\n    for (int s = 0; s < nsteps; s++) {\n        memcpy(Yn, Y"),
    ("nested step: first weight 1/2",
     W3 + "\n    for (int step = 0; step < nsteps; step++) {", W2 + "\n    for (int step = 0; step < nsteps; step++) {"),
    ("open budget without the precipitation",
     "csum_add(&tot, pc[(size_t)j * g->nx + i]);\n        orc_budgets(g, Y, csum_value(&tot), budgets);\n    }\n    free(Yn);",
     "csum_add(&tot, pc[(size_t)j * g->nx + i]);\n        orc_budgets(g, Y, 0.0, budgets);\n    }\n    free(Yn);"),
    ("nested step's budget without the precipitation",
     "for (size_t q = 0; q < plane; q++) csum_add(&tot, pc[q]);\n        orc_budgets(g, Y, csum_value(&tot), budgets);",
     "for (size_t q = 0; q < plane; q++) csum_add(&tot, pc[q]);\n        orc_budgets(g, Y, 0.0, budgets);"),
    ("7-point stencil wraps i by ny",
     "iu = wrap(i + 1, nx);", "iu = wrap(i + 1, ny);"),
    ("window without the forcing",
     "rk3_patch(g, &p, P, mu, mv, mw, tend, dt, margin, 2);", "rk3_patch(g, &p, P, mu, mv, mw, NULL, dt, margin, 2);"),
    ("open domain without the forcing",
     "if (tend && f > 0) r += tend[o - (size_t)nz * ny * nx];",
     "if (0 && tend && f > 0) r += tend[o - (size_t)nz * ny * nx];"),
    ("precipitation of a column overwritten each step",
     "if (precip_col) precip_col[(size_t)lj * p->pw + li] += pr;",
     "if (precip_col) precip_col[(size_t)lj * p->pw + li] = pr;"),
    ("mean j flux of the stage-2 momentum",
     "Mv[k * plane + q] += wgt * Vs[k * plane + q];", "Mv[k * plane + q] += wgt * Vp[k * plane + q];"),
    ("sampled damping cells with i and j swapped",
     "i = ijk[3 * c];\n            j = ijk[3 * c + 1];", "j = ijk[3 * c];\n            i = ijk[3 * c + 1];"),
    ("Thomas first row divided by the next diagonal",
     "cp[0] = c[0] / b[0];", "cp[0] = c[0] / b[1];"),
    ("level centres from the upper face",
     "zc[k] = zf[k] + 0.5 * g->dz[k];", "zc[k] = zf[k + 1] + 0.5 * g->dz[k];"),
    ("diffusion weight without dt",
     "gf[k + 1] = dt * rhof * K / dzc;", "gf[k + 1] = rhof * K / dzc;"),
    ("diffusion right-hand side without dz",
     "d[k] = g->dz[k] * Y[f * fs + k * cs];", "d[k] = Y[f * fs + k * cs];"),
    ("diffusion result stored as phi",
     "Y[f * fs + k * cs] = Y[k * cs] * x[k];", "Y[f * fs + k * cs] = x[k];"),
    ("acoustic upper coefficient with the level above's dz",
     "up[r] = k < nz - 1 ? tau * beta / dz[k] : 0.0;", "up[r] = k < nz - 1 ? tau * beta / dz[k + 1] : 0.0;"),
    ("acoustic density equation's off-centring swapped",
     "rhs[r] = rho0c[k] * s[k] - tau * Dh[k] - tau * (1.0 - beta) * (Wk1 - Wk) / dz[k];",
     "rhs[r] = rho0c[k] * s[k] - tau * Dh[k] - tau * beta * (Wk1 - Wk) / dz[k];"),
    ("acoustic back substitution sign",
     "x = (rhs[r] - up[r] * x) / di[r];", "x = (rhs[r] + up[r] * x) / di[r];"),
    ("mean fluxes summed instead of averaged",
     "Mu, Mv, Mw, 1.0 / nq);", "Mu, Mv, Mw, 1.0);"),
    ("damping target without the reference state",
     "const double target = ref[q] + ptb;", "const double target = ptb;"),
    ("7-point stencil's bottom ghost mirrors",
     "const int kd = k > 0 ? k - 1 : 0,", "const int kd = k > 0 ? k - 1 : 1,"),
    ("tangent face coefficient sign",
     "c[1] = 1.0 + 0.5 * a - 0.5 * b; c[2] = 0.5 * b; c[3] = 0.0;",
     "c[1] = 1.0 - 0.5 * a - 0.5 * b; c[2] = 0.5 * b; c[3] = 0.0;"),
    ("tangent and adjoint divide j differences by dx",
     "(dir == 1 ? 1.0 / g->dy : 1.0 / g->dz[k])", "(dir == 1 ? 1.0 / g->dx : 1.0 / g->dz[k])"),
    ("tangent and adjoint take the vertical flux a level low",
     "return dir == 2 ? gidx(g, k + 1, j, i) : gidx(g, k, j, i);", "return dir == 2 ? gidx(g, k, j, i) : gidx(g, k, j, i);"),
    ("column tangent's relaxation drops the density term",
     "r * (THETA_REF0 + THETA_REF_LAPSE * zc[k]) * dY3[k]) / (1.0 + r);",
     "r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + r);"),
    ("column adjoint's sedimentation without dz",
     "lq[k] = nu * g->dz[k] / (g->dz[k] + dt * g->vsed);", "lq[k] = nu / (g->dz[k] + dt * g->vsed);"),
    ("column adjoint's diffusion right-hand side without the density",
     "d[k] = w->Yb[k] * lu[k];", "d[k] = lu[k];"),
    ("column adjoint's upper face term with the lower face's weight",
     "if (k < nz - 1) lr -= w->kcf[k + 1] * (psi[k] - psi[k + 1]) * (ph[k] - ph[k + 1]);",
     "if (k < nz - 1) lr -= w->kcf[k] * (psi[k] - psi[k + 1]) * (ph[k] - ph[k + 1]);"),
    ("column adjoint's result without dz",
     "lu[k] = g->dz[k] * psi[k];", "lu[k] = psi[k];"),
    ("column adjoint's relaxation drops the reference profile",
     "lam[k] += lt * r * (THETA_REF0 + THETA_REF_LAPSE * zc[k]) / (1.0 + r);", "lam[k] += lt * r / (1.0 + r);"),
    ("south ghost rows in reverse order",
     "if (j < 0) return ghost[halo_index(g, 2, f - 1, k, j + 2, i)];",
     "if (j < 0) return ghost[halo_index(g, 2, f - 1, k, -1 - j, i)];"),
    ("south and north strips as long as the west and east ones",
     "const size_t len = strip < 2 ? (size_t)g->ny : (size_t)g->nx;",
     "const size_t len = strip < 2 ? (size_t)g->ny : (size_t)g->ny;"),
    ("7-point stencil's lower j neighbour two rows away",
     "const int jd = wrap(j - 1, ny), ju = wrap(j + 1, ny);", "const int jd = wrap(j - 2, ny), ju = wrap(j + 1, ny);"),
    ("damping weight of the first dataset taken as 1 - tratio",
     "const double ptb = mtratio * (ref[q] + b0[q])", "const double ptb = (1.0 - tratio) * (ref[q] + b0[q])"),
    ("acoustic vertical force with the face density below",
     "const double g = tau * cs2 * rho0f[f] / dzc;", "const double g = tau * cs2 * rho0f[f - 1] / dzc;"),
    ("acoustic elimination of the right-hand side sign",
     "rhs[r] -= m * rhs[r - 1];", "rhs[r] += m * rhs[r - 1];"),
    ("nested step keeps the old V",
     "memcpy(V, Va, C * sizeof(double));", "memcpy(V, V, C * sizeof(double));"),
    ("linear scheme recorded as the 2r branch",
     "br = 2;\n        L = (d0 + 2.0 * d1) / 3.0;", "br = 1;\n        L = (d0 + 2.0 * d1) / 3.0;"),
    ("branch trajectory builds each stage on the previous one",
     "S[e] = Y[e] + c[q] * R[e];", "S[e] = S[e] + c[q] * R[e];"),
    ("step adjoint's first stage with the second weight",
     "mu_r[e] = c[0] * l1[e];", "mu_r[e] = c[1] * l1[e];"),
    ("a stage may get no short step",
     "return n < 1 ? 1 : n;", "return n;"),
    ("acoustic momentum unknown stored a face low",
     "else Wn[(r + 1) / 2] = x;", "else Wn[(r - 1) / 2] = x;"),
    ("acoustic lower coefficient's sign",
     "lo[r] = k > 0 ? -tau * beta / dz[k] : 0.0;", "lo[r] = k > 0 ? tau * beta / dz[k] : 0.0;"),
    ("acoustic density equation reads the lids' momenta",
     "const double Wk = k > 0 ? W[k] : 0.0, Wk1 = k < nz - 1 ? W[k + 1] : 0.0;",
     "const double Wk = W[k], Wk1 = W[k + 1];"),
    ("first-order upwind recorded as the cap branch",
     "br = 0;\n        L = 0.0;\n    } else if (lim == 1)", "br = 3;\n        L = 0.0;\n    } else if (lim == 1)"),
    ("relaxation toward 300 K at every height",
     "th = (th + r * (THETA_REF0 + THETA_REF_LAPSE * zc[k])) / (1.0 + r);\n            Y[fs + k * cs]",
     "th = (th + r * (THETA_REF0)) / (1.0 + r);\n            Y[fs + k * cs]"),
    ("precipitation with an extra factor dx",
     "*precip += dt * P * g->dx * g->dy;", "*precip += dt * P * g->dx * g->dy * g->dx;"),
]


def _run_pins(so, timeout=600):
    env = dict(os.environ, ORACLE_LIBRARY=so, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    return r.returncode, (r.stdout + r.stderr)[-2000:]


def _mutant(tmp, idx, name, old, new, src):
    c = os.path.join(tmp, f"mutant{idx}.c")
    with open(c, "w") as fh:
        fh.write(src.replace(old, new))
    so = oracle.compile_library(c, os.path.join(tmp, f"libmutant{idx}.so"))
    return name, _run_pins(so)


def test_every_slip_fails_a_pin(tmp_path):
    src = open(SRC).read()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, f"'{name}': the original text occurs {src.count(old)} times"
        assert old != new
    tmp = str(tmp_path)
    # control: the unmutated source, built and loaded the same way, passes
    control = oracle.compile_library(SRC, os.path.join(tmp, "libcontrol.so"))
    rc, log = _run_pins(control)
    assert rc == 0, "the unmutated copy fails the pins:\n" + log
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = [ex.submit(_mutant, tmp, q, name, old, new, src) for q, (name, old, new) in enumerate(MUTANTS)]
        results = [f.result() for f in futs]
    # returncode 1: tests ran and at least one failed (not a crash or a collection error)
    survived = [(name, rc, log) for name, (rc, log) in results if rc != 1]
    assert not survived, "\n\n".join(f"'{n}' (rc {rc}):\n{log}" for n, rc, log in survived)
