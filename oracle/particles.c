/*
 * Particle-in-cell kernels, FP64: CIC field gather on the Yee grid, the
 * relativistic Boris push, the move with reflecting walls, and charge-
 * conserving Esirkepov current deposition.
 *
 * Paper: Methodology -- PIC macro-particles weighted by density-volume
 * fraction are advanced by the Boris pusher; particles that cross a domain
 * boundary have their velocity reversed; charge conservation is checked at
 * every step.  The paper does not name the deposition; the charge-conserving
 * scheme of Esirkepov (Comput. Phys. Commun. 135, 144 (2001)) with the
 * first-order (CIC) shape is used.
 *
 * Boris (Boris 1970; relativistic form as in Birdsall & Langdon):
 *   u-  = u^{n-1/2} + (q dt / 2m) E
 *   t   = (q dt / 2m gamma-) B,   s = 2 t / (1 + t.t)
 *   u'  = u- + u- x t,            u+ = u- + u' x s
 *   u^{n+1/2} = u+ + (q dt / 2m) E
 *   x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}
 *
 * Esirkepov (CIC), per node (i,j,k) of the 3-node window that holds both the
 * old and the new shape, with S0, S1 the 1D shape factors and DS = S1 - S0:
 *   W_x = DS_x (S0_y S0_z + DS_y S0_z / 2 + S0_y DS_z / 2 + DS_y DS_z / 3)
 * (and cyclic), and J_x(i+1/2) - J_x(i-1/2) = -q w W_x / (dt dy dz).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>

static inline long IDX(const orc_grid *g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)k);
}
static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

static int axis_n(const orc_grid *g, int a) { return a == 0 ? g->nx : (a == 1 ? g->ny : g->nz); }

/* resolve an index along axis a: wraps when periodic; -1 when it is outside a
 * non-periodic axis (the value there is zero) */
static int resolve(const orc_grid *g, int a, int i) {
    int n = axis_n(g, a);
    if (g->bc[a] == 0) return wrapi(i, n);
    return (i < 0 || i > n - 1) ? -1 : i;
}

/* CIC interpolation of one staggered component with offsets o[3] in {0, 1/2} */
static double interp(const orc_grid *g, const double *F, const double o[3], const double p[3]) {
    int base[3]; double f[3];
    for (int a = 0; a < 3; ++a) {
        double s = p[a] - o[a];
        int i = (int)floor(s);
        int n = axis_n(g, a);
        if (g->bc[a] != 0 && o[a] == 0.0 && i > n - 2) i = n - 2;  /* particle exactly on the top wall */
        base[a] = i; f[a] = s - i;
    }
    double acc = 0.0;
    for (int c = 0; c < 2; ++c) {
        int kk = resolve(g, 2, base[2] + c); if (kk < 0) continue;
        double wz = c ? f[2] : 1.0 - f[2];
        for (int b = 0; b < 2; ++b) {
            int jj = resolve(g, 1, base[1] + b); if (jj < 0) continue;
            double wy = b ? f[1] : 1.0 - f[1];
            for (int a = 0; a < 2; ++a) {
                int ii = resolve(g, 0, base[0] + a); if (ii < 0) continue;
                double wx = a ? f[0] : 1.0 - f[0];
                acc += wx * wy * wz * F[IDX(g, ii, jj, kk)];
            }
        }
    }
    return acc;
}

/* Quadratic (TSC) shape, Esirkepov's order 2: S(d) = 3/4 - d^2 for |d| <= 1/2,
 * (3/2 - |d|)^2 / 2 for 1/2 <= |d| <= 3/2, 0 beyond; a particle covers the
 * node nearest to it and its two neighbours. */
double orc_tsc(double d) {
    const double a = fabs(d);
    if (a <= 0.5) return 0.75 - a * a;
    if (a <= 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

/* TSC interpolation of one staggered component (offsets o[3] in {0, 1/2}) */
static double interp2(const orc_grid *g, const double *F, const double o[3], const double p[3]) {
    int m[3];
    double s[3];
    for (int a = 0; a < 3; ++a) {
        s[a] = p[a] - o[a];
        m[a] = (int)floor(s[a] + 0.5);
    }
    double acc = 0.0;
    for (int c = -1; c <= 1; ++c) {
        int kk = resolve(g, 2, m[2] + c); if (kk < 0) continue;
        double wz = orc_tsc(s[2] - (m[2] + c));
        for (int b = -1; b <= 1; ++b) {
            int jj = resolve(g, 1, m[1] + b); if (jj < 0) continue;
            double wy = orc_tsc(s[1] - (m[1] + b));
            for (int a = -1; a <= 1; ++a) {
                int ii = resolve(g, 0, m[0] + a); if (ii < 0) continue;
                acc += orc_tsc(s[0] - (m[0] + a)) * wy * wz * F[IDX(g, ii, jj, kk)];
            }
        }
    }
    return acc;
}

void orc_gather(const orc_grid *g, const double *E[3], const double *B[3],
                double xi, double yi, double zi, double e[3], double b[3]) {
    static const double off[6][3] = {
        {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},       /* Ex Ey Ez */
        {0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}  /* Bx By Bz */
    };
    const double p[3] = {xi, yi, zi};
    for (int c = 0; c < 3; ++c) {
        e[c] = g->order == 2 ? interp2(g, E[c], off[c], p) : interp(g, E[c], off[c], p);
        b[c] = g->order == 2 ? interp2(g, B[c], off[3 + c], p) : interp(g, B[c], off[3 + c], p);
    }
}

void orc_boris(double qm_dt_half, const double e[3], const double b[3], double u[3]) {
    double um[3], up[3], t[3], s[3], ud[3];
    for (int c = 0; c < 3; ++c) um[c] = u[c] + qm_dt_half * e[c];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int c = 0; c < 3; ++c) t[c] = qm_dt_half * b[c] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int c = 0; c < 3; ++c) s[c] = 2.0 * t[c] / (1.0 + t2);
    ud[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    ud[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    ud[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    up[0] = um[0] + (ud[1] * s[2] - ud[2] * s[1]);
    up[1] = um[1] + (ud[2] * s[0] - ud[0] * s[2]);
    up[2] = um[2] + (ud[0] * s[1] - ud[1] * s[0]);
    for (int c = 0; c < 3; ++c) u[c] = up[c] + qm_dt_half * e[c];
}

/* The relativistic pushers of Vay (Phys. Plasmas 15, 056701 (2008)) and of
 * Higuera & Cary (Phys. Plasmas 24, 052104 (2017)), both with h = q dt / 2m,
 * tau = h B.  They share the implicit step that rotates a momentum w about B
 * with the Lorentz factor of the new momentum:
 *   sigma = gamma_w^2 - tau^2,  u* = w . tau,
 *   gamma_new^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + u*^2))) / 2,
 *   t = tau / gamma_new,  s = 1 / (1 + t^2),
 *   R(w) = s (w + (w . t) t + w x t).
 * Vay:  w = u + h (2E + v x B) with v = u / gamma(u);  u_new = R(w).
 * HC:   w = u + h E;  u+ = R(w);  u_new = u+ + h E + u+ x t.
 * Both move a particle whose velocity is the drift E x B / B^2 (E.B = 0,
 * |E| < |B|) on a straight line with unchanged momentum, which Boris does not
 * for relativistic drifts. */
static void rotate_implicit(const double w[3], const double tau[3], double out[3], double t[3]) {
    const double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    const double us = w[0] * tau[0] + w[1] * tau[1] + w[2] * tau[2];
    const double sigma = 1.0 + w2 - tau2;
    const double g = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + us * us))));
    for (int c = 0; c < 3; ++c) t[c] = tau[c] / g;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double s = 1.0 / (1.0 + t2);
    const double wt = w[0] * t[0] + w[1] * t[1] + w[2] * t[2];
    out[0] = s * (w[0] + wt * t[0] + (w[1] * t[2] - w[2] * t[1]));
    out[1] = s * (w[1] + wt * t[1] + (w[2] * t[0] - w[0] * t[2]));
    out[2] = s * (w[2] + wt * t[2] + (w[0] * t[1] - w[1] * t[0]));
}

void orc_vay(double h, const double e[3], const double b[3], double u[3]) {
    const double g0 = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double v[3] = {u[0] / g0, u[1] / g0, u[2] / g0};
    const double tau[3] = {h * b[0], h * b[1], h * b[2]};
    double w[3], t[3];
    w[0] = u[0] + 2.0 * h * e[0] + (v[1] * tau[2] - v[2] * tau[1]);
    w[1] = u[1] + 2.0 * h * e[1] + (v[2] * tau[0] - v[0] * tau[2]);
    w[2] = u[2] + 2.0 * h * e[2] + (v[0] * tau[1] - v[1] * tau[0]);
    rotate_implicit(w, tau, u, t);
}

void orc_higuera_cary(double h, const double e[3], const double b[3], double u[3]) {
    const double tau[3] = {h * b[0], h * b[1], h * b[2]};
    const double w[3] = {u[0] + h * e[0], u[1] + h * e[1], u[2] + h * e[2]};
    double up[3], t[3];
    rotate_implicit(w, tau, up, t);
    u[0] = up[0] + h * e[0] + (up[1] * t[2] - up[2] * t[1]);
    u[1] = up[1] + h * e[1] + (up[2] * t[0] - up[0] * t[2]);
    u[2] = up[2] + h * e[2] + (up[0] * t[1] - up[1] * t[0]);
}

/* 1D CIC shape of a particle at position p on nodes base, base+1, base+2 */
static void shape3(double p, int base, double S[3]) {
    for (int k = 0; k < 3; ++k) {
        double d = fabs(p - (double)(base + k));
        S[k] = d < 1.0 ? 1.0 - d : 0.0;
    }
}

void orc_esirkepov(const orc_grid *g, double qw, double x0, double y0, double z0,
                   double x1, double y1, double z1, double *J[3]) {
    const double p0[3] = {x0, y0, z0}, p1[3] = {x1, y1, z1};
    int base[3]; double S0[3][3], DS[3][3];
    for (int a = 0; a < 3; ++a) {
        int i0 = (int)floor(p0[a]), i1 = (int)floor(p1[a]);
        base[a] = i0 < i1 ? i0 : i1;
        double s1[3];
        shape3(p0[a], base[a], S0[a]);
        shape3(p1[a], base[a], s1);
        for (int k = 0; k < 3; ++k) DS[a][k] = s1[k] - S0[a][k];
    }
    const double dvol[3] = {g->dy * g->dz, g->dx * g->dz, g->dx * g->dy};
    /* component c: axis c carries the prefix sum; axes p, q are the others */
    for (int c = 0; c < 3; ++c) {
        const int p = (c + 1) % 3, q = (c + 2) % 3;
        const double fac = -qw / (g->dt * dvol[c]);
        for (int bq = 0; bq < 3; ++bq)
        for (int bp = 0; bp < 3; ++bp) {
            double acc = 0.0;
            for (int a = 0; a < 2; ++a) {
                double W = DS[c][a] * (S0[p][bp] * S0[q][bq] + 0.5 * DS[p][bp] * S0[q][bq]
                                       + 0.5 * S0[p][bp] * DS[q][bq] + DS[p][bp] * DS[q][bq] / 3.0);
                acc += W;
                if (acc == 0.0) continue;
                int idx[3];
                idx[c] = resolve(g, c, base[c] + a);
                idx[p] = resolve(g, p, base[p] + bp);
                idx[q] = resolve(g, q, base[q] + bq);
                if (idx[0] < 0 || idx[1] < 0 || idx[2] < 0) continue;
                J[c][IDX(g, idx[0], idx[1], idx[2])] += fac * acc;
            }
        }
    }
}

/* Esirkepov with the quadratic shape: per axis the window of 4 nodes that
 * holds both the old and the new 3-node support (base = the smaller of the
 * two nearest nodes, minus one), the same W formula as for CIC, prefix-summed
 * over the 3 faces between the window's nodes. */
void orc_esirkepov2(const orc_grid *g, double qw, double x0, double y0, double z0,
                    double x1, double y1, double z1, double *J[3]) {
    const double p0[3] = {x0, y0, z0}, p1[3] = {x1, y1, z1};
    int base[3];
    double S0[3][4], DS[3][4];
    for (int a = 0; a < 3; ++a) {
        const int m0 = (int)floor(p0[a] + 0.5), m1 = (int)floor(p1[a] + 0.5);
        base[a] = (m0 < m1 ? m0 : m1) - 1;
        for (int k = 0; k < 4; ++k) {
            S0[a][k] = orc_tsc(p0[a] - (base[a] + k));
            DS[a][k] = orc_tsc(p1[a] - (base[a] + k)) - S0[a][k];
        }
    }
    const double dvol[3] = {g->dy * g->dz, g->dx * g->dz, g->dx * g->dy};
    for (int c = 0; c < 3; ++c) {
        const int p = (c + 1) % 3, q = (c + 2) % 3;
        const double fac = -qw / (g->dt * dvol[c]);
        for (int bq = 0; bq < 4; ++bq)
        for (int bp = 0; bp < 4; ++bp) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a) {
                double W = DS[c][a] * (S0[p][bp] * S0[q][bq] + 0.5 * DS[p][bp] * S0[q][bq]
                                       + 0.5 * S0[p][bp] * DS[q][bq] + DS[p][bp] * DS[q][bq] / 3.0);
                acc += W;
                if (acc == 0.0) continue;
                int idx[3];
                idx[c] = resolve(g, c, base[c] + a);
                idx[p] = resolve(g, p, base[p] + bp);
                idx[q] = resolve(g, q, base[q] + bq);
                if (idx[0] < 0 || idx[1] < 0 || idx[2] < 0) continue;
                J[c][IDX(g, idx[0], idx[1], idx[2])] += fac * acc;
            }
        }
    }
}

void orc_push_deposit(const orc_grid *g, const double *E[3], const double *B[3],
                      double *J[3], orc_species *s) {
    const double dt = g->dt;
    const double d[3] = {g->dx, g->dy, g->dz};
    const int n[3] = {g->nx, g->ny, g->nz};
    for (long p = 0; p < s->n; ++p) {
        const double q = s->zq ? s->q * s->zq[p] : s->q;
        double x0[3] = {s->x[p], s->y[p], s->z[p]};
        double e[3], b[3], u[3] = {s->ux[p], s->uy[p], s->uz[p]};
        orc_gather(g, E, B, x0[0], x0[1], x0[2], e, b);
        if (s->eb) {
            for (int c = 0; c < 3; ++c) { s->eb[6 * p + c] = e[c]; s->eb[6 * p + 3 + c] = b[c]; }
        }
        if (s->pusher == ORC_PUSH_VAY) orc_vay(q * dt / (2.0 * s->m), e, b, u);
        else if (s->pusher == ORC_PUSH_HC) orc_higuera_cary(q * dt / (2.0 * s->m), e, b, u);
        else orc_boris(q * dt / (2.0 * s->m), e, b, u);
        const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double x1[3];
        for (int a = 0; a < 3; ++a) {
            x1[a] = x0[a] + dt * u[a] / (gam * d[a]);
            if (g->bc[a] != 0) {             /* reflecting wall: reverse the normal momentum */
                const double L = (double)(n[a] - 1);
                if (x1[a] < 0.0)      { x1[a] = -x1[a];          u[a] = -u[a]; }
                else if (x1[a] > L)   { x1[a] = 2.0 * L - x1[a]; u[a] = -u[a]; }
            }
        }
        if (q != 0.0 && g->order == 2) orc_esirkepov2(g, q * s->w[p], x0[0], x0[1], x0[2], x1[0], x1[1], x1[2], J);
        else if (q != 0.0) orc_esirkepov(g, q * s->w[p], x0[0], x0[1], x0[2], x1[0], x1[1], x1[2], J);
        for (int a = 0; a < 3; ++a) {
            if (g->bc[a] == 0) {             /* periodic image in [0, n) */
                double L = (double)n[a];
                if (x1[a] < 0.0) x1[a] += L;
                else if (x1[a] >= L) x1[a] -= L;
                if (x1[a] >= L) x1[a] = 0.0;
            }
        }
        s->x[p] = x1[0]; s->y[p] = x1[1]; s->z[p] = x1[2];
        s->ux[p] = u[0]; s->uy[p] = u[1]; s->uz[p] = u[2];
    }
}

/* Record E^n, B^n at the particles' positions into s->eb (photons: the
 * fields that drive pair creation, gathered before the photon moves). */
void orc_gather_species(const orc_grid *g, const double *E[3], const double *B[3], orc_species *s) {
    for (long p = 0; p < s->n; ++p) {
        double e[3], b[3];
        orc_gather(g, E, B, s->x[p], s->y[p], s->z[p], e, b);
        for (int c = 0; c < 3; ++c) { s->eb[6 * p + c] = e[c]; s->eb[6 * p + 3 + c] = b[c]; }
    }
}
