/*
 * Cold relativistic fluid, FP64.
 *
 * Paper: Methodology -- bulk plasma in stable regions is a fluid (continuity
 * and momentum equations with relativistic gamma factors); clamping is used
 * against numerical instability.  The build keeps the cold (pressureless)
 * part:
 *   dn/dt + div(n v) = 0,   d(n u)/dt + div(n u v) = (q/m) n (E + v x B),
 *   u = gamma v, gamma = sqrt(1 + u^2).
 * Warm variant (the paper's fluid model carries an adiabatic pressure): with
 * p = K n^Gamma (K = 0: cold) the momentum equation gains -grad p / m, applied
 * with the Lorentz force before the transport, so that the new velocity moves
 * the density (a leapfrog, stable for sound waves with dt c_s < 2 d):
 *   u* <- u* - dt (P(i+1/2) - P(i-1/2)) / (d m n_i) along each axis,
 * P(i+1/2) = (p_i + p_{i+1}) / 2 on inner faces and the node's own p on the
 * outer face of an absorbing axis (a wall reflects the pressure), evaluated
 * with n^n at nodes with n > n_floor (elsewhere u* keeps its value).
 * The paper gives no discretisation.  Reading used here: first-order upwind
 * (donor cell) in conservative form on the control volumes around the nodes,
 * with the Lorentz force applied first as a Boris rotation of u at each node
 * (E and B averaged from the Yee positions to the node):
 *   1. u* = Boris(u^{n-1/2}; E^n, B^n at the node), v* = u* / gamma*
 *   2. at the face between nodes i and i+1 along axis a:
 *      s = (v*_a(i) + v*_a(i+1)) / 2,
 *      F = max(s,0) n_i + min(s,0) n_{i+1},
 *      G = max(s,0) (n u*)_i + min(s,0) (n u*)_{i+1}
 *      (no flux through the outer faces of an absorbing axis)
 *   3. n^{n+1} = n^n - dt sum_a (F(i+1/2) - F(i-1/2)) / d_a,
 *      (n u)^{n+1} = n^n u* - dt sum_a (G(i+1/2) - G(i-1/2)) / d_a
 *   4. J_a(i+1/2) += q F(i+1/2): the face of the node control volume is the
 *      Yee edge of E_a, so rho = q n obeys the discrete continuity equation
 *      with the deposited J exactly
 *   5. clamp: n < 0 -> 0 (counted); u^{n+1/2} = (n u)^{n+1} / n^{n+1} where
 *      n^{n+1} > n_floor, else 0.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static inline long IDX(const orc_grid *g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)k);
}
static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* value of a staggered field at index (i,j,k), zero outside an absorbing axis */
static double fval(const orc_grid *g, const double *F, int i, int j, int k) {
    const int n[3] = {g->nx, g->ny, g->nz};
    int idx[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (g->bc[a] == 0) idx[a] = wrapi(idx[a], n[a]);
        else if (idx[a] < 0 || idx[a] > n[a] - 1) return 0.0;
    }
    return F[IDX(g, idx[0], idx[1], idx[2])];
}

/* E and B averaged to node (i,j,k) from their Yee positions */
void orc_node_fields(const orc_grid *g, const double *E[3], const double *B[3], int i, int j, int k,
                     double e[3], double b[3]) {
    e[0] = 0.5 * (fval(g, E[0], i - 1, j, k) + fval(g, E[0], i, j, k));
    e[1] = 0.5 * (fval(g, E[1], i, j - 1, k) + fval(g, E[1], i, j, k));
    e[2] = 0.5 * (fval(g, E[2], i, j, k - 1) + fval(g, E[2], i, j, k));
    b[0] = 0.25 * (fval(g, B[0], i, j - 1, k - 1) + fval(g, B[0], i, j, k - 1) + fval(g, B[0], i, j - 1, k) +
                   fval(g, B[0], i, j, k));
    b[1] = 0.25 * (fval(g, B[1], i - 1, j, k - 1) + fval(g, B[1], i, j, k - 1) + fval(g, B[1], i - 1, j, k) +
                   fval(g, B[1], i, j, k));
    b[2] = 0.25 * (fval(g, B[2], i - 1, j - 1, k) + fval(g, B[2], i, j - 1, k) + fval(g, B[2], i - 1, j, k) +
                   fval(g, B[2], i, j, k));
}

static double pressure(double K, double gam, double n) { return K > 0.0 && n > 0.0 ? K * pow(n, gam) : 0.0; }

long orc_fluid_step(const orc_grid *g, const double *E[3], const double *B[3], double *J[3], double q, double m,
                    double *n, double *u[3], double n_floor, double K, double gam) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const long N = (long)nx * ny * nz;
    const int nn[3] = {nx, ny, nz};
    const double d[3] = {g->dx, g->dy, g->dz};
    double *us[3], *vs[3];
    for (int c = 0; c < 3; ++c) {
        us[c] = (double *)malloc(sizeof(double) * N);
        vs[c] = (double *)malloc(sizeof(double) * N);
    }
    /* 1. Lorentz force at the nodes */
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const long c = IDX(g, i, j, k);
        double e[3], b[3], uu[3] = {u[0][c], u[1][c], u[2][c]};
        orc_node_fields(g, E, B, i, j, k, e, b);
        orc_boris(q * g->dt / (2.0 * m), e, b, uu);
        if (K > 0.0 && n[c] > n_floor) {
            const int idx[3] = {i, j, k};
            const double pc = pressure(K, gam, n[c]);
            for (int a = 0; a < 3; ++a) {
                int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                double plo = pc, phi = pc;       /* outer faces of an absorbing axis: the node's own p */
                if (g->bc[a] == 0 || idx[a] > 0) { lo[a] = wrapi(idx[a] - 1, nn[a]); plo = 0.5 * (pc + pressure(K, gam, n[IDX(g, lo[0], lo[1], lo[2])])); }
                if (g->bc[a] == 0 || idx[a] < nn[a] - 1) { hi[a] = wrapi(idx[a] + 1, nn[a]); phi = 0.5 * (pc + pressure(K, gam, n[IDX(g, hi[0], hi[1], hi[2])])); }
                uu[a] -= g->dt * (phi - plo) / (d[a] * m * n[c]);
            }
        }
        const double gmn = sqrt(1.0 + uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
        for (int a = 0; a < 3; ++a) { us[a][c] = uu[a]; vs[a][c] = uu[a] / gmn; }
    }
    /* 2.-4. face fluxes (face i+1/2 of each node along each axis) */
    double *dn = (double *)calloc(N, sizeof(double));
    double *dm[3];
    for (int a = 0; a < 3; ++a) dm[a] = (double *)calloc(N, sizeof(double));
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const int idx[3] = {i, j, k};
        const long c = IDX(g, i, j, k);
        for (int a = 0; a < 3; ++a) {
            int nb[3] = {i, j, k};
            if (g->bc[a] != 0 && idx[a] == nn[a] - 1) continue;  /* closed outer face */
            nb[a] = wrapi(idx[a] + 1, nn[a]);
            const long c1 = IDX(g, nb[0], nb[1], nb[2]);
            const double s = 0.5 * (vs[a][c] + vs[a][c1]);
            const double sp = s > 0.0 ? s : 0.0, sm = s < 0.0 ? s : 0.0;
            const double F = sp * n[c] + sm * n[c1];
            dn[c] -= F / d[a];
            dn[c1] += F / d[a];
            for (int b2 = 0; b2 < 3; ++b2) {
                const double G = sp * n[c] * us[b2][c] + sm * n[c1] * us[b2][c1];
                dm[b2][c] -= G / d[a];
                dm[b2][c1] += G / d[a];
            }
            J[a][c] += q * F;
        }
    }
    /* 5. update and clamp */
    long clamped = 0;
    for (long c = 0; c < N; ++c) {
        const double n1 = n[c] + g->dt * dn[c];
        double mom[3];
        for (int a = 0; a < 3; ++a) mom[a] = n[c] * us[a][c] + g->dt * dm[a][c];
        if (n1 < 0.0) ++clamped;
        n[c] = n1 > 0.0 ? n1 : 0.0;
        for (int a = 0; a < 3; ++a) u[a][c] = n1 > n_floor ? mom[a] / n1 : 0.0;
    }
    for (int a = 0; a < 3; ++a) { free(us[a]); free(vs[a]); free(dm[a]); }
    free(dn);
    return clamped;
}

/* kinetic energy of a fluid species: sum n m (gamma - 1) dV */
double orc_fluid_energy(const orc_grid *g, double m, const double *n, const double *u[3]) {
    const long N = (long)g->nx * g->ny * g->nz;
    const double dV = g->dx * g->dy * g->dz;
    double acc = 0.0;
    for (long c = 0; c < N; ++c) {
        const double u2 = u[0][c] * u[0][c] + u[1][c] * u[1][c] + u[2][c] * u[2][c];
        acc += n[c] * m * u2 / (sqrt(1.0 + u2) + 1.0);
    }
    return acc * dV;
}
