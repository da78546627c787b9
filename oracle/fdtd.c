/*
 * Yee FDTD field solver and first-order Mur absorbing boundary, FP64.
 *
 * Paper: Methodology -- the field update is an explicit FDTD solution of
 * Maxwell's equations on a uniform Cartesian grid with a fixed time step set
 * by the Courant limit, and open boundaries are first-order Mur absorbers
 * that keep past boundary values and use the coefficient (c dt - d)/(c dt + d).
 *
 * Staggering (Yee 1966): E_x at (i+1/2, j, k), E_y at (i, j+1/2, k),
 * E_z at (i, j, k+1/2); B_x at (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2),
 * B_z at (i+1/2, j+1/2, k); J with E; rho at nodes.  Array index i holds the
 * value at i (integer position) or at i+1/2 (half-integer position).
 *
 * The magnetic update is split into two half steps so that E^n and B^n are
 * co-temporal when particles gather them:
 *   B^{n+1/2} = B^n - dt/2 curl E^n,
 *   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2}),
 *   B^{n+1}   = B^{n+1/2} - dt/2 curl E^{n+1}.
 *
 * Non-periodic axis a with n_a nodes spans node positions 0..n_a-1; a value
 * at a half-integer position along a exists only for index <= n_a-2 and is
 * held at zero otherwise.  A tangential E value on a boundary plane (index 0
 * or n_a-1 along a non-periodic axis other than its own direction) is not
 * reachable by the Yee stencil and is set by Mur:
 *   E_0^{n+1} = E_1^n + ((dt - d_a)/(dt + d_a)) (E_1^{n+1} - E_0^n),
 * with E_1 the neighbour one node inwards along a.  A value on the boundary
 * of several axes (an edge) takes the lowest-index such axis; values on one
 * boundary are set before values on two, so every neighbour used is final.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <stdlib.h>
#include <string.h>

static inline long IDX(const orc_grid *g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)k);
}
static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* does a component with half-integer offset along axis a exist at index i? */
static inline int half_ok(const orc_grid *g, int a, int i) {
    int n = a == 0 ? g->nx : (a == 1 ? g->ny : g->nz);
    return g->bc[a] == 0 || i <= n - 2;
}

void orc_fdtd_b_half(const orc_grid *g, const double *E[3], double *B[3]) {
    const double h = 0.5 * g->dt;
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const int ip = wrapi(i + 1, nx), jp = wrapi(j + 1, ny), kp = wrapi(k + 1, nz);
        const long c = IDX(g, i, j, k);
        /* B_x at (i, j+1/2, k+1/2): curl_x E = dEz/dy - dEy/dz */
        if (half_ok(g, 1, j) && half_ok(g, 2, k)) {
            double cx = (E[2][IDX(g, i, jp, k)] - E[2][c]) / g->dy
                      - (E[1][IDX(g, i, j, kp)] - E[1][c]) / g->dz;
            B[0][c] -= h * cx;
        }
        /* B_y at (i+1/2, j, k+1/2): curl_y E = dEx/dz - dEz/dx */
        if (half_ok(g, 0, i) && half_ok(g, 2, k)) {
            double cy = (E[0][IDX(g, i, j, kp)] - E[0][c]) / g->dz
                      - (E[2][IDX(g, ip, j, k)] - E[2][c]) / g->dx;
            B[1][c] -= h * cy;
        }
        /* B_z at (i+1/2, j+1/2, k): curl_z E = dEy/dx - dEx/dy */
        if (half_ok(g, 0, i) && half_ok(g, 1, j)) {
            double cz = (E[1][IDX(g, ip, j, k)] - E[1][c]) / g->dx
                      - (E[0][IDX(g, i, jp, k)] - E[0][c]) / g->dy;
            B[2][c] -= h * cz;
        }
    }
}

/* boundary axes of E component `comp` at node (i,j,k): bit a set when the
 * node lies on a boundary plane of non-periodic axis a != comp */
static int e_boundary_mask(const orc_grid *g, int comp, int i, int j, int k) {
    int n[3] = {g->nx, g->ny, g->nz}, idx[3] = {i, j, k}, m = 0;
    for (int a = 0; a < 3; ++a) {
        if (a == comp || g->bc[a] == 0) continue;
        if (idx[a] == 0 || idx[a] == n[a] - 1) m |= 1 << a;
    }
    return m;
}

static int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }

void orc_fdtd_e(const orc_grid *g, double *E[3], const double *B[3], const double *J[3]) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const long N = (long)nx * ny * nz;
    const double dt = g->dt;
    double *old[3];
    for (int c = 0; c < 3; ++c) {
        old[c] = (double *)malloc(sizeof(double) * N);
        memcpy(old[c], E[c], sizeof(double) * N);
    }
    /* Yee update of every existing E value that is not on a boundary plane */
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const int im = wrapi(i - 1, nx), jm = wrapi(j - 1, ny), km = wrapi(k - 1, nz);
        const long c = IDX(g, i, j, k);
        if (half_ok(g, 0, i) && e_boundary_mask(g, 0, i, j, k) == 0) {
            double cx = (B[2][c] - B[2][IDX(g, i, jm, k)]) / g->dy
                      - (B[1][c] - B[1][IDX(g, i, j, km)]) / g->dz;
            E[0][c] += dt * (cx - J[0][c]);
        }
        if (half_ok(g, 1, j) && e_boundary_mask(g, 1, i, j, k) == 0) {
            double cy = (B[0][c] - B[0][IDX(g, i, j, km)]) / g->dz
                      - (B[2][c] - B[2][IDX(g, im, j, k)]) / g->dx;
            E[1][c] += dt * (cy - J[1][c]);
        }
        if (half_ok(g, 2, k) && e_boundary_mask(g, 2, i, j, k) == 0) {
            double cz = (B[1][c] - B[1][IDX(g, im, j, k)]) / g->dx
                      - (B[0][c] - B[0][IDX(g, i, jm, k)]) / g->dy;
            E[2][c] += dt * (cz - J[2][c]);
        }
    }
    /* Mur: faces first (one boundary axis), then edges (two) */
    const double d[3] = {g->dx, g->dy, g->dz};
    const int n[3] = {nx, ny, nz};
    for (int phase = 1; phase <= 2; ++phase)
    for (int comp = 0; comp < 3; ++comp)
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        int idx[3] = {i, j, k};
        if (!half_ok(g, comp, idx[comp])) continue;
        int m = e_boundary_mask(g, comp, i, j, k);
        if (popc3(m) != phase) continue;
        int a = (m & 1) ? 0 : ((m & 2) ? 1 : 2);
        int nb[3] = {i, j, k};
        nb[a] = idx[a] == 0 ? 1 : n[a] - 2;
        const long c0 = IDX(g, i, j, k), c1 = IDX(g, nb[0], nb[1], nb[2]);
        const double coef = (dt - d[a]) / (dt + d[a]);
        E[comp][c0] = old[comp][c1] + coef * (E[comp][c1] - old[comp][c0]);
    }
    for (int c = 0; c < 3; ++c) free(old[c]);
}
