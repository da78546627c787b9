/*
 * Regime criterion and fluid <-> particle conversion, FP64.
 *
 * Paper: Methodology -- fluid models describe the stable regions and PIC the
 * unstable ones, with learned switching between them; charge and energy are
 * checked during regime switches; unstable steps showed high charge density
 * values.  The paper does not define the instability criterion nor the
 * conversion.  Readings used here (parity unpinned beyond the conservation
 * invariants below):
 *
 * Criterion (label of a node): kinetic if any of
 *   |E| >= a_thr (relativistic field; E at the node, laser-normalised),
 *   n_e >= n_thr (density spike / near-critical plasma; electron density of
 *     the fluid plus the CIC density of the electron macro-particles),
 *   dt div v <= -c_thr (imminent trajectory crossing of the electron fluid;
 *     central differences of the fluid velocity at the nodes),
 *   chi = kappa gamma |E| >= chi_thr (quantum parameter estimate with the
 *     fluid gamma),
 * then dilated by `dilate` nodes (Chebyshev distance).
 *
 * Conversion with a new mask (1 = kinetic):
 *   fluid -> particles at kinetic nodes with n > n_floor: ppc macro-particles
 *     at Philox-uniform positions in the node's dual cell [i-1/2, i+1/2)^3
 *     (clipped to the domain), each with the fluid's u and weight n dV / ppc;
 *     key (seed, target species), counter (node, epoch, k, 6), ids
 *     splitmix64-derived from (node, epoch, k); the fluid at the node is
 *     removed.  The residual background charge rho_bg takes the difference
 *     between the removed fluid charge q n and the CIC charge of the new
 *     particles, so div E - rho - rho_bg is unchanged.
 *   particles -> fluid for particles whose nearest node is fluid: n and n u
 *     are deposited with the CIC weights on the 8 surrounding nodes (the node
 *     charge is then exactly what the particle contributed) and the particle
 *     is removed; the fluid u at each node is (n u) / n.
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

void orc_regime_criterion(const orc_grid *g, const double *E[3], const double *B[3], const double *ne,
                          const double *fu[3], double kappa, double a_thr, double n_thr, double c_thr,
                          double chi_thr, int dilate, unsigned char *mask) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const long N = (long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
    const double d[3] = {g->dx, g->dy, g->dz};
    unsigned char *raw = (unsigned char *)calloc(N, 1);
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        const long c = IDX(g, i, j, k);
        double e[3], b[3];
        orc_node_fields(g, E, B, i, j, k, e, b);
        const double emag = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        int kin = emag >= a_thr || ne[c] >= n_thr;
        double u2 = 0.0;
        if (fu) {
            u2 = fu[0][c] * fu[0][c] + fu[1][c] * fu[1][c] + fu[2][c] * fu[2][c];
            /* velocity divergence by central differences (one-sided at absorbing walls) */
            double div = 0.0;
            const int idx[3] = {i, j, k};
            for (int a = 0; a < 3; ++a) {
                int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                double span = 2.0 * d[a];
                if (g->bc[a] == 0) {
                    lo[a] = wrapi(idx[a] - 1, n[a]);
                    hi[a] = wrapi(idx[a] + 1, n[a]);
                } else {
                    lo[a] = idx[a] > 0 ? idx[a] - 1 : idx[a];
                    hi[a] = idx[a] < n[a] - 1 ? idx[a] + 1 : idx[a];
                    span = (hi[a] - lo[a]) * d[a];
                }
                const long cl = IDX(g, lo[0], lo[1], lo[2]), ch = IDX(g, hi[0], hi[1], hi[2]);
                const double vl = fu[a][cl] / sqrt(1.0 + fu[0][cl] * fu[0][cl] + fu[1][cl] * fu[1][cl] +
                                                   fu[2][cl] * fu[2][cl]);
                const double vh = fu[a][ch] / sqrt(1.0 + fu[0][ch] * fu[0][ch] + fu[1][ch] * fu[1][ch] +
                                                   fu[2][ch] * fu[2][ch]);
                if (span > 0.0) div += (vh - vl) / span;
            }
            kin = kin || g->dt * div <= -c_thr;
        }
        kin = kin || kappa * sqrt(1.0 + u2) * emag >= chi_thr;
        raw[c] = (unsigned char)kin;
    }
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        int any = 0;
        for (int dk = -dilate; dk <= dilate && !any; ++dk)
        for (int dj = -dilate; dj <= dilate && !any; ++dj)
        for (int di = -dilate; di <= dilate && !any; ++di) {
            int q[3] = {i + di, j + dj, k + dk}, ok = 1;
            for (int a = 0; a < 3; ++a) {
                if (g->bc[a] == 0) q[a] = wrapi(q[a], n[a]);
                else if (q[a] < 0 || q[a] > n[a] - 1) ok = 0;
            }
            if (ok && raw[IDX(g, q[0], q[1], q[2])]) any = 1;
        }
        mask[IDX(g, i, j, k)] = (unsigned char)any;
    }
    free(raw);
}

/* CIC charge of one particle added to a node array (times `scale`) */
static void cic_add(const orc_grid *g, double x, double y, double z, double val, double *arr) {
    const int n[3] = {g->nx, g->ny, g->nz};
    const double p[3] = {x, y, z};
    int base[3]; double f[3];
    for (int a = 0; a < 3; ++a) {
        int i = (int)floor(p[a]);
        if (g->bc[a] != 0 && i > n[a] - 2) i = n[a] - 2;
        base[a] = i; f[a] = p[a] - i;
    }
    for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
        int q[3] = {base[0] + a, base[1] + b, base[2] + c}, ok = 1;
        for (int ax = 0; ax < 3; ++ax) {
            if (g->bc[ax] == 0) q[ax] = wrapi(q[ax], n[ax]);
            else if (q[ax] < 0 || q[ax] > n[ax] - 1) ok = 0;
        }
        if (!ok) continue;
        const double wgt = (a ? f[0] : 1 - f[0]) * (b ? f[1] : 1 - f[1]) * (c ? f[2] : 1 - f[2]);
        arr[IDX(g, q[0], q[1], q[2])] += wgt * val;
    }
}

/* fluid -> particles; returns the number of particles written to out (cap) */
/* quiet start: the ppc particles of a node sit on an lx x ly x lz lattice of the
 * node's dual cell (lx >= ly >= lz, as close to cubic as ppc allows), at the
 * centres of its sub-cells; lz is the largest divisor of ppc not above its
 * cube root, ly the largest divisor of ppc / lz not above its square root */
static void lattice_dims(int ppc, int l[3]) {
    int lz = 1, ly = 1;
    for (int d = 1; d * d * d <= ppc; ++d)
        if (ppc % d == 0) lz = d;
    const int r = ppc / lz;
    for (int d = 1; d * d <= r; ++d)
        if (r % d == 0) ly = d;
    l[0] = r / ly;
    l[1] = ly;
    l[2] = lz;
}

long orc_fluid_to_particles(const orc_grid *g, const unsigned char *mask, double q, double *n, double *u[3],
                            double n_floor, int ppc, uint32_t seed, uint32_t sp_index, uint32_t epoch,
                            orc_species *out, long cap, double *rho_bg, int quiet) {
    int lat[3];
    lattice_dims(ppc, lat);
    const int nn[3] = {g->nx, g->ny, g->nz};
    const double dV = g->dx * g->dy * g->dz;
    long m = 0;
    for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
        const long c = IDX(g, i, j, k);
        if (!mask[c] || !(n[c] > n_floor)) continue;
        const double w = n[c] * dV / ppc;
        rho_bg[c] += q * n[c];  /* the removed fluid charge density */
        const int idx[3] = {i, j, k};
        for (int p = 0; p < ppc; ++p) {
            const uint32_t ctr[4] = {(uint32_t)c, epoch, (uint32_t)p, 6u};
            const uint32_t key[2] = {seed, sp_index};
            uint32_t r[4];
            orc_philox4x32_10(ctr, key, r);
            double pos[3];
            const int lm[3] = {p % lat[0], (p / lat[0]) % lat[1], p / (lat[0] * lat[1])};
            for (int a = 0; a < 3; ++a) {
                double lo = idx[a] - 0.5, hi = idx[a] + 0.5;
                if (g->bc[a] != 0) { if (lo < 0.0) lo = 0.0; if (hi > nn[a] - 1) hi = nn[a] - 1; }
                const double frac = quiet ? (lm[a] + 0.5) / lat[a] : orc_u01(r[a]);
                pos[a] = lo + (hi - lo) * frac;
                if (g->bc[a] == 0) { if (pos[a] < 0.0) pos[a] += nn[a]; if (pos[a] >= nn[a]) pos[a] -= nn[a]; }
            }
            cic_add(g, pos[0], pos[1], pos[2], -q * w / dV, rho_bg);
            if (m < cap) {
                out->x[m] = pos[0]; out->y[m] = pos[1]; out->z[m] = pos[2];
                out->ux[m] = u[0][c]; out->uy[m] = u[1][c]; out->uz[m] = u[2][c];
                out->w[m] = w;
                out->id[m] = (1ULL << 62) | orc_derived_id((uint64_t)c | ((uint64_t)epoch << 40), p, 6u) >> 2;
            }
            ++m;
        }
        n[c] = 0.0;
        u[0][c] = u[1][c] = u[2][c] = 0.0;
    }
    return m;
}

/* particles -> fluid; alive[p] cleared for converted particles; returns the count */
long orc_particles_to_fluid(const orc_grid *g, const unsigned char *mask, orc_species *s, double *n,
                            double *u[3], double n_floor, unsigned char *alive) {
    const int nn[3] = {g->nx, g->ny, g->nz};
    const long N = (long)g->nx * g->ny * g->nz;
    const double dV = g->dx * g->dy * g->dz;
    double *mom[3];
    for (int a = 0; a < 3; ++a) {
        mom[a] = (double *)malloc(sizeof(double) * N);
        for (long c = 0; c < N; ++c) mom[a][c] = n[c] * u[a][c];
    }
    long conv = 0;
    for (long p = 0; p < s->n; ++p) {
        alive[p] = 1;
        const double pos[3] = {s->x[p], s->y[p], s->z[p]};
        int nd[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floor(pos[a] + 0.5);
            if (g->bc[a] == 0) i = wrapi(i, nn[a]);
            else if (i > nn[a] - 1) i = nn[a] - 1;
            nd[a] = i;
        }
        if (mask[IDX(g, nd[0], nd[1], nd[2])]) continue;
        const double wn = s->w[p] / dV;
        cic_add(g, pos[0], pos[1], pos[2], wn, n);
        cic_add(g, pos[0], pos[1], pos[2], wn * s->ux[p], mom[0]);
        cic_add(g, pos[0], pos[1], pos[2], wn * s->uy[p], mom[1]);
        cic_add(g, pos[0], pos[1], pos[2], wn * s->uz[p], mom[2]);
        alive[p] = 0;
        ++conv;
    }
    for (long c = 0; c < N; ++c)
        for (int a = 0; a < 3; ++a) u[a][c] = n[c] > n_floor ? mom[a][c] / n[c] : 0.0;
    for (int a = 0; a < 3; ++a) free(mom[a]);
    return conv;
}
