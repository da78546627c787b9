/*
 * Diagnostics, FP64: energies, charge density and the discrete divergence.
 *
 * Paper: Methodology -- total energy is the sum of electromagnetic, kinetic
 * and thermal parts; charge and energy conservation are checked during steps
 * and at regime switches.  In laser-normalised units the field energy is
 * (1/2) sum (E^2 + B^2) dV and a particle of weight w, mass m carries
 * w m (gamma - 1); both in units m_e c^2 n_c (c/w0)^3.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>
#include <string.h>

static inline long IDX(const orc_grid *g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)k);
}
static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

void orc_energy_fields(const orc_grid *g, const double *E[3], const double *B[3], double out[2]) {
    const long N = (long)g->nx * g->ny * g->nz;
    const double dV = g->dx * g->dy * g->dz;
    double we = 0.0, wb = 0.0;
    for (long c = 0; c < N; ++c) {
        we += E[0][c] * E[0][c] + E[1][c] * E[1][c] + E[2][c] * E[2][c];
        wb += B[0][c] * B[0][c] + B[1][c] * B[1][c] + B[2][c] * B[2][c];
    }
    out[0] = 0.5 * we * dV;
    out[1] = 0.5 * wb * dV;
}

double orc_energy_particles(const orc_species *s) {
    double acc = 0.0;
    for (long p = 0; p < s->n; ++p) {
        double u2 = s->ux[p] * s->ux[p] + s->uy[p] * s->uy[p] + s->uz[p] * s->uz[p];
        /* gamma - 1 written as u^2 / (gamma + 1) to keep digits for slow particles */
        acc += s->w[p] * s->m * u2 / (sqrt(1.0 + u2) + 1.0);
    }
    return acc;
}

void orc_charge_density(const orc_grid *g, const orc_species *s, double *rho) {
    const double dV = g->dx * g->dy * g->dz;
    const int n[3] = {g->nx, g->ny, g->nz};
    if (g->order == 2) {   /* quadratic shape on the nearest node and its two neighbours */
        for (long p = 0; p < s->n; ++p) {
            const double q = s->zq ? s->q * s->zq[p] : s->q;
            const double pos[3] = {s->x[p], s->y[p], s->z[p]};
            int m[3];
            for (int a = 0; a < 3; ++a) m[a] = (int)floor(pos[a] + 0.5);
            for (int c = -1; c <= 1; ++c)
            for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a) {
                int idx[3] = {m[0] + a, m[1] + b, m[2] + c};
                int skip = 0;
                for (int ax = 0; ax < 3; ++ax) {
                    if (g->bc[ax] == 0) idx[ax] = wrapi(idx[ax], n[ax]);
                    else if (idx[ax] < 0 || idx[ax] >= n[ax]) skip = 1;
                }
                if (skip) continue;
                const double wgt = orc_tsc(pos[0] - (m[0] + a)) * orc_tsc(pos[1] - (m[1] + b)) *
                                   orc_tsc(pos[2] - (m[2] + c));
                rho[IDX(g, idx[0], idx[1], idx[2])] += q * s->w[p] * wgt / dV;
            }
        }
        return;
    }
    for (long p = 0; p < s->n; ++p) {
        const double q = s->zq ? s->q * s->zq[p] : s->q;
        const double pos[3] = {s->x[p], s->y[p], s->z[p]};
        int base[3]; double f[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floor(pos[a]);
            if (g->bc[a] != 0 && i > n[a] - 2) i = n[a] - 2;
            base[a] = i; f[a] = pos[a] - i;
        }
        for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            int ii = base[0] + a, jj = base[1] + b, kk = base[2] + c;
            if (g->bc[0] == 0) ii = wrapi(ii, n[0]); else if (ii < 0 || ii >= n[0]) continue;
            if (g->bc[1] == 0) jj = wrapi(jj, n[1]); else if (jj < 0 || jj >= n[1]) continue;
            if (g->bc[2] == 0) kk = wrapi(kk, n[2]); else if (kk < 0 || kk >= n[2]) continue;
            double wgt = (a ? f[0] : 1 - f[0]) * (b ? f[1] : 1 - f[1]) * (c ? f[2] : 1 - f[2]);
            rho[IDX(g, ii, jj, kk)] += q * s->w[p] * wgt / dV;
        }
    }
}

void orc_div_e(const orc_grid *g, const double *E[3], double *div) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
        int im = i - 1, jm = j - 1, km = k - 1;
        double exm = 0, eym = 0, ezm = 0;
        if (g->bc[0] == 0) exm = E[0][IDX(g, wrapi(im, nx), j, k)]; else if (im >= 0) exm = E[0][IDX(g, im, j, k)];
        if (g->bc[1] == 0) eym = E[1][IDX(g, i, wrapi(jm, ny), k)]; else if (jm >= 0) eym = E[1][IDX(g, i, jm, k)];
        if (g->bc[2] == 0) ezm = E[2][IDX(g, i, j, wrapi(km, nz))]; else if (km >= 0) ezm = E[2][IDX(g, i, j, km)];
        const long c = IDX(g, i, j, k);
        div[c] = (E[0][c] - exm) / g->dx + (E[1][c] - eym) / g->dy + (E[2][c] - ezm) / g->dz;
    }
}

/* SI constants (CODATA 2018) used only for unit conversion */
#define ORC_C    299792458.0
#define ORC_QE   1.602176634e-19
#define ORC_ME   9.1093837015e-31
#define ORC_EPS0 8.8541878128e-12

/* Plasma-frequency scales for an electron density n [m^-3] (paper, Results:
 * E_0 = m_e c w_p / e, B_0 = E_0 / c, J_0 = e n c, rho_0 = e n).
 * out = {w_p [1/s], E_0 [V/m], B_0 [T], J_0 [A/m^2], rho_0 [C/m^3]} */
void orc_plasma_scales(double n, double out[5]) {
    double wp = sqrt(n * ORC_QE * ORC_QE / (ORC_EPS0 * ORC_ME));
    out[0] = wp;
    out[1] = ORC_ME * ORC_C * wp / ORC_QE;
    out[2] = out[1] / ORC_C;
    out[3] = ORC_QE * n * ORC_C;
    out[4] = ORC_QE * n;
}

/* Laser-normalised reference scales for a wavelength lambda [m]:
 * out = {w0 [1/s], n_c [m^-3], E_ref = m_e c w0 / e [V/m], length c/w0 [m]} */
void orc_laser_scales(double lambda, double out[4]) {
    double w0 = 2.0 * 3.14159265358979323846 * ORC_C / lambda;
    out[0] = w0;
    out[1] = ORC_EPS0 * ORC_ME * w0 * w0 / (ORC_QE * ORC_QE);
    out[2] = ORC_ME * ORC_C * w0 / ORC_QE;
    out[3] = ORC_C / w0;
}
