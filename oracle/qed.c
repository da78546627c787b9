/*
 * Strong-field QED in the locally-constant-field approximation, FP64:
 * photon emission (radiation reaction) by e-/e+ and Breit-Wheeler pair
 * creation by photons, with Monte Carlo events on the optical-depth method.
 *
 * Paper: Methodology -- radiation reaction and QED pair production are
 * modelled with Airy-function approximations using the local field.
 *
 * Rates per unit time [1/w0] (Ritus 1985; Baier & Katkov 1968; Erber 1966),
 * with kappa = hbar w0 / (m c^2) = E_ref / E_s:
 *   chi_e = kappa sqrt((gamma E + u x B)^2 - (u.E)^2)           (u = gamma beta)
 *   chi_g = kappa sqrt((eps E + k x B)^2 - (k.E)^2)             (k photon momentum, eps = |k|, in m c)
 *   emission of a photon carrying the fraction xi of the lepton energy gamma m c^2:
 *     dW/dxi = (alpha / kappa) (1/gamma) F_em(chi, xi),
 *     F_em = -[ Ai_1(z) + ((1 - xi) + 1/(1 - xi)) Ai'(z) / z ],  z = (xi / (chi (1 - xi)))^{2/3}
 *   pair creation with the electron taking the fraction xi of eps m c^2:
 *     dW/dxi = (alpha / kappa) (1/eps) F_pair(chi, xi),
 *     F_pair = Ai_1(z) - (xi/(1 - xi) + (1 - xi)/xi) Ai'(z) / z,  z = (1 / (chi xi (1 - xi)))^{2/3}
 *   with Ai_1(z) = int_z^inf Ai.  Totals h(chi) = int F_em, T(chi) = int F_pair.
 * These are the Airy forms of the synchrotron (Bessel K_{2/3}, int K_{1/3})
 * spectra, obtained with Ai(z) = sqrt(z/3) K_{1/3}(zeta) / pi,
 * Ai'(z) = -z K_{2/3}(zeta) / (pi sqrt 3), zeta = (2/3) z^{3/2}.
 *
 * Emission integrals use mu = ln(xi / (1 - xi)) - ln chi, for which
 * z = exp(2 mu / 3) exactly and the spectrum lives in mu in [-30, 5] for
 * every chi; below mu = -30 the integrand is 2 |Ai'(0)| / z (the small-xi
 * limit) and is integrated in closed form.  Composite 8-point Gauss-Legendre
 * panels of width 1/4.  Pair integrals: over t = ln(xi/(1 - xi)) in
 * [-30, 0] (xi in (0, 1/2], the spectrum is symmetric; for chi >> 1 it
 * extends down to xi ~ 1/chi), panels of width 1/8.
 *
 * Monte Carlo (one event per particle per step at most):
 *   lepton: tau -= W_em dt; when tau <= 0, a Philox draw (counter
 *   (id_lo, id_hi, step, 2), key (seed, species)) gives r0 -> xi by inverting
 *   the cumulative spectrum, r1 -> the new tau = -ln r1, r2 -> the photon's
 *   tau.  The photon gets energy eps = xi gamma (capped at gamma - 1), the
 *   lepton keeps its direction with gamma' = gamma - eps (exact energy balance);
 *   photons with eps >= eps_min become particles, softer ones are tallied.
 *   photon: tau -= W_pair dt (only for eps >= 2); when tau <= 0, a draw with
 *   counter (id_lo, id_hi, step, 3) gives r0 -> xi, r1, r2 -> the taus of the
 *   new electron and positron, which move along k with energies xi eps and
 *   (1 - xi) eps (a part below m c^2 is tallied); the photon is removed.
 *   Derived ids: splitmix64 (Vigna) of the parent id mixed with (step, tag).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>

#define ALPHA_FS 7.2973525693e-3

static const double GL_X[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                               0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
static const double GL_W[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                               0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

double orc_qed_em_density(double chi, double xi) {
    if (!(xi > 0.0 && xi < 1.0) || !(chi > 0.0)) return 0.0;
    const double z = pow(xi / (chi * (1.0 - xi)), 2.0 / 3.0);
    return -(orc_airy_int(z) + ((1.0 - xi) + 1.0 / (1.0 - xi)) * orc_airy_aip(z) / z);
}

double orc_qed_pair_density(double chi, double xi) {
    if (!(xi > 0.0 && xi < 1.0) || !(chi > 0.0)) return 0.0;
    const double z = pow(1.0 / (chi * xi * (1.0 - xi)), 2.0 / 3.0);
    if (z > 700.0) return 0.0;
    return orc_airy_int(z) - (xi / (1.0 - xi) + (1.0 - xi) / xi) * orc_airy_aip(z) / z;
}

/* emission integrand in mu, times xi^p (p = 0: number, p = 1: energy) */
static double em_mu(double chi, double mu, int p) {
    const double e = chi * exp(mu);
    const double xi = e / (1.0 + e), omx = 1.0 / (1.0 + e);
    const double z = exp(2.0 * mu / 3.0);
    const double F = -(orc_airy_int(z) + (omx + 1.0 / omx) * orc_airy_aip(z) / z);
    return F * xi * omx * (p ? xi : 1.0);
}

#define MU_LO (-30.0)
#define MU_HI 5.0
#define MU_PANEL 0.25

/* closed-form integral of the small-xi limit 2|Ai'(0)|/z over xi < xi(mu_lo) */
static double em_tail(double chi, int p) {
    const double xa = chi * exp(MU_LO) / (1.0 + chi * exp(MU_LO));
    const double c = -2.0 * orc_airy_aip(0.0) * pow(chi, 2.0 / 3.0);
    return p ? c * 0.75 * pow(xa, 4.0 / 3.0) : c * 3.0 * pow(xa, 1.0 / 3.0);
}

static double em_panel(double chi, double a, double b, int p) {
    const double hm = 0.5 * (b - a), cm = 0.5 * (b + a);
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += GL_W[k] * em_mu(chi, cm + hm * GL_X[k], p);
    return s * hm;
}

static double em_integral(double chi, int p) {
    double s = em_tail(chi, p);
    for (double a = MU_LO; a < MU_HI - 1e-12; a += MU_PANEL) s += em_panel(chi, a, a + MU_PANEL, p);
    return s;
}

double orc_qed_h(double chi) { return chi > 0.0 ? em_integral(chi, 0) : 0.0; }
double orc_qed_power(double chi) { return chi > 0.0 ? em_integral(chi, 1) : 0.0; }

/* pair integrand in t = ln(xi/(1-xi)): F_pair(xi) dxi/dt */
static double pair_t(double chi, double t) {
    const double xi = 1.0 / (1.0 + exp(-t));
    return orc_qed_pair_density(chi, xi) * xi * (1.0 - xi);
}

static double pair_panel(double chi, double a, double b) {
    const double hm = 0.5 * (b - a), cm = 0.5 * (b + a);
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += GL_W[k] * pair_t(chi, cm + hm * GL_X[k]);
    return s * hm;
}

#define PAIR_T0 (-30.0)
#define PAIR_PANELS 240  /* width 1/8 over [-30, 0] */
double orc_qed_T(double chi) {
    if (!(chi > 0.0)) return 0.0;
    const double w = -PAIR_T0 / PAIR_PANELS;
    double s = 0.0;
    for (int i = 0; i < PAIR_PANELS; ++i) s += pair_panel(chi, PAIR_T0 + i * w, PAIR_T0 + (i + 1) * w);
    return 2.0 * s;
}

/* invert the cumulative emission spectrum: returns xi with CDF(xi) = r */
double orc_qed_em_sample(double chi, double r) {
    const double total = orc_qed_h(chi);
    double target = r * total;
    double acc = em_tail(chi, 0);
    if (target <= acc) {
        /* inside the closed-form tail: CDF ~ xi^{1/3} */
        const double xa = chi * exp(MU_LO) / (1.0 + chi * exp(MU_LO));
        return xa * pow(target / acc, 3.0);
    }
    for (double a = MU_LO; a < MU_HI - 1e-12; a += MU_PANEL) {
        const double pv = em_panel(chi, a, a + MU_PANEL, 0);
        if (acc + pv >= target) {
            double lo = a, hi = a + MU_PANEL;
            for (int it = 0; it < 60; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (acc + em_panel(chi, a, mid, 0) < target) lo = mid; else hi = mid;
            }
            const double e = chi * exp(0.5 * (lo + hi));
            return e / (1.0 + e);
        }
        acc += pv;
    }
    const double e = chi * exp(MU_HI);
    return e / (1.0 + e);
}

/* invert the cumulative pair spectrum over (0, 1) (t from -30 to 30) */
double orc_qed_pair_sample(double chi, double r) {
    const double total = orc_qed_T(chi);
    const double target = r * total;
    const double w = -PAIR_T0 / PAIR_PANELS;
    double acc = 0.0;
    for (int i = 0; i < 2 * PAIR_PANELS; ++i) {
        const double a = PAIR_T0 + i * w, b = a + w;
        const double pv = pair_panel(chi, a, b);
        if (acc + pv >= target || i == 2 * PAIR_PANELS - 1) {
            double lo = a, hi = b;
            for (int it = 0; it < 60; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (acc + pair_panel(chi, a, mid) < target) lo = mid; else hi = mid;
            }
            return 1.0 / (1.0 + exp(-0.5 * (lo + hi)));
        }
        acc += pv;
    }
    return 0.5;
}

double orc_chi(double kappa, const double e[3], const double b[3], const double u[3], int photon) {
    const double g = photon ? sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
                            : sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double f0 = g * e[0] + (u[1] * b[2] - u[2] * b[1]);
    const double f1 = g * e[1] + (u[2] * b[0] - u[0] * b[2]);
    const double f2 = g * e[2] + (u[0] * b[1] - u[1] * b[0]);
    const double ue = u[0] * e[0] + u[1] * e[1] + u[2] * e[2];
    const double s = f0 * f0 + f1 * f1 + f2 * f2 - ue * ue;
    return kappa * sqrt(s > 0.0 ? s : 0.0);
}

uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_derived_id(uint64_t id, long step, unsigned tag) {
    return orc_splitmix64(id ^ orc_splitmix64(((uint64_t)step << 8) | tag));
}

/* initial optical depth of a particle: -ln u, u from counter (id_lo, id_hi, 2^32-1, 4) */
double orc_qed_tau0(uint64_t id, uint32_t seed, uint32_t sp_index) {
    const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), 0xFFFFFFFFu, 4u};
    const uint32_t key[2] = {seed, sp_index};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    return -log(orc_u01(r[0]));
}

/* One emission pass over leptons (after their push; eb = E^n, B^n at x^n).
 * Photons with energy >= eps_min go to `ph` (up to cap); returns their count.
 * tallies[0] += w * eps of photons not kept; tallies[1] += number of events. */
long orc_qed_emit(orc_species *s, double *tau, double kappa, double dt, double eps_min, uint32_t seed,
                  uint32_t sp_index, long step, orc_species *ph, double *ph_tau, long cap, double *tallies) {
    long nph = 0;
    const double pref = ALPHA_FS / kappa;
    for (long p = 0; p < s->n; ++p) {
        double u[3] = {s->ux[p], s->uy[p], s->uz[p]};
        const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double gam = sqrt(1.0 + u2);
        const double chi = orc_chi(kappa, s->eb + 6 * p, s->eb + 6 * p + 3, u, 0);
        if (!(chi > 0.0)) continue;
        tau[p] -= pref * orc_qed_h(chi) / gam * dt;
        if (tau[p] > 0.0) continue;
        const uint64_t id = s->id[p];
        const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step, 2u};
        const uint32_t key[2] = {seed, sp_index};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        const double xi = orc_qed_em_sample(chi, orc_u01(r[0]));
        tau[p] = -log(orc_u01(r[1]));
        double eps = xi * gam;
        if (eps > gam - 1.0) eps = gam - 1.0;
        const double g1 = gam - eps;
        const double un = sqrt(u2), u1 = sqrt(g1 * g1 - 1.0 > 0.0 ? g1 * g1 - 1.0 : 0.0);
        const double scale = un > 0.0 ? u1 / un : 0.0;
        s->ux[p] = u[0] * scale; s->uy[p] = u[1] * scale; s->uz[p] = u[2] * scale;
        tallies[1] += 1.0;
        if (eps >= eps_min && ph && nph < cap && un > 0.0) {
            ph->x[nph] = s->x[p]; ph->y[nph] = s->y[p]; ph->z[nph] = s->z[p];
            ph->ux[nph] = eps * u[0] / un; ph->uy[nph] = eps * u[1] / un; ph->uz[nph] = eps * u[2] / un;
            ph->w[nph] = s->w[p];
            ph->id[nph] = orc_derived_id(id, step, 2u);
            ph_tau[nph] = -log(orc_u01(r[2]));
            ++nph;
        } else {
            tallies[0] += s->w[p] * eps;
        }
    }
    return nph;
}

/* Photon push: ballistic at c (positions in cell units). */
void orc_photon_move(const orc_grid *g, orc_species *s) {
    const double d[3] = {g->dx, g->dy, g->dz};
    const int n[3] = {g->nx, g->ny, g->nz};
    for (long p = 0; p < s->n; ++p) {
        double k[3] = {s->ux[p], s->uy[p], s->uz[p]};
        const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        double x[3] = {s->x[p], s->y[p], s->z[p]};
        for (int a = 0; a < 3; ++a) {
            x[a] += g->dt * (kn > 0.0 ? k[a] / kn : 0.0) / d[a];
            if (g->bc[a] != 0) {
                const double L = (double)(n[a] - 1);
                if (x[a] < 0.0) { x[a] = -x[a]; k[a] = -k[a]; }
                else if (x[a] > L) { x[a] = 2.0 * L - x[a]; k[a] = -k[a]; }
            } else {
                const double L = (double)n[a];
                if (x[a] < 0.0) x[a] += L;
                else if (x[a] >= L) x[a] -= L;
                if (x[a] >= L) x[a] = 0.0;
            }
        }
        s->x[p] = x[0]; s->y[p] = x[1]; s->z[p] = x[2];
        s->ux[p] = k[0]; s->uy[p] = k[1]; s->uz[p] = k[2];
    }
}

/* One pair pass over photons (after their move; eb = E^n, B^n at x^n).
 * alive[p] is cleared for converted photons; new e-/e+ go to el/po.
 * tallies[0] += energy below the rest mass of the pair members that could not
 * be given momentum, tallies[1] += events.  Returns the number of pairs. */
long orc_qed_pairs(orc_species *s, double *tau, unsigned char *alive, double kappa, double dt, uint32_t seed,
                   uint32_t sp_index, long step, orc_species *el, double *el_tau, orc_species *po, double *po_tau,
                   long cap, double *tallies) {
    long np = 0;
    const double pref = ALPHA_FS / kappa;
    for (long p = 0; p < s->n; ++p) {
        alive[p] = 1;
        const double k[3] = {s->ux[p], s->uy[p], s->uz[p]};
        const double eps = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        if (eps < 2.0) continue;
        const double chi = orc_chi(kappa, s->eb + 6 * p, s->eb + 6 * p + 3, k, 1);
        if (!(chi > 0.0)) continue;
        tau[p] -= pref * orc_qed_T(chi) / eps * dt;
        if (tau[p] > 0.0) continue;
        const uint64_t id = s->id[p];
        const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step, 3u};
        const uint32_t key[2] = {seed, sp_index};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        const double xi = orc_qed_pair_sample(chi, orc_u01(r[0]));
        alive[p] = 0;
        tallies[1] += 1.0;
        if (np >= cap) continue;
        const double ee = xi * eps, ep = (1.0 - xi) * eps;
        const double ue = ee > 1.0 ? sqrt(ee * ee - 1.0) : 0.0, up = ep > 1.0 ? sqrt(ep * ep - 1.0) : 0.0;
        if (ee < 1.0) tallies[0] += s->w[p] * (1.0 - ee);
        if (ep < 1.0) tallies[0] += s->w[p] * (1.0 - ep);
        el->x[np] = s->x[p]; el->y[np] = s->y[p]; el->z[np] = s->z[p];
        po->x[np] = s->x[p]; po->y[np] = s->y[p]; po->z[np] = s->z[p];
        el->ux[np] = ue * k[0] / eps; el->uy[np] = ue * k[1] / eps; el->uz[np] = ue * k[2] / eps;
        po->ux[np] = up * k[0] / eps; po->uy[np] = up * k[1] / eps; po->uz[np] = up * k[2] / eps;
        el->w[np] = po->w[np] = s->w[p];
        el->id[np] = orc_derived_id(id, step, 3u);
        po->id[np] = orc_derived_id(id, step, 5u);
        el_tau[np] = -log(orc_u01(r[1]));
        po_tau[np] = -log(orc_u01(r[2]));
        ++np;
    }
    return np;
}
