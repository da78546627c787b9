/*
 * Field ionization, FP64: ADK tunnelling and multiphoton rates blended by a
 * sigmoid in the Keldysh parameter, and the per-step Monte Carlo event.
 *
 * Paper: Methodology -- ionization blends Ammosov-Delone-Krainov tunnelling
 * and multiphoton rates with a sigmoid transition at Keldysh parameter ~1.5.
 *
 * ADK (Ammosov, Delone, Krainov, Sov. Phys. JETP 64, 1191 (1986)), static
 * field, atomic units, for removing an electron with orbital quantum numbers
 * (l, m) from an ion whose charge after ionization is Z:
 *   n* = Z / sqrt(2 Ip),  l* = n* - 1,
 *   C^2 = 2^{2n*} / (n* Gamma(n*+l*+1) Gamma(n*-l*)),
 *   f(l,m) = (2l+1) (l+|m|)! / (2^|m| |m|! (l-|m|)!),
 *   w = C^2 f Ip (2 (2Ip)^{3/2} / F)^{2n*-|m|-1} exp(-2 (2Ip)^{3/2} / (3F)).
 * Keldysh (Sov. Phys. JETP 20, 1307 (1965)): gamma = w0 sqrt(2 Ip) / F.
 * Multiphoton: w_MPI = sigma_K I^K with K = ceil(Ip / w0) photons and I ~ F^2.
 * The paper gives no sigma_K; it is fixed by continuity with ADK at the
 * blend centre F* (gamma(F*) = 1.5): w_MPI(F) = w_ADK(F*) (F/F*)^{2K}.
 * Blend: S(gamma) = 1 / (1 + exp(-(gamma - 1.5)/Delta)), Delta = 0.1 (the
 * paper gives no width).  The paper does not say what is blended; a linear
 * mix of the two rates lets the F^{2K} multiphoton law dominate deep in the
 * tunnelling regime (for neutral carbon at F = 0.3 a.u. the term S w_MPI is
 * ~4e5 a.u. against w_ADK ~ 6), so the blend is taken on the logarithm:
 *   ln w = S ln w_MPI + (1 - S) ln w_ADK.
 * m = 0 throughout.
 *
 * Monte Carlo: an ion in charge state Z with Z < Zmax ionizes at most once
 * per step, with probability P = 1 - exp(-w dt), when the Philox uniform
 * drawn from key (seed, species), counter (id_lo, id_hi, step, 1) is below P.
 * The new electron starts at the ion's new position with the ion's new
 * momentum per unit mass (u = gamma beta is the same for equal velocities) and
 * the ion's weight; its id is 2^63 | (ion_id << 3) | (Z + 1).
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>

static double fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

double orc_adk_rate(double F, double Ip, double Z, int l, int m) {
    if (!(F > 0.0)) return 0.0;
    const int am = m < 0 ? -m : m;
    const double ns = Z / sqrt(2.0 * Ip), ls = ns - 1.0;
    const double C2 = pow(2.0, 2.0 * ns) / (ns * tgamma(ns + ls + 1.0) * tgamma(ns - ls));
    const double flm = (2.0 * l + 1.0) * fact(l + am) / (pow(2.0, am) * fact(am) * fact(l - am));
    const double k3 = pow(2.0 * Ip, 1.5);
    return C2 * flm * Ip * pow(2.0 * k3 / F, 2.0 * ns - am - 1.0) * exp(-2.0 * k3 / (3.0 * F));
}

/* the same formula as a logarithm (no underflow at weak field), m = 0 */
static double adk_log_rate(double F, double Ip, double Z, int l) {
    const double ns = Z / sqrt(2.0 * Ip), ls = ns - 1.0;
    const double C2 = pow(2.0, 2.0 * ns) / (ns * tgamma(ns + ls + 1.0) * tgamma(ns - ls));
    const double k3 = pow(2.0 * Ip, 1.5);
    return log(C2 * (2.0 * l + 1.0) * Ip) + (2.0 * ns - 1.0) * log(2.0 * k3 / F) - 2.0 * k3 / (3.0 * F);
}

double orc_keldysh(double F, double Ip, double w0) { return w0 * sqrt(2.0 * Ip) / F; }

double orc_mpi_rate(double F, double Ip, double Z, int l, double w0) {
    if (!(F > 0.0)) return 0.0;
    const double K = ceil(Ip / w0);
    const double Fs = w0 * sqrt(2.0 * Ip) / 1.5;
    const double ws = orc_adk_rate(Fs, Ip, Z, l, 0);
    return exp(log(ws) + 2.0 * K * log(F / Fs));
}

double orc_blend_weight(double gamma) { return 1.0 / (1.0 + exp(-(gamma - 1.5) / 0.1)); }

double orc_ionization_rate(double F, double Ip, double Z, int l, double w0) {
    if (!(F > 0.0)) return 0.0;
    const double S = orc_blend_weight(orc_keldysh(F, Ip, w0));
    const double K = ceil(Ip / w0);
    const double Fs = w0 * sqrt(2.0 * Ip) / 1.5;
    const double ln_mpi = adk_log_rate(Fs, Ip, Z, l) + 2.0 * K * log(F / Fs);
    const double ln_adk = adk_log_rate(F, Ip, Z, l);
    return exp(S * ln_mpi + (1.0 - S) * ln_adk);
}

long orc_ionize(orc_species *ions, const double *eb, int zmax, const double *Ip_au, const int *lq,
                double w0_au, double Eref_over_Ea, double dt_au, uint32_t seed, uint32_t sp_index, long step,
                orc_species *out, long cap, double *energy_au) {
    long n_new = 0;
    for (long p = 0; p < ions->n; ++p) {
        const int Z = (int)ions->zq[p];
        if (Z >= zmax) continue;
        const double *e = eb + 6 * p;
        const double F = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) * Eref_over_Ea;
        const double w = orc_ionization_rate(F, Ip_au[Z], (double)(Z + 1), lq[Z], w0_au);
        const double P = -expm1(-w * dt_au);
        const uint64_t id = ions->id[p];
        const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step, 1u};
        const uint32_t key[2] = {seed, sp_index};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        if (!(orc_u01(r[0]) < P)) continue;
        ions->zq[p] = Z + 1;
        *energy_au += ions->w[p] * Ip_au[Z];
        if (n_new < cap) {
            out->x[n_new] = ions->x[p]; out->y[n_new] = ions->y[p]; out->z[n_new] = ions->z[p];
            out->ux[n_new] = ions->ux[p]; out->uy[n_new] = ions->uy[p]; out->uz[n_new] = ions->uz[p];
            out->w[n_new] = ions->w[p];
            out->id[n_new] = (1ULL << 63) | (id << 3) | (uint64_t)(Z + 1);
        }
        ++n_new;
    }
    return n_new;
}
