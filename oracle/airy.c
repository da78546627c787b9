/*
 * Airy functions for x >= 0 by quadrature of the modified Bessel function
 * integral, FP64.
 *
 * Paper: Methodology -- radiation reaction and pair production use Airy-function
 * approximations with the local field (locally-constant-field rates).
 *
 *   K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt                 (x > 0)
 *   int_x^inf K_nu(s) ds = int_0^inf exp(-x cosh t) cosh(nu t) / cosh t dt
 *   Ai(z)  = (1/pi) sqrt(z/3) K_{1/3}(zeta),     zeta = (2/3) z^{3/2}
 *   Ai'(z) = -(z / (pi sqrt 3)) K_{2/3}(zeta)
 *   int_z^inf Ai(t) dt = (1 / (pi sqrt 3)) int_zeta^inf K_{1/3}(s) ds
 *   Ai(0) = 1 / (3^{2/3} Gamma(2/3)),  Ai'(0) = -1 / (3^{1/3} Gamma(1/3))
 * (Abramowitz & Stegun 9.6.24, 10.4.14, 10.4.16).  The integrands are even
 * and analytic in t, so the trapezoid rule on [0, inf) converges
 * exponentially; the sum stops once the terms fall below 1e-18 of the total.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>

#define ORC_PI 3.14159265358979323846

static double kint(double nu, double x, int divide_by_cosh) {
    /* step: the integrand is analytic in a strip of half-width pi/2 (error ~
     * exp(-pi^2/h)); for large x it is a Gaussian of width 1/sqrt(x) around
     * t = 0, resolved by h <= 0.5/sqrt(x) */
    const double h = x > 16.0 ? 0.5 / sqrt(x) : 1.0 / 8.0;
    double sum = 0.5 * exp(-x);
    for (int i = 1; i < 200000; ++i) {
        const double t = i * h;
        const double ch = cosh(t);
        double term = 0.5 * (exp(-x * ch + nu * t) + exp(-x * ch - nu * t));
        if (divide_by_cosh) term /= ch;
        sum += term;
        if (term < 1e-18 * sum && x * ch > 1.0) break;
        if (t > 120.0) break;
    }
    return h * sum;
}

double orc_bessel_k(double nu, double x) { return kint(nu, x, 0); }
double orc_bessel_k_int(double nu, double x) { return kint(nu, x, 1); }

double orc_airy_ai(double z) {
    if (z == 0.0) return 1.0 / (pow(3.0, 2.0 / 3.0) * tgamma(2.0 / 3.0));
    const double zeta = 2.0 / 3.0 * z * sqrt(z);
    return sqrt(z / 3.0) / ORC_PI * orc_bessel_k(1.0 / 3.0, zeta);
}

double orc_airy_aip(double z) {
    if (z == 0.0) return -1.0 / (pow(3.0, 1.0 / 3.0) * tgamma(1.0 / 3.0));
    const double zeta = 2.0 / 3.0 * z * sqrt(z);
    return -z / (ORC_PI * sqrt(3.0)) * orc_bessel_k(2.0 / 3.0, zeta);
}

double orc_airy_int(double z) {
    const double zeta = 2.0 / 3.0 * z * sqrt(z);
    return orc_bessel_k_int(1.0 / 3.0, zeta) / (ORC_PI * sqrt(3.0));
}
