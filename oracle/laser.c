/*
 * Gaussian laser soft source, FP64.
 *
 * Paper: Methodology -- the laser is a Gaussian pulse whose electric field
 * components get temporal and spatial envelopes according to polarisation;
 * intensity, duration and spot size are parameters.
 *
 * Reading used here (the paper gives no formula): a current sheet on the plane
 * x = x_src, J_pol = -2 A(t) f(y, z) / dx, radiates E_pol = A f to both sides
 * in normalised units (c = 1).  A(t) = a0 exp(-2 ln2 (t - t_peak)^2 / tau^2)
 * sin(t - t_peak) with tau the FWHM of the intensity, evaluated at the
 * current's time level t = (n + 1/2) dt; f = exp(-r^2 / w0^2) with w0 the
 * 1/e^2 intensity radius, r measured from (y_c, z_c) [cells] to the J_pol
 * position of the Yee cell.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"
#include <math.h>

void orc_laser_source(const orc_grid *g, int x_src, int pol, double a0, double tau, double t_peak,
                      double w0, double y_c, double z_c, long step, double *J[3]) {
    const double t = ((double)step + 0.5) * g->dt - t_peak;
    const double A = a0 * exp(-2.0 * log(2.0) * t * t / (tau * tau)) * sin(t);
    for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j) {
        if (pol == 1 && g->bc[1] != 0 && j > g->ny - 2) continue;  /* J_y at j+1/2 must exist */
        if (pol == 2 && g->bc[2] != 0 && k > g->nz - 2) continue;
        const double y = (j + (pol == 1 ? 0.5 : 0.0) - y_c) * g->dy;
        const double z = (k + (pol == 2 ? 0.5 : 0.0) - z_c) * g->dz;
        const double f = exp(-(y * y + z * z) / (w0 * w0));
        const long c = (long)x_src + (long)g->nx * ((long)j + (long)g->ny * k);
        J[pol][c] += -2.0 * A * f / g->dx;
    }
}
