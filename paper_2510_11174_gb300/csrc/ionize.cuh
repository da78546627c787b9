// Device lookup of the blended ADK / multiphoton ionization rate table
// (arXiv 2510.11174, Methodology: ADK tunnelling and multiphoton rates blended
// with a sigmoid transition at Keldysh parameter ~1.5).  The table holds
// ln w(F) for each charge state on a uniform grid in ln F (F in atomic units),
// built in FP64 by k_build_ion_lut; lookups interpolate ln w linearly in ln F.
#pragma once
#include "hyb_internal.cuh"

namespace hyb {

// rate [1/atomic time] of charge state Z at field strength F [atomic units]
__device__ __forceinline__ float ion_rate_lookup(const SpDev &sp, int Z, float F) {
    if (!(F > 0.0f)) return 0.0f;
    float x = (logf(F) - sp.lnF0) * sp.inv_h;
    if (x < 0.0f) return 0.0f;  // below 1e-4 a.u. every rate is negligible
    const float xmax = (float)(ION_NL - 1);
    if (x >= xmax) x = xmax - 1e-3f;
    const int i = (int)x;
    const float f = x - (float)i;
    const float *t = sp.lnw + (long long)Z * ION_NL;
    return expf(t[i] + f * (t[i + 1] - t[i]));
}

// probability of one ionization event in a step: P = 1 - exp(-w dt)
__device__ __forceinline__ float ion_probability(const SpDev &sp, int Z, float Enorm) {
    const float w = ion_rate_lookup(sp, Z, Enorm * sp.e_ratio);
    return -expm1f(-w * sp.dt_au);
}

}  // namespace hyb
