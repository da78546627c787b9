// Device lookup of the blended ADK / multiphoton ionization rate table
// (arXiv 2510.11174, Methodology: ADK tunnelling and multiphoton rates blended
// with a sigmoid transition at Keldysh parameter ~1.5).  The table holds
// ln w(F) for each charge state on a grid uniform in log2 F (F in atomic
// units, ION_NPO points per octave from 2^ION_E0), built in FP64 by
// k_build_ion_lut; lookups interpolate ln w linearly in log2 F.
#pragma once
#include "hyb_internal.cuh"

namespace hyb {


// rate [1/atomic time] of charge state Z at field strength F [atomic units]
__device__ __forceinline__ float ion_rate_lookup(const SpDev &sp, int Z, float F) {
    if (!(F > 0.0f)) return 0.0f;
    int i;
    float f;
    log2_grid(F, ION_E0, ION_NPO, i, f);
    if (i < 0) return 0.0f;  // below 2^-14 a.u. every rate is negligible
    if (i >= ION_NL - 1) {
        i = ION_NL - 2;
        f = 1.0f;
    }
    const float *t = sp.lnw + (long long)Z * ION_NL;
    return expf(t[i] + f * (t[i + 1] - t[i]));
}

// probability of one ionization event in a step: P = 1 - exp(-w dt)
__device__ __forceinline__ float ion_probability(const SpDev &sp, int Z, float Enorm) {
    const float w = ion_rate_lookup(sp, Z, Enorm * sp.e_ratio);
    return -expm1f(-w * sp.dt_au);
}

}  // namespace hyb
