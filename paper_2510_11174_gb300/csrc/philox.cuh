// Philox4x32-10 counter-based generator for device code, from its published
// definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies by the Philox
// multipliers, xor of the high halves with the other words and the round key,
// and a word permutation; the key advances by the two Weyl constants between
// rounds.  A counter-based stream makes every stochastic event (ionization,
// photon emission, pair creation, particle sampling, dropout masks)
// reproducible and independent of execution order (arXiv 2510.11174,
// Methodology: fixed randomness for reproducible runs).
#pragma once
#include <stdint.h>

namespace hyb {

struct u32x4 {
    uint32_t v[4];
};

__host__ __device__ inline u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    u32x4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// 23 random bits centred in their bin, (2m+1) 2^-24: exact in FP32, in (0, 1)
__host__ __device__ inline float u01f(uint32_t x) { return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f); }

// purposes (counter word 3) of the random draws of a particle in a step
enum : uint32_t { RNG_IONIZE = 1u, RNG_QED_EMIT = 2u, RNG_QED_PAIR = 3u, RNG_QED_TAU = 4u };

}  // namespace hyb
