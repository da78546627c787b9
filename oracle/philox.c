/*
 * Philox4x32-10 counter-based generator, written from its published
 * definition: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11, section 4.  Ten rounds; each round multiplies words 0
 * and 2 by the two Philox multipliers, xors the high halves with the other
 * two words and the round key, and permutes; the key is bumped by the two
 * Weyl constants between rounds.
 *
 * The paper (Methodology, reproducibility paragraph) relies on fixed
 * randomness for reproducible runs; a counter-based generator gives every
 * stochastic event its own stream keyed by (seed, species) and counted by
 * (particle id, step, purpose), independent of execution order.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"

static void mulhilo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(M0, c0, &hi0, &lo0);
        mulhilo(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_u01(uint32_t x) {
    /* 23 random bits centred in their bin: (2m+1) 2^-24 with 2m+1 < 2^24, so
     * the value is exact in FP32 and lies strictly inside (0, 1) */
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}
