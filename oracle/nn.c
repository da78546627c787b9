/*
 * Dropout masks of the regime classifier, from the oracle's own Philox.
 *
 * Paper: Methodology and Results -- Monte Carlo dropout provides the
 * uncertainty of the network's prediction (dropout kept active at inference,
 * statistics over repeated passes).  Mask of channel c of layer l at cell
 * (b, lin) in pass P: Philox4x32-10 with key (seed, 0xD0) and counter
 * (lin, b, (l << 16) | (c >> 2), P); the channel is kept unless the uniform
 * from word (c & 3) is below p.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"

void orc_dropout_mask(unsigned char *keep, int B, int C, long V, uint32_t seed, uint32_t pass, uint32_t layer,
                      double p) {
    for (int b = 0; b < B; ++b)
    for (int c0 = 0; c0 < C; c0 += 4)
    for (long v = 0; v < V; ++v) {
        const uint32_t ctr[4] = {(uint32_t)v, (uint32_t)b, (layer << 16) | ((uint32_t)c0 >> 2), pass};
        const uint32_t key[2] = {seed, 0xD0u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        for (int j = 0; j < 4 && c0 + j < C; ++j)
            keep[((long)b * C + c0 + j) * V + v] = !(orc_u01(r[j]) < p);
    }
}
