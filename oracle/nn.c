/*
 * Dropout masks of the regime classifier, from the oracle's own Philox.
 *
 * Paper: Methodology and Results -- Monte Carlo dropout provides the
 * uncertainty of the network's prediction (dropout kept active at inference,
 * statistics over repeated passes).  Mask of channel c of layer l at cell
 * (b, lin) in pass P: Philox4x32-10 with key (seed, 0xD0) and counter
 * (lin, b, (l << 16) | (c / 8), P) gives eight 16-bit fields (field j = half
 * j % 2 of word j / 2, low half first); channel c is kept when field c % 8 is
 * at least round(p 2^16), i.e. with probability 1 - round(p 2^16) / 2^16.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include "orc.h"

#include <math.h>

/* The same masks for cells named by their index in a larger volume: position
 * v of the output takes the stream of cell cells[v] (a sub-box of a grid). */
void orc_dropout_mask_cells(unsigned char *keep, int B, int C, long V, const long *cells, uint32_t seed,
                            uint32_t pass, uint32_t layer, double p) {
    const long thr = lround(p * 65536.0);
    for (int b = 0; b < B; ++b)
    for (int c0 = 0; c0 < C; c0 += 8)
    for (long v = 0; v < V; ++v) {
        const uint32_t ctr[4] = {(uint32_t)cells[v], (uint32_t)b, (layer << 16) | ((uint32_t)c0 / 8u), pass};
        const uint32_t key[2] = {seed, 0xD0u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        for (int j = 0; j < 8 && c0 + j < C; ++j) {
            const long field = (long)((r[j / 2] >> (16 * (j % 2))) & 0xFFFFu);
            keep[((long)b * C + c0 + j) * V + v] = field >= thr;
        }
    }
}

void orc_dropout_mask(unsigned char *keep, int B, int C, long V, uint32_t seed, uint32_t pass, uint32_t layer,
                      double p) {
    const long thr = lround(p * 65536.0);
    for (int b = 0; b < B; ++b)
    for (int c0 = 0; c0 < C; c0 += 8)
    for (long v = 0; v < V; ++v) {
        const uint32_t ctr[4] = {(uint32_t)v, (uint32_t)b, (layer << 16) | ((uint32_t)c0 / 8u), pass};
        const uint32_t key[2] = {seed, 0xD0u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        for (int j = 0; j < 8 && c0 + j < C; ++j) {
            const long field = (long)((r[j / 2] >> (16 * (j % 2))) & 0xFFFFu);
            keep[((long)b * C + c0 + j) * V + v] = field >= thr;
        }
    }
}
