// Deterministic scatter of particle quantities onto the grid nodes.
//
// A CTA that owns a tile accumulates into a shared-memory frame of G^3 nodes
// (G = T + 3, origin one node below the tile's first node), which holds every
// node a CIC stencil, an Esirkepov stencil or a dual-cell particle of the tile
// can reach.  Values are accumulated in 64-bit fixed point: a value v adds
// round(v * 2^k) to an integer.  Integer addition is associative, so a frame
// does not depend on the order of the particles in the tile or of the warps
// that add them, and a run repeats bit for bit.  The exponent k is chosen per
// tile from a bound on the largest sum a frame node can reach (the tile's
// particle count times the largest |value| of one particle), so that no sum
// exceeds 2^62; for a tile of 4096 particles the quantum 2^-k is then about
// 2^-50 of the largest single contribution (FP32 keeps 2^-24 of each partial
// sum).  A frame is written out as FP32 (the integer times 2^-k, one rounding)
// and the frames that cover a node are summed in a fixed order.
#pragma once
#include "hyb_internal.cuh"

namespace hyb {

// frame edge in nodes: a shape of order k (1 CIC, 2 quadratic) reaches k nodes
// below the tile and k + 1 above it, so the frame spans T + 2k + 1 nodes
// starting k nodes below the tile's first node
__host__ __device__ constexpr int frame_G(int T, int order = 1) { return T + 2 * order + 1; }

// 2^k as FP32 for k in [-126, 127] (exact)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// exponent k with bound * 2^k < 2^62 (bound <= 0 or not finite: nothing to scale)
__device__ __forceinline__ int fix_exponent(double bound) {
    if (!(bound > 0.0) || !(bound < 1e300)) return 0;
    int e;
    frexp(bound, &e);  // bound < 2^e
    const int k = 62 - e;
    return k > 126 ? 126 : (k < -126 ? -126 : k);
}

// fixed-point image of a value already multiplied by 2^k
__device__ __forceinline__ unsigned long long fix_of(float scaled) {
    return (unsigned long long)__float2ll_rn(scaled);
}

__device__ __forceinline__ float fix_to_float(unsigned long long s, float inv_scale) {
    return __ll2float_rn((long long)s) * inv_scale;
}

// largest |v| over the block as the bits of a non-negative float (which order
// like integers): warp maximum, then one slot per warp in `slots`; the caller
// synchronises and reads block_max_read
__device__ __forceinline__ void block_max_put(float v, int *slots) {
    int b = __float_as_int(fabsf(v));
    b = __reduce_max_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0) slots[threadIdx.x >> 5] = b;
}
__device__ __forceinline__ float block_max_read(const int *slots) {
    int b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, slots[w]);
    return __int_as_float(b);
}

// Frames that cover node i along axis a: the frame of tile tt (shape order k)
// covers nodes tt*T - k .. tt*T + T + k; node i sits at r = i - own*T in
// [0, T) of its own tile, at local r + k in that tile's frame; the previous
// tile's frame reaches it when r <= k (at local r + T + k), the next tile's
// when r >= T - k (at local r - T + k).
__device__ __forceinline__ int frame_cands(const GridDev &g, int a, int i, int order, int tile[3], int loc[3]) {
    const int T = g.T, nt = g.nt[a];
    const int own = i >> g.tshift, r = i - own * T;
    int n = 0;
    if (r <= order) {
        int pt = own - 1;
        if (pt < 0 && g.bc[a] == 0) pt += nt;
        if (pt >= 0) { tile[n] = pt; loc[n] = r + T + order; ++n; }
    }
    tile[n] = own; loc[n] = r + order; ++n;
    if (r >= T - order) {
        int nt2 = own + 1;
        if (nt2 >= nt && g.bc[a] == 0) nt2 -= nt;
        if (nt2 < nt) { tile[n] = nt2; loc[n] = r - T + order; ++n; }
    }
    return n;
}

// sum over the frames covering node (i, j, k) of component q of a frame set
// with `ncomp` components per tile (frames of tiles whose flag is 0 are skipped)
template <int NC>
__device__ __forceinline__ void frame_gather(const GridDev &g, const float *__restrict__ scratch,
                                             const int *__restrict__ valid, int ncomp, int order, int i, int j,
                                             int k, float acc[NC]) {
    const int G = frame_G(g.T, order), G3 = G * G * G;
    int tx[3], lx[3], ty[3], ly[3], tz[3], lz[3];
    const int nxc = frame_cands(g, 0, i, order, tx, lx);
    const int nyc = frame_cands(g, 1, j, order, ty, ly);
    const int nzc = frame_cands(g, 2, k, order, tz, lz);
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = 0.0f;
    for (int cz = 0; cz < nzc; ++cz)
        for (int cy = 0; cy < nyc; ++cy)
            for (int cx = 0; cx < nxc; ++cx) {
                const long long t = tx[cx] + (long long)g.nt[0] * (ty[cy] + (long long)g.nt[1] * tz[cz]);
                if (!valid[t]) continue;
                const float *fr = scratch + t * (long long)ncomp * G3 + (lz[cz] * G + ly[cy]) * G + lx[cx];
#pragma unroll
                for (int q = 0; q < NC; ++q) acc[q] += fr[q * G3];
            }
}

}  // namespace hyb
