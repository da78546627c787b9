// Device helpers shared by the particle kernels: tile membership, slot
// allocation, the initial optical depth and particle creation through a
// species' migration buffer.
#pragma once
#include "hyb_internal.cuh"
#include "philox.cuh"

namespace hyb {

__device__ __forceinline__ int tile_of_cell(const GridDev &g, int a, float p) {
    int c = (int)floorf(p);
    c = c < 0 ? 0 : (c > g.n[a] - 1 ? g.n[a] - 1 : c);
    return c >> g.tshift;
}

__device__ __forceinline__ int tile_index(const GridDev &g, float x, float y, float z) {
    return tile_of_cell(g, 0, x) + g.nt[0] * (tile_of_cell(g, 1, y) + g.nt[1] * tile_of_cell(g, 2, z));
}

// warp-aggregated slot allocation from a global counter (the active lanes of
// the calling warp get consecutive slots)
__device__ __forceinline__ int warp_append(int *counter) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int b = 0;
    if (lane == leader) b = atomicAdd(counter, __popc(mask));
    b = __shfl_sync(mask, b, leader);
    return b + __popc(mask & ((1u << lane) - 1u));
}

// a particle placed straight into tile t, which must hold no holes (a compacted
// tile); the lanes of a warp that target the same tile share one atomic.  A
// full tile latches ST_OVERFLOW and drops the particle (the count is clamped
// back to the capacity by launch_clamp_counts).
__device__ __forceinline__ void tile_put(const SpDev &d, int t, const float x[3], const float u[3], float w,
                                         uint64_t id, float tau, int *status) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, t);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int b = 0;
    if (lane == leader) b = atomicAdd(&d.count[t], __popc(peers));
    b = __shfl_sync(peers, b, leader);
    const int slot = b + __popc(peers & ((1u << lane) - 1u));
    if (slot >= d.cap) {
        atomicOr(status, ST_OVERFLOW);
        return;
    }
    const long long s = (long long)t * d.cap + slot;
    d.x[s] = x[0]; d.y[s] = x[1]; d.z[s] = x[2];
    d.ux[s] = u[0]; d.uy[s] = u[1]; d.uz[s] = u[2];
    d.w[s] = w;
    if (d.zq) d.zq[s] = 0.0f;
    if (d.tau) d.tau[s] = tau;
    d.id[s] = id;
}

// initial optical depth of a particle: -ln u, u from counter (id_lo, id_hi, 2^32-1, 4)
__device__ __forceinline__ float tau_initial(uint64_t id, uint32_t seed, uint32_t key1) {
    const u32x4 r = philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), 0xFFFFFFFFu, RNG_QED_TAU, seed, key1);
    return -logf(u01f(r.v[0]));
}

// a particle created by an event joins species d through its migration buffer
// (tau < 0: draw the initial optical depth from the particle's own stream)
__device__ __forceinline__ void spawn(const SpDev &d, const float x[3], const float u[3], float w, uint64_t id,
                                      int dest, long long step, uint32_t seed, float tau, int *status) {
    (void)step;
    const int m = warp_append(d.mig_count);
    if (m >= d.mig_cap) {
        atomicOr(status, ST_OVERFLOW);
        return;
    }
    d.mx[m] = x[0]; d.my[m] = x[1]; d.mz[m] = x[2];
    d.mux[m] = u[0]; d.muy[m] = u[1]; d.muz[m] = u[2];
    d.mw[m] = w;
    if (d.zq) d.mzq[m] = 0.0f;
    if (d.tau) d.mtau[m] = tau >= 0.0f ? tau : tau_initial(id, seed, d.tau_index);
    d.mid[m] = id;
    d.mdest[m] = dest;
}

}  // namespace hyb
