// Regime switching: the physics criterion (or the classifier's decision), the
// dilated mask, and the charge-exact fluid <-> particle conversions
// (arXiv 2510.11174, Methodology: fluid models in stable regions, PIC where
// the learned switch flags instability; charge and energy checked during
// regime switches).  The paper does not define the criterion; the reading is
// stated with hyb_regime_desc in include/hyb.h.
//
// Every scatter onto the nodes here (CIC electron density, particle moments
// deposited into a fluid, the charge of converted particles) goes through the
// per-tile fixed-point frames of frames.cuh and a fixed-order gather, so a
// classification repeats bit for bit like the step.
#include <algorithm>

#include "frames.cuh"
#include "hyb_internal.cuh"
#include "particles.cuh"
#include "qed.cuh"

namespace hyb {

__device__ __forceinline__ float node_e(const GridDev &g, const float *__restrict__ E, int i, int j, int k,
                                        float e[3]) {
    auto fv = [&](const float *F, int a, int b, int c) -> float {
        int idx[3] = {a, b, c};
        for (int ax = 0; ax < 3; ++ax) {
            if (g.bc[ax] == 0) idx[ax] = idx[ax] < 0 ? idx[ax] + g.n[ax] : (idx[ax] >= g.n[ax] ? idx[ax] - g.n[ax] : idx[ax]);
            else if (idx[ax] < 0 || idx[ax] > g.n[ax] - 1) return 0.0f;
        }
        return F[cidx(g, idx[0], idx[1], idx[2])];
    };
    const long long N = g.N;
    e[0] = 0.5f * (fv(E, i - 1, j, k) + fv(E, i, j, k));
    e[1] = 0.5f * (fv(E + N, i, j - 1, k) + fv(E + N, i, j, k));
    e[2] = 0.5f * (fv(E + 2 * N, i, j, k - 1) + fv(E + 2 * N, i, j, k));
    return sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
}

// CIC weights of a particle position along axis a: base node (clamped below
// the top wall of an absorbing axis) and the fraction toward the next node
__device__ __forceinline__ void cic_axis(const GridDev &g, int a, float p, int &b, float &f) {
    int i = (int)floorf(p);
    if (g.bc[a] && i > g.n[a] - 2) i = g.n[a] - 2;
    b = i;
    f = p - (float)i;
}

// the tile's frame origin (one node below its first node) per axis
__device__ __forceinline__ void tile_origin(const GridDev &g, int t, int o[3]) {
    o[0] = (t % g.nt[0]) * g.T - 1;
    o[1] = ((t / g.nt[0]) % g.nt[1]) * g.T - 1;
    o[2] = (t / (g.nt[0] * g.nt[1])) * g.T - 1;
}

// add v times the CIC weights of a particle at pos (unwrapped, inside the
// frame) to component q of a fixed-point frame
__device__ __forceinline__ void frame_cic(const GridDev &g, unsigned long long *fr, int G, const int o[3],
                                          const float pos[3], float v) {
    int b[3];
    float f[3];
    for (int a = 0; a < 3; ++a) cic_axis(g, a, pos[a], b[a], f[a]);
    for (int c = 0; c < 8; ++c) {
        const float wgt = ((c & 1) ? f[0] : 1.0f - f[0]) * (((c >> 1) & 1) ? f[1] : 1.0f - f[1]) *
                          ((c >> 2) ? f[2] : 1.0f - f[2]);
        const int l0 = b[0] + (c & 1) - o[0], l1 = b[1] + ((c >> 1) & 1) - o[1], l2 = b[2] + (c >> 2) - o[2];
        if (wgt != 0.0f) atomicAdd(&fr[(l2 * G + l1) * G + l0], fix_of(wgt * v));
    }
}

// a particle position of tile t is inside the tile's cells (what the frames assume)
__device__ __forceinline__ bool in_tile(const GridDev &g, const int o[3], const float pos[3]) {
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
        int ci = (int)floorf(pos[a]);
        if (g.bc[a] && ci > g.n[a] - 2) ci = g.n[a] - 2;
        ok = ok && isfinite(pos[a]) && ci >= o[a] + 1 && ci <= o[a] + g.T;
    }
    return ok;
}

// electron density (charge = 0: n_e = -q w / dV) or charge density (charge =
// 1: q w / dV, times the charge state where the species has one) from the
// macro-particles of the species in `which` (bit s: species s), CIC: one
// fixed-point frame per tile, then a fixed-order gather
__global__ void __launch_bounds__(256) k_density_frames(GridDev g, const SpDev *__restrict__ sps, int nsp,
                                                         unsigned which, int charge, float *__restrict__ scratch,
                                                         int *__restrict__ valid, int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *fr = reinterpret_cast<unsigned long long *>(smraw);
    __shared__ int s_max[32];
    const int t = blockIdx.x, G = frame_G(g.T), G3 = G * G * G;
    const float idV = 1.0f / (g.d[0] * g.d[1] * g.d[2]);
    int total = 0;
    float vmax = 0.0f;
    for (int si = 0; si < nsp; ++si) {
        if (!((which >> si) & 1u)) continue;
        const SpDev &sp = sps[si];
        const int n = min(sp.count[t], sp.cap);
        total += n;
        const float *zq = charge ? sp.zq : nullptr;
        for (int p = threadIdx.x; p < n; p += blockDim.x)
            vmax = fmaxf(vmax, fabsf(sp.q * idV * sp.w[(long long)t * sp.cap + p] * (zq ? zq[(long long)t * sp.cap + p] : 1.0f)));
    }
    if (total == 0) {
        if (threadIdx.x == 0) valid[t] = 0;
        return;
    }
    block_max_put(vmax, s_max);
    for (int l = threadIdx.x; l < G3; l += blockDim.x) fr[l] = 0ULL;
    __syncthreads();
    const int k = fix_exponent((double)total * (double)block_max_read(s_max));
    const float sc = pow2f(k);
    int o[3];
    tile_origin(g, t, o);
    for (int si = 0; si < nsp; ++si) {
        if (!((which >> si) & 1u)) continue;
        const SpDev &sp = sps[si];
        const int n = min(sp.count[t], sp.cap);
        const long long base = (long long)t * sp.cap;
        const float qv = (charge ? sp.q : -sp.q) * idV * sc;  // electrons: n_e = -q w / dV
        const float *zq = charge ? sp.zq : nullptr;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const float pos[3] = {sp.x[base + p], sp.y[base + p], sp.z[base + p]};
            if (!in_tile(g, o, pos)) {
                atomicOr(status, ST_BADPOS);
                continue;
            }
            frame_cic(g, fr, G, o, pos, qv * sp.w[base + p] * (zq ? zq[base + p] : 1.0f));
        }
    }
    __syncthreads();
    float *dst = scratch + (long long)t * G3;
    const float inv = pow2f(-k);
    for (int l = threadIdx.x; l < G3; l += blockDim.x) dst[l] = fix_to_float(fr[l], inv);
    if (threadIdx.x == 0) valid[t] = 1;
}

__global__ void k_density_gather(GridDev g, const float *__restrict__ scratch, const int *__restrict__ valid,
                                 float *__restrict__ ne) {
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    float acc[1];
    frame_gather<1>(g, scratch, valid, 1, 1, i, j, k, acc);
    ne[((long long)k * ny + j) * nx + i] = acc[0];
}

__global__ void k_criterion(GridDev g, const float *__restrict__ E, const float *__restrict__ ne, FluidDev fe,
                            int has_fluid, float kappa, float a_thr, float n_thr, float c_thr, float chi_thr,
                            uint8_t *__restrict__ raw) {
    const int nx = g.n[0], ny = g.n[1];
    const int idx[3] = {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)blockIdx.y, (int)blockIdx.z};
    if (idx[0] >= nx) return;
    const long long c = ((long long)idx[2] * ny + idx[1]) * nx + idx[0];
    float e[3];
    const float emag = node_e(g, E, idx[0], idx[1], idx[2], e);
    float dens = ne[c] + (has_fluid ? fe.n[c] : 0.0f);
    bool kin = emag >= a_thr || dens >= n_thr;
    float u2 = 0.0f;
    if (has_fluid) {
        const float *U[3] = {fe.ux, fe.uy, fe.uz};
        u2 = U[0][c] * U[0][c] + U[1][c] * U[1][c] + U[2][c] * U[2][c];
        float div = 0.0f;
        for (int a = 0; a < 3; ++a) {
            int lo[3] = {idx[0], idx[1], idx[2]}, hi[3] = {idx[0], idx[1], idx[2]};
            float span = 2.0f * g.d[a];
            if (g.bc[a] == 0) {
                lo[a] = idx[a] == 0 ? g.n[a] - 1 : idx[a] - 1;
                hi[a] = idx[a] == g.n[a] - 1 ? 0 : idx[a] + 1;
            } else {
                lo[a] = idx[a] > 0 ? idx[a] - 1 : idx[a];
                hi[a] = idx[a] < g.n[a] - 1 ? idx[a] + 1 : idx[a];
                span = (float)(hi[a] - lo[a]) * g.d[a];
            }
            const long long cl = cidx(g, lo[0], lo[1], lo[2]), ch = cidx(g, hi[0], hi[1], hi[2]);
            const float vl = U[a][cl] / sqrtf(1.0f + U[0][cl] * U[0][cl] + U[1][cl] * U[1][cl] + U[2][cl] * U[2][cl]);
            const float vh = U[a][ch] / sqrtf(1.0f + U[0][ch] * U[0][ch] + U[1][ch] * U[1][ch] + U[2][ch] * U[2][ch]);
            if (span > 0.0f) div += (vh - vl) / span;
        }
        kin = kin || g.dt * div <= -c_thr;
    }
    kin = kin || kappa * sqrtf(1.0f + u2) * emag >= chi_thr;
    raw[c] = kin ? 1 : 0;
}

// classifier decision; with `merge` the node also stays kinetic where the
// physics criterion already marked it
__global__ void k_decide(long long N, const float *__restrict__ pm, const float *__restrict__ ps, float k_sigma,
                         int merge, uint8_t *__restrict__ raw) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const bool kin = pm[c] + k_sigma * ps[c] >= 0.5f;
    raw[c] = (kin || (merge && raw[c])) ? 1 : 0;
}

__global__ void k_clamp_counts(int ntiles, SpDev sp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    if (sp.count[t] > sp.cap) sp.count[t] = sp.cap;
    if (2 * sp.count[t] > sp.cap) atomicOr(sp.fill_flags, 1 << sp.sp_index);
}

// max filter of radius r along axis a (Chebyshev dilation is three of these)
// grid (ceil(nx / blockDim.x), ny, nz)
__global__ void k_dilate(GridDev g, int a, int r, const uint8_t *__restrict__ in, uint8_t *__restrict__ out) {
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long c = ((long long)k * ny + j) * nx + i;
    const int i0 = a == 0 ? i : (a == 1 ? j : k), n = g.n[a];
    const long long st = a == 0 ? 1 : (a == 1 ? (long long)nx : (long long)nx * ny);
    // every load independent of the others (no early exit), so they overlap
    uint8_t m = 0;
#pragma unroll
    for (int d = -8; d <= 8; ++d) {
        if (d < -r || d > r) continue;
        int q = i0 + d;
        if (g.bc[a] == 0) q = r < n ? (q < 0 ? q + n : (q >= n ? q - n : q)) : ((q % n) + n) % n;
        else if (q < 0 || q > n - 1) continue;
        m |= in[c + (q - i0) * st];
    }
    out[c] = m ? 1 : 0;
}

// the maximum filter along x over whole 32-bit words (four nodes per thread,
// nx % 4 == 0, r <= 4): the words left and right of a node's word hold every
// byte within r of it
__global__ void k_dilate4x(GridDev g, int r, const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    const int nx4 = g.n[0] >> 2, ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx4) return;
    const long long row = ((long long)k * ny + j) * nx4;
    const bool per = g.bc[0] == 0;
    const uint32_t w = in[row + i];
    const uint32_t L = i > 0 ? in[row + i - 1] : (per ? in[row + nx4 - 1] : 0u);
    const uint32_t R = i < nx4 - 1 ? in[row + i + 1] : (per ? in[row] : 0u);
    const uint64_t lw = ((uint64_t)w << 32) | L;  // byte b: node 4 i - 4 + b
    const uint64_t rw = ((uint64_t)R << 32) | w;  // byte b: node 4 i + b
    uint32_t m = w;
    for (int d = 1; d <= r; ++d) m |= (uint32_t)(lw >> (8 * (4 - d))) | (uint32_t)(rw >> (8 * d));
    out[row + i] = m;
}

// the same maximum filter along y or z (a = 1, 2) for four consecutive x
// nodes at once (nx % 4 == 0): whole 32-bit words of the mask
__global__ void k_dilate4(GridDev g, int a, int r, const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    const int nx4 = g.n[0] >> 2, ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx4) return;
    const long long c = ((long long)k * ny + j) * nx4 + i;
    const int i0 = a == 1 ? j : k, n = g.n[a];
    const long long st = a == 1 ? (long long)nx4 : (long long)nx4 * ny;
    uint32_t m = 0;
#pragma unroll
    for (int d = -8; d <= 8; ++d) {
        if (d < -r || d > r) continue;
        int q = i0 + d;
        if (g.bc[a] == 0) q = r < n ? (q < 0 ? q + n : (q >= n ? q - n : q)) : ((q % n) + n) % n;
        else if (q < 0 || q > n - 1) continue;
        m |= in[c + (q - i0) * st];
    }
    out[c] = m;  // bytes are 0 or 1, so OR is the maximum
}

// fluid -> particles at the nodes that switch to kinetic; one CTA per tile
// walks the tile's nodes.  rho_bg takes (removed fluid charge) - (CIC charge of
// the new particles): both go into the tile's fixed-point frame, which
// k_rho_gather adds to rho_bg in a fixed order.
// sub-lattice of a quiet start: lx >= ly >= lz with lx ly lz = ppc, lz the
// largest divisor of ppc with lz^3 <= ppc, ly the largest divisor of ppc / lz
// with ly^2 <= ppc / lz
__host__ __device__ inline void quiet_lattice(int ppc, int l[3]) {
    int lz = 1, ly = 1;
    for (int d = 1; d * d * d <= ppc; ++d)
        if (ppc % d == 0) lz = d;
    const int r = ppc / lz;
    for (int d = 1; d * d <= r; ++d)
        if (r % d == 0) ly = d;
    l[0] = r / ly;
    l[1] = ly;
    l[2] = lz;
}

__global__ void __launch_bounds__(256) k_fluid_to_particles(GridDev g, const uint8_t *__restrict__ mask,
                                                             const uint8_t *__restrict__ prev, FluidDev f, SpDev dst,
                                                             int ppc, int quiet, uint32_t epoch,
                                                             float *__restrict__ scratch, int *__restrict__ valid,
                                                             int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *fr = reinterpret_cast<unsigned long long *>(smraw);
    __shared__ int s_max[32];
    const int t = blockIdx.x, T = g.T, G = frame_G(T), G3 = G * G * G, T3 = T * T * T;
    int o[3];
    tile_origin(g, t, o);
    const int nx = g.n[0], ny = g.n[1];
    auto node_of = [&](int l, int idx[3]) -> long long {
        idx[0] = o[0] + 1 + l % T;
        idx[1] = o[1] + 1 + (l / T) % T;
        idx[2] = o[2] + 1 + l / (T * T);
        return ((long long)idx[2] * ny + idx[1]) * nx + idx[0];
    };
    // only nodes that switch to kinetic now: fluid that flows into a node
    // that was kinetic already stays fluid there
    auto converts = [&](long long c) { return mask[c] && !prev[c] && f.n[c] > f.n_floor; };
    float qmax = 0.0f;
    int any = 0;
    for (int l = threadIdx.x; l < T3; l += blockDim.x) {
        int idx[3];
        const long long c = node_of(l, idx);
        if (converts(c)) {
            qmax = fmaxf(qmax, fabsf(f.q * f.n[c]));
            any = 1;
        }
    }
    if (!__syncthreads_or(any)) {
        if (threadIdx.x == 0) valid[t] = 0;
        return;
    }
    block_max_put(qmax, s_max);
    for (int l = threadIdx.x; l < G3; l += blockDim.x) fr[l] = 0ULL;
    __syncthreads();
    // each converting node adds q n at itself and -q n spread by CIC: a node's
    // sum is at most 2 T^3 max |q n|
    const int k = fix_exponent(2.0 * (double)T3 * (double)block_max_read(s_max));
    const float sc = pow2f(k);
    const float dV = g.d[0] * g.d[1] * g.d[2];
    int lat[3];
    quiet_lattice(ppc, lat);
    for (int l = threadIdx.x; l < T3; l += blockDim.x) {
        int idx[3];
        const long long c = node_of(l, idx);
        if (!converts(c)) continue;
        const float n = f.n[c];
        const float w = n * dV / (float)ppc;
        {
            const int l0 = idx[0] - o[0], l1 = idx[1] - o[1], l2 = idx[2] - o[2];
            atomicAdd(&fr[(l2 * G + l1) * G + l0], fix_of(f.q * n * sc));
        }
        const float u[3] = {f.ux[c], f.uy[c], f.uz[c]};
        for (int p = 0; p < ppc; ++p) {
            const u32x4 r = philox4x32_10((uint32_t)c, epoch, (uint32_t)p, 6u, g.seed, dst.sp_index);
            const int lm[3] = {p % lat[0], (p / lat[0]) % lat[1], p / (lat[0] * lat[1])};
            float pos[3], upos[3];
            for (int a = 0; a < 3; ++a) {
                float lo = (float)idx[a] - 0.5f, hi = (float)idx[a] + 0.5f;
                if (g.bc[a]) {
                    lo = fmaxf(lo, 0.0f);
                    hi = fminf(hi, (float)(g.n[a] - 1));
                }
                const float frac = quiet ? ((float)lm[a] + 0.5f) / (float)lat[a] : u01f(r.v[a]);
                upos[a] = lo + (hi - lo) * frac;
                pos[a] = upos[a];
                if (g.bc[a] == 0) {
                    if (pos[a] < 0.0f) pos[a] += (float)g.n[a];
                    if (pos[a] >= (float)g.n[a]) pos[a] -= (float)g.n[a];
                    if (pos[a] >= (float)g.n[a]) pos[a] = 0.0f;
                }
            }
            // CIC charge of the new particle leaves rho_bg (the unwrapped
            // position indexes the frame; the gather wraps periodic axes)
            frame_cic(g, fr, G, o, upos, -dst.q * w / dV * sc);
            const uint64_t id = (1ULL << 62) | (derived_id((uint64_t)c | ((uint64_t)epoch << 40), p, 6u) >> 2);
            const float tau = dst.tau ? tau_initial(id, g.seed, dst.tau_index) : 0.0f;
            tile_put(dst, tile_index(g, pos[0], pos[1], pos[2]), pos, u, w, id, tau, status);
        }
        f.n[c] = 0.0f;
        f.ux[c] = f.uy[c] = f.uz[c] = 0.0f;
    }
    __syncthreads();
    float *out = scratch + (long long)t * G3;
    const float inv = pow2f(-k);
    for (int l = threadIdx.x; l < G3; l += blockDim.x) out[l] = fix_to_float(fr[l], inv);
    if (threadIdx.x == 0) valid[t] = 1;
}

__global__ void k_rho_gather(GridDev g, const float *__restrict__ scratch, const int *__restrict__ valid,
                             float *__restrict__ rho_bg) {
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    float acc[1];
    frame_gather<1>(g, scratch, valid, 1, 1, i, j, k, acc);
    const long long c = ((long long)k * ny + j) * nx + i;
    if (acc[0] != 0.0f) rho_bg[c] += acc[0];
}

// particles whose nearest node is fluid: CIC-deposit n and n u into the tile's
// fixed-point frame (4 components), then remove them; k_moments_gather adds
// the frames to the fluid in a fixed order
__global__ void __launch_bounds__(256) k_particles_to_fluid(GridDev g, const uint8_t *__restrict__ mask, SpDev sp,
                                                             float *__restrict__ scratch, int *__restrict__ valid,
                                                             int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *fr = reinterpret_cast<unsigned long long *>(smraw);  // n, n ux, n uy, n uz
    __shared__ int s_holes;
    __shared__ int s_max[2][32];
    const int t = blockIdx.x, G = frame_G(g.T), G3 = G * G * G;
    const int n = min(sp.count[t], sp.cap);
    const long long base = (long long)t * sp.cap;
    const float idV = 1.0f / (g.d[0] * g.d[1] * g.d[2]);
    int o[3];
    tile_origin(g, t, o);
    auto nearest_fluid = [&](const float pos[3]) {
        int nd[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floorf(pos[a] + 0.5f);
            if (g.bc[a] == 0) i = i >= g.n[a] ? i - g.n[a] : i;
            else if (i > g.n[a] - 1) i = g.n[a] - 1;
            nd[a] = i;
        }
        return mask[cidx(g, nd[0], nd[1], nd[2])] == 0;
    };
    float wmax = 0.0f, wumax = 0.0f;
    int any = 0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const long long s = base + p;
        const float pos[3] = {sp.x[s], sp.y[s], sp.z[s]};
        if (!nearest_fluid(pos)) continue;
        const float wn = sp.w[s] * idV;
        wmax = fmaxf(wmax, fabsf(wn));
        wumax = fmaxf(wumax, fabsf(wn) * fmaxf(fabsf(sp.ux[s]), fmaxf(fabsf(sp.uy[s]), fabsf(sp.uz[s]))));
        any = 1;
    }
    if (threadIdx.x == 0) s_holes = 0;
    if (!__syncthreads_or(any)) {
        if (threadIdx.x == 0) {
            valid[t] = 0;
            sp.hole_count[t] = 0;
            sp.hole_used[t] = 0;
        }
        return;
    }
    block_max_put(wmax, s_max[0]);
    block_max_put(wumax, s_max[1]);
    for (int l = threadIdx.x; l < 4 * G3; l += blockDim.x) fr[l] = 0ULL;
    __syncthreads();
    const int kn = fix_exponent((double)n * (double)block_max_read(s_max[0]));
    const int ku = fix_exponent((double)n * (double)block_max_read(s_max[1]));
    const float sn = pow2f(kn), su = pow2f(ku);
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const long long s = base + p;
        const float pos[3] = {sp.x[s], sp.y[s], sp.z[s]};
        if (!nearest_fluid(pos)) continue;
        if (!in_tile(g, o, pos)) {
            atomicOr(status, ST_BADPOS);
            continue;
        }
        const float wn = sp.w[s] * idV;
        frame_cic(g, fr, G, o, pos, wn * sn);
        frame_cic(g, fr + G3, G, o, pos, wn * sp.ux[s] * su);
        frame_cic(g, fr + 2 * G3, G, o, pos, wn * sp.uy[s] * su);
        frame_cic(g, fr + 3 * G3, G, o, pos, wn * sp.uz[s] * su);
        const int h = atomicAdd(&s_holes, 1);
        sp.holes[base + h] = p;
        sp.x[s] = -1.0f;
    }
    __syncthreads();
    float *out = scratch + (long long)t * 4 * G3;
    const float in_ = pow2f(-kn), iu = pow2f(-ku);
    for (int l = threadIdx.x; l < 4 * G3; l += blockDim.x) out[l] = fix_to_float(fr[l], l < G3 ? in_ : iu);
    if (threadIdx.x == 0) {
        valid[t] = 1;
        sp.hole_count[t] = s_holes;
        sp.hole_used[t] = 0;
    }
}

// fluid += the deposited moments: n' = n + sum n_p, u' = (n u + sum n_p u_p) / n'
// (u' = 0 where n' is at or below the floor)
__global__ void k_moments_gather(GridDev g, const float *__restrict__ scratch, const int *__restrict__ valid,
                                 FluidDev f) {
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    float acc[4];
    frame_gather<4>(g, scratch, valid, 4, 1, i, j, k, acc);
    const long long c = ((long long)k * ny + j) * nx + i;
    const float n0 = f.n[c];
    if (acc[0] == 0.0f && acc[1] == 0.0f && acc[2] == 0.0f && acc[3] == 0.0f) {
        if (!(n0 > f.n_floor)) f.ux[c] = f.uy[c] = f.uz[c] = 0.0f;
        return;
    }
    const float n1 = n0 + acc[0];
    const bool keep = n1 > f.n_floor;
    const float mx = n0 * f.ux[c] + acc[1], my = n0 * f.uy[c] + acc[2], mz = n0 * f.uz[c] + acc[3];
    f.n[c] = n1;
    f.ux[c] = keep ? mx / n1 : 0.0f;
    f.uy[c] = keep ? my / n1 : 0.0f;
    f.uz[c] = keep ? mz / n1 : 0.0f;
}

static inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

// Criterion (or classifier decision) -> dilated mask -> conversions.
// charges and densities of the fluids (a kernel parameter)
struct FluidCharges {
    float q[HYB_MAX_FLUIDS];
    const float *n_[HYB_MAX_FLUIDS];
    int n;
};

// rho += q n of every fluid + rho_bg
__global__ void k_rho_fluids(long long N, FluidCharges fs, const float *__restrict__ rho_bg, float *__restrict__ rho) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= N) return;
    float r = rho[c] + (rho_bg ? rho_bg[c] : 0.0f);
    for (int f = 0; f < fs.n; ++f) r += fs.q[f] * fs.n_[f][c];
    rho[c] = r;
}

// charge density at the nodes into rho (device FP32 [nz][ny][nx])
hyb_status charge_density(hyb_ctx *c, float *rho) {
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    unsigned which = 0;
    for (size_t si = 0; si < c->sp.size() && si < 32; ++si)
        if (c->sp[si].dev.kind == 0) which |= 1u << si;
    if (which) {
        const int fG = frame_G(g.T);
        const size_t sm1 = sizeof(unsigned long long) * (size_t)fG * fG * fG;
        k_density_frames<<<g.ntiles, 256, sm1, st>>>(g, c->sp_dev, (int)c->sp.size(), which, 1, c->jscratch,
                                                     c->jvalid, c->status);
        k_density_gather<<<node_grid(g), node_block(g), 0, st>>>(g, c->jscratch, c->jvalid, rho);
    } else {
        cudaMemsetAsync(rho, 0, sizeof(float) * g.N, st);
    }
    FluidCharges fs;
    memset(&fs, 0, sizeof(fs));
    for (size_t f = 0; f < c->fluids.size() && fs.n < HYB_MAX_FLUIDS; ++f) {
        fs.q[fs.n] = c->fluids[f].q;
        fs.n_[fs.n++] = c->fluids[f].n;
    }
    k_rho_fluids<<<nblk(g.N), 256, 0, st>>>(g.N, fs, c->rho_bg, rho);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("charge density: ") + cudaGetErrorString(e));
    return HYB_OK;
}

struct FluidFloors {
    float floor_[HYB_MAX_FLUIDS];
};

// x-planes that hold matter: a fluid above its floor at some node of the
// plane, or a particle in a cell of the plane (plane floor(x), at most nx - 1)
__global__ void k_matter_fluid(GridDev g, FluidCharges fs, FluidFloors fl, int *__restrict__ flag) {
    const int nx = g.n[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long c = ((long long)k * g.n[1] + j) * nx + i;
    bool any = false;
    for (int f = 0; f < fs.n; ++f) any = any || fs.n_[f][c] > fl.floor_[f];
    if (any) flag[i] = 1;  // every writer stores the same value
}

// one block per tile: the planes of its particles gathered in shared memory
// first (a tile spans T planes), then written once
__global__ void __launch_bounds__(256) k_matter_particles(GridDev g, SpDev sp, int *__restrict__ flag) {
    __shared__ int sflag[32];
    const int t = blockIdx.x, T = g.T, nx = g.n[0];
    const int x0 = (t % g.nt[0]) * T;
    if (threadIdx.x < 32) sflag[threadIdx.x] = 0;
    __syncthreads();
    const int n = min(sp.count[t], sp.cap);
    const long long base = (long long)t * sp.cap;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        const float x = sp.x[base + l];
        int p = (int)floorf(x);
        p = p < 0 ? 0 : (p > nx - 1 ? nx - 1 : p);
        if (p >= x0 && p < x0 + T && T <= 32) sflag[p - x0] = 1;
        else flag[p] = 1;
    }
    __syncthreads();
    if ((int)threadIdx.x < T && T <= 32 && sflag[threadIdx.x] && x0 + (int)threadIdx.x < nx) flag[x0 + threadIdx.x] = 1;
}

hyb_status matter_x_range(hyb_ctx *c, int reach, int *xa, int *xb) {
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    const int nx = g.n[0];
    if (!c->xflag) {
        if (ctx_alloc(c, (void **)&c->xflag, sizeof(int) * (size_t)nx)) return set_error(HYB_ENOMEM, "matter flags");
        if (cudaMallocHost((void **)&c->xflag_host, sizeof(int) * (size_t)nx) != cudaSuccess)
            return set_error(HYB_ENOMEM, "pinned matter flags");
    }
    HYB_CUDA_TRY(cudaMemsetAsync(c->xflag, 0, sizeof(int) * (size_t)nx, st));
    FluidCharges fs;
    FluidFloors fl;
    memset(&fs, 0, sizeof(fs));
    memset(&fl, 0, sizeof(fl));
    for (size_t f = 0; f < c->fluids.size() && fs.n < HYB_MAX_FLUIDS; ++f) {
        fl.floor_[fs.n] = c->fluids[f].n_floor;
        fs.n_[fs.n++] = c->fluids[f].n;
    }
    if (fs.n > 0) k_matter_fluid<<<node_grid(g), node_block(g), 0, st>>>(g, fs, fl, c->xflag);
    for (size_t si = 0; si < c->sp.size(); ++si)
        k_matter_particles<<<g.ntiles, 256, 0, st>>>(g, c->sp[si].dev, c->xflag);
    HYB_CUDA_TRY(cudaMemcpyAsync(c->xflag_host, c->xflag, sizeof(int) * (size_t)nx, cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));
    int lo = nx, hi = -1;
    for (int x = 0; x < nx; ++x)
        if (c->xflag_host[x]) {
            lo = std::min(lo, x);
            hi = x;
        }
    if (hi < 0) {
        *xa = *xb = 0;
        return HYB_OK;
    }
    // on a periodic x-axis a range that reaches an end wraps round: take every plane
    if (g.bc[0] == 0 && (lo - reach < 0 || hi + 1 + reach > nx)) {
        *xa = 0;
        *xb = nx;
        return HYB_OK;
    }
    *xa = std::max(0, lo - reach);
    *xb = std::min(nx, hi + 1 + reach);
    return HYB_OK;
}

// x-planes where some fluid's density is not exactly zero
__global__ void k_fluid_nonzero(GridDev g, FluidCharges fs, int *__restrict__ flag) {
    const int nx = g.n[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long c = ((long long)k * g.n[1] + j) * nx + i;
    bool any = false;
    for (int f = 0; f < fs.n; ++f) any = any || fs.n_[f][c] != 0.0f;
    if (any) flag[i] = 1;  // every writer stores the same value
}

hyb_status clear_fluid_range(hyb_ctx *c, cudaStream_t st) {
    c->fluid_xr_until = -1;
    HYB_CUDA_TRY(cudaMemsetAsync(c->fluid_xr, 0, 2 * sizeof(int), st));
    return HYB_OK;
}

// The fluid kernels may skip the planes farther than `reach` from every plane
// with nonzero fluid density for the next `reach` steps: fluid spreads at most
// one node per step, and the transport of step k needs u* only where the
// density may be nonzero after k steps (a face between two empty nodes carries
// no flux).  An empty node outside the range keeps u = 0, which the update of
// every node has set since the latest load (so at least one step must have
// run since then); conversions happen only in hyb_classify, before this.
hyb_status set_fluid_range(hyb_ctx *c) {
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    const int nx = g.n[0], reach = c->regime.reach;
    if (reach <= 0 || c->fluids.empty() || c->fluids_idle || c->step <= c->fluid_fresh_step)
        return clear_fluid_range(c, st);
    if (!c->xflag) {
        if (ctx_alloc(c, (void **)&c->xflag, sizeof(int) * (size_t)nx)) return set_error(HYB_ENOMEM, "matter flags");
        if (cudaMallocHost((void **)&c->xflag_host, sizeof(int) * (size_t)nx) != cudaSuccess)
            return set_error(HYB_ENOMEM, "pinned matter flags");
    }
    HYB_CUDA_TRY(cudaMemsetAsync(c->xflag, 0, sizeof(int) * (size_t)nx, st));
    FluidCharges fs;
    memset(&fs, 0, sizeof(fs));
    for (size_t f = 0; f < c->fluids.size() && fs.n < HYB_MAX_FLUIDS; ++f) fs.n_[fs.n++] = c->fluids[f].n;
    k_fluid_nonzero<<<node_grid(g), node_block(g), 0, st>>>(g, fs, c->xflag);
    HYB_CUDA_TRY(cudaMemcpyAsync(c->xflag_host, c->xflag, sizeof(int) * (size_t)nx, cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));
    int lo = nx, hi = -1;
    for (int x = 0; x < nx; ++x)
        if (c->xflag_host[x]) {
            lo = std::min(lo, x);
            hi = x;
        }
    if (hi < 0) return clear_fluid_range(c, st);  // no fluid density anywhere
    const int xa = std::max(0, lo - reach), xb = std::min(nx, hi + 1 + reach);
    if ((g.bc[0] == 0 && (lo - reach < 0 || hi + 1 + reach > nx)) || (xa == 0 && xb == nx))
        return clear_fluid_range(c, st);  // nothing to gain (or a periodic range that wraps round)
    c->fluid_xr_host[0] = xa;
    c->fluid_xr_host[1] = xb;
    HYB_CUDA_TRY(cudaMemcpyAsync(c->fluid_xr, c->fluid_xr_host, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));  // the pinned source may change at the next classification
    c->fluid_xr_until = c->step + reach;
    return HYB_OK;
}

hyb_status regime_update(hyb_ctx *c, const float *pm, const float *ps) {
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    const hyb_regime_desc &rd = c->regime;
    uint8_t *raw = c->mask_tmp, *mask = c->mask;
    cudaMemcpyAsync(c->mask_prev, mask, (size_t)g.N, cudaMemcpyDeviceToDevice, st);
    const bool all = rd.policy == HYB_REGIME_ALL_KINETIC;
    const bool physics = !all && (!pm || rd.policy == HYB_REGIME_UNION);
    long long launches = 0;
    const int fG = frame_G(g.T), fG3 = fG * fG * fG;
    if (all) cudaMemsetAsync(raw, 1, (size_t)g.N, st);
    if (physics) {
        unsigned which = 0;
        for (size_t si = 0; si < c->sp.size(); ++si)
            if (c->sp[si].dev.kind == 0 && c->sp[si].q < 0.0 && !c->sp[si].has_zq) which |= 1u << si;
        if (which) {
            const size_t sm1 = sizeof(unsigned long long) * (size_t)fG3;
            k_density_frames<<<g.ntiles, 256, sm1, st>>>(g, c->sp_dev, (int)c->sp.size(), which, 0, c->jscratch,
                                                         c->jvalid, c->status);
            k_density_gather<<<node_grid(g), node_block(g), 0, st>>>(g, c->jscratch, c->jvalid, c->ne);
            launches += 2;
        } else {
            cudaMemsetAsync(c->ne, 0, sizeof(float) * g.N, st);
        }
        int fe = -1;
        for (size_t f = 0; f < c->fluids.size(); ++f)
            if (c->fluids[f].q < 0.0f) {
                fe = (int)f;
                break;
            }
        FluidDev fd;
        memset(&fd, 0, sizeof(fd));
        if (fe >= 0) fd = c->fluids[fe];
        const double lambda = c->desc.lambda_um * 1e-6;
        const float kappa = lambda > 0.0 ? (float)(1.054571817e-34 * 2.0 * M_PI * 299792458.0 / lambda /
                                                   (9.1093837015e-31 * 299792458.0 * 299792458.0))
                                         : 0.0f;
        ++launches;
        k_criterion<<<node_grid(g), node_block(g), 0, st>>>(g, c->E, c->ne, fd, fe >= 0, kappa, (float)rd.a_thr, (float)rd.n_thr,
                                               (float)rd.c_thr, (float)rd.chi_thr, raw);
    }
    if (pm && !all && ++launches) k_decide<<<nblk(g.N), 256, 0, st>>>(g.N, pm, ps, (float)rd.k_sigma, physics ? 1 : 0, raw);
    // Chebyshev dilation: max filters along x, y, z (raw -> mask -> raw -> mask)
    const dim3 db = node_block(g), dg = node_grid(g);
    if (g.n[0] % 4 == 0 && ((uintptr_t)mask & 3) == 0 && ((uintptr_t)raw & 3) == 0) {
        // word-wide: four nodes per thread
        const int nx4 = g.n[0] / 4, b4 = nx4 >= 128 ? 128 : 32 * ((nx4 + 31) / 32);
        const dim3 dg4((unsigned)((nx4 + b4 - 1) / b4), (unsigned)g.n[1], (unsigned)g.n[2]);
        if (rd.dilate <= 4) k_dilate4x<<<dg4, b4, 0, st>>>(g, rd.dilate, (const uint32_t *)raw, (uint32_t *)mask);
        else k_dilate<<<dg, db, 0, st>>>(g, 0, rd.dilate, raw, mask);
        k_dilate4<<<dg4, b4, 0, st>>>(g, 1, rd.dilate, (const uint32_t *)mask, (uint32_t *)raw);
        k_dilate4<<<dg4, b4, 0, st>>>(g, 2, rd.dilate, (const uint32_t *)raw, (uint32_t *)mask);
    } else {
        k_dilate<<<dg, db, 0, st>>>(g, 0, rd.dilate, raw, mask);
        k_dilate<<<dg, db, 0, st>>>(g, 1, rd.dilate, mask, raw);
        k_dilate<<<dg, db, 0, st>>>(g, 2, rd.dilate, raw, mask);
    }
    launches += 3;
    // conversions
    for (size_t f = 0; f < c->fluids.size(); ++f) {
        const int sid = rd.to_species[f];
        if (sid < 0 || sid >= (int)c->sp.size()) continue;
        const SpDev &dst = c->sp[sid].dev;
        // the tiles are compact between steps: new particles go straight into them
        const size_t sm1 = sizeof(unsigned long long) * (size_t)fG3;
        k_fluid_to_particles<<<g.ntiles, 256, sm1, st>>>(g, mask, c->mask_prev, c->fluids[f], dst,
                                                         rd.ppc > 0 ? rd.ppc : 8, rd.quiet ? 1 : 0, c->epoch,
                                                         c->jscratch, c->jvalid, c->status);
        k_rho_gather<<<node_grid(g), node_block(g), 0, st>>>(g, c->jscratch, c->jvalid, c->rho_bg);
        k_clamp_counts<<<(g.ntiles + 255) / 256, 256, 0, st>>>(g.ntiles, dst);
        k_particles_to_fluid<<<g.ntiles, 256, 4 * sm1, st>>>(g, mask, dst, c->jscratch, c->jvalid, c->status);
        k_moments_gather<<<node_grid(g), node_block(g), 0, st>>>(g, c->jscratch, c->jvalid, c->fluids[f]);
        launch_compact(g, dst, st);
        launches += 6;
    }
    c->launches_classify += launches;
    // after an all-kinetic classification that converted every fluid the
    // fluids hold no density and the step leaves their update out (a full-PIC
    // run); any other classification brings it back
    bool idle = all;
    for (size_t f = 0; f < c->fluids.size(); ++f)
        if (rd.to_species[f] < 0 || rd.to_species[f] >= (int)c->sp.size()) idle = false;
    if (idle != c->fluids_idle) {
        c->fluids_idle = idle;
        c->graph_valid = false;
    }
    c->epoch += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("regime update: ") + cudaGetErrorString(e));
    return HYB_OK;
}

}  // namespace hyb
