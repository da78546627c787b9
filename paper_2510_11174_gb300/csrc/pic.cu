// Particle-in-cell kernels: CIC field gather on the Yee grid, relativistic Boris
// push, move with reflecting walls, and charge-conserving Esirkepov current
// deposition into shared-memory tiles (arXiv 2510.11174, Methodology: PIC
// macro-particles weighted by density-volume fraction, advanced by the Boris
// pusher; particles crossing a domain boundary have their velocity reversed;
// charge conservation is checked at every step).
//
// Data layout: particles of a species live in fixed-capacity tiles of T^3
// cells, SoA FP32 (x, y, z in cell units; u = gamma*beta; weight).  One CTA
// owns one tile: it stages E and B of the tile plus a one-node halo in shared
// memory, pushes every particle of every species in the tile, accumulates J in
// a shared-memory frame of (T+3)^3 nodes (halo 1 below, 2 above, which holds
// every node an Esirkepov stencil of a particle that started in the tile can
// touch) in 64-bit fixed point (frames.cuh), and writes that frame to a
// per-tile scratch slab.  A second kernel sums, for every node, the frames
// that cover it in a fixed order, so J is assembled without global atomics and
// repeats bit for bit whatever order the particles and warps take.
// Particles that left their tile are copied to a migration buffer and
// re-inserted by the rebin kernel; vacated slots are compacted afterwards.
//
// Boris (relativistic, Birdsall & Langdon):
//   u- = u + (q dt/2m) E;  t = (q dt/2m gamma-) B;  s = 2t/(1+t.t)
//   u' = u- + u- x t;  u+ = u- + u' x s;  u_new = u+ + (q dt/2m) E
// Esirkepov, CIC shape, on the 3-node window that holds both shapes:
//   W_x = DS_x (S0_y S0_z + DS_y S0_z/2 + S0_y DS_z/2 + DS_y DS_z/3) (cyclic),
//   J_x(i+1/2) - J_x(i-1/2) = -q w W_x / (dt dy dz).
#include "frames.cuh"
#include "hyb_internal.cuh"
#include "ionize.cuh"
#include "philox.cuh"
#include "qed.cuh"
#include "particles.cuh"

namespace hyb {

// field frame edge: a shape of order k gathers from k nodes below the tile to k - 1 above it
__host__ __device__ constexpr int frame_F(int T, int order = 1) { return T + 2 * order; }

static constexpr int PUSH_THREADS = 256;
static constexpr int PUSH_QCAP = 64;  // per-warp queue of cell-crossing particles

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// the current frame (3 components, 64-bit fixed point), the fields, then the
// per-warp queues (two float4 per entry)
size_t push_smem_bytes(int T, int order) {
    const int F = frame_F(T, order), G = frame_G(T, order);
    return align16(sizeof(unsigned long long) * 3 * (size_t)G * G * G) + align16(sizeof(float) * 6 * (size_t)F * F * F) +
           2 * sizeof(float4) * (PUSH_THREADS / 32) * PUSH_QCAP;
}

// CIC weights of one axis for integer and half-integer staggering, relative to
// the frame origin o (global node index of local 0)
struct AxisW {
    int li, lh;     // local base index (integer / half-integer grid)
    float fi, fh;   // fractional offsets
};

__device__ __forceinline__ AxisW axis_weights(const GridDev &g, int a, float p, int o) {
    AxisW r;
    int i = (int)floorf(p);
    if (g.bc[a] && i > g.n[a] - 2) i = g.n[a] - 2;  // particle on the top wall
    r.li = i - o;
    r.fi = p - (float)i;
    const float s = p - 0.5f;
    const int h = (int)floorf(s);
    r.lh = h - o;
    r.fh = s - (float)h;
    return r;
}

// trilinear interpolation as seven linear interpolations (x, then y, then z)
template <int F>
__device__ __forceinline__ float interp8(const float *__restrict__ f, int bx, int by, int bz, float fx, float fy,
                                         float fz) {
    const float *r00 = f + (bz * F + by) * F + bx;   // rows (y, z), (y + 1, z), (y, z + 1), (y + 1, z + 1)
    const float *r10 = r00 + F, *r01 = r00 + F * F, *r11 = r01 + F;
    const float a00 = fmaf(fx, r00[1] - r00[0], r00[0]);
    const float a10 = fmaf(fx, r10[1] - r10[0], r10[0]);
    const float a01 = fmaf(fx, r01[1] - r01[0], r01[0]);
    const float a11 = fmaf(fx, r11[1] - r11[0], r11[0]);
    const float b0 = fmaf(fy, a10 - a00, a00);
    const float b1 = fmaf(fy, a11 - a01, a01);
    return fmaf(fz, b1 - b0, b0);
}

// Boris (relativistic, Birdsall & Langdon), h = q dt / 2m
__device__ __forceinline__ void boris_push(float h, const float e[3], const float b[3], float u[3]) {
    float um[3], tt[3], ss[3], ud[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) um[c] = u[c] + h * e[c];
    const float gm = sqrtf(1.0f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) tt[c] = h * b[c] * (1.0f / gm);
    const float t2 = tt[0] * tt[0] + tt[1] * tt[1] + tt[2] * tt[2];
    const float s2 = 2.0f / (1.0f + t2);
#pragma unroll
    for (int c = 0; c < 3; ++c) ss[c] = tt[c] * s2;
    ud[0] = um[0] + (um[1] * tt[2] - um[2] * tt[1]);
    ud[1] = um[1] + (um[2] * tt[0] - um[0] * tt[2]);
    ud[2] = um[2] + (um[0] * tt[1] - um[1] * tt[0]);
    u[0] = um[0] + (ud[1] * ss[2] - ud[2] * ss[1]) + h * e[0];
    u[1] = um[1] + (ud[2] * ss[0] - ud[0] * ss[2]) + h * e[1];
    u[2] = um[2] + (ud[0] * ss[1] - ud[1] * ss[0]) + h * e[2];
}

// the implicit rotation of the Vay and Higuera-Cary pushers: w turned about
// tau = h B with the Lorentz factor of the result,
//   gamma^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + (w.tau)^2))) / 2, sigma = 1 + w^2 - tau^2,
//   t = tau / gamma, s = 1 / (1 + t^2), R(w) = s (w + (w.t) t + w x t)
__device__ __forceinline__ void rotate_implicit(const float w[3], const float tau[3], float out[3], float t[3]) {
    const float w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const float tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    const float us = w[0] * tau[0] + w[1] * tau[1] + w[2] * tau[2];
    const float sigma = 1.0f + w2 - tau2;
    const float g = sqrtf(0.5f * (sigma + sqrtf(sigma * sigma + 4.0f * (tau2 + us * us))));
    const float ig = 1.0f / g;
#pragma unroll
    for (int c = 0; c < 3; ++c) t[c] = tau[c] * ig;
    const float s = 1.0f / (1.0f + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const float wt = w[0] * t[0] + w[1] * t[1] + w[2] * t[2];
    out[0] = s * (w[0] + wt * t[0] + (w[1] * t[2] - w[2] * t[1]));
    out[1] = s * (w[1] + wt * t[1] + (w[2] * t[0] - w[0] * t[2]));
    out[2] = s * (w[2] + wt * t[2] + (w[0] * t[1] - w[1] * t[0]));
}

// Vay (Phys. Plasmas 15, 056701, 2008): w = u + h (2E + v x B), u_new = R(w)
__device__ __forceinline__ void vay_push(float h, const float e[3], const float b[3], float u[3]) {
    const float ig = 1.0f / sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const float tau[3] = {h * b[0], h * b[1], h * b[2]};
    const float v[3] = {u[0] * ig, u[1] * ig, u[2] * ig};
    const float w[3] = {u[0] + 2.0f * h * e[0] + (v[1] * tau[2] - v[2] * tau[1]),
                        u[1] + 2.0f * h * e[1] + (v[2] * tau[0] - v[0] * tau[2]),
                        u[2] + 2.0f * h * e[2] + (v[0] * tau[1] - v[1] * tau[0])};
    float t[3];
    rotate_implicit(w, tau, u, t);
}

// Higuera & Cary (Phys. Plasmas 24, 052104, 2017): w = u + h E, u+ = R(w),
// u_new = u+ + h E + u+ x t
__device__ __forceinline__ void higuera_cary_push(float h, const float e[3], const float b[3], float u[3]) {
    const float tau[3] = {h * b[0], h * b[1], h * b[2]};
    const float w[3] = {u[0] + h * e[0], u[1] + h * e[1], u[2] + h * e[2]};
    float up[3], t[3];
    rotate_implicit(w, tau, up, t);
    u[0] = up[0] + h * e[0] + (up[1] * t[2] - up[2] * t[1]);
    u[1] = up[1] + h * e[1] + (up[2] * t[0] - up[0] * t[2]);
    u[2] = up[2] + h * e[2] + (up[0] * t[1] - up[1] * t[0]);
}

__device__ __forceinline__ void shape3(float p, int gbase, float S[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float d = fabsf(p - (float)(gbase + k));
        S[k] = d < 1.0f ? 1.0f - d : 0.0f;
    }
}

// Esirkepov deposit of a particle that stays in its cell.  Per axis the shape
// is (1 - f, f) on the cell's two nodes, f moving from f0 to f1 = f0 + d; W_c
// is nonzero only on the cell's lower c-face, at its 2 x 2 transverse nodes,
// where the transverse factor is the mean of S_p S_q along the straight path:
// with m = (f0 + f1) / 2, int f_p f_q = m_p m_q + d_p d_q / 12 = X, and the
// other three nodes take m_q - X, m_p - X and 1 - m_p - m_q + X.
// fac[c] = q w jfac_c 2^k; the current is fac[c] (S1 - S0)(lower node) = -fac[c] d_c.
template <int G>
__device__ __forceinline__ void deposit_same_cell(unsigned long long *__restrict__ sj, const float x0[3],
                                                  const float x1[3], const int o[3], const float fac[3]) {
    constexpr int G3 = G * G * G;
    int lb[3];
    float m[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c0 = floorf(x0[a]);
        lb[a] = (int)c0 - o[a];
        const float f0 = x0[a] - c0, f1 = x1[a] - c0;
        d[a] = f1 - f0;
        m[a] = 0.5f * (f0 + f1);
    }
    const int base = (lb[2] * G + lb[1]) * G + lb[0];
    constexpr int off[3] = {1, G, G * G};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0f) continue;
        const int pa = (c + 1) % 3, qa = (c + 2) % 3;
        const float X = fmaf(d[pa] * d[qa], 1.0f / 12.0f, m[pa] * m[qa]);
        const float v01 = m[qa] - X, v10 = m[pa] - X;
        const float v00 = (1.0f - m[pa]) - v01;
        const float sc = -fac[c] * d[c];
        unsigned long long *J = sj + c * G3 + base;
        atomicAdd(J, fix_of(sc * v00));
        atomicAdd(J + off[pa], fix_of(sc * v10));
        atomicAdd(J + off[qa], fix_of(sc * v01));
        atomicAdd(J + off[pa] + off[qa], fix_of(sc * X));
    }
}

// Esirkepov deposit on the 3-node window of each axis (a particle that
// crossed a cell face): W_c = DS_c (S0_p S0_q + DS_p S0_q / 2 + S0_p DS_q / 2 +
// DS_p DS_q / 3), prefix-summed along c
template <int G>
__device__ __forceinline__ void deposit_general(unsigned long long *__restrict__ sj, const float x0[3],
                                                const float x1[3], const int o[3], float qw, const float jfac[3]) {
    constexpr int G3 = G * G * G;
    int lb[3];
    float S0[3][3], DS[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i0 = (int)floorf(x0[a]), i1 = (int)floorf(x1[a]);
        const int gb = i0 < i1 ? i0 : i1;
        lb[a] = gb - o[a];
        float S1[3];
        shape3(x0[a], gb, S0[a]);
        shape3(x1[a], gb, S1);
#pragma unroll
        for (int k = 0; k < 3; ++k) DS[a][k] = S1[k] - S0[a][k];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int pa = (c + 1) % 3, qa = (c + 2) % 3;
        const float fac = qw * jfac[c];
        unsigned long long *Jc = sj + c * G3;
#pragma unroll
        for (int bq = 0; bq < 3; ++bq) {
            // transverse factor S0p (S0q + DSq/2) + DSp (S0q/2 + DSq/3)
            const float caq = fmaf(0.5f, DS[qa][bq], S0[qa][bq]);
            const float cbq = fmaf(1.0f / 3.0f, DS[qa][bq], 0.5f * S0[qa][bq]);
#pragma unroll
            for (int bp = 0; bp < 3; ++bp) {
                const float cross = fmaf(DS[pa][bp], cbq, S0[pa][bp] * caq);
                float acc = 0.0f;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    acc += DS[c][a] * cross;
                    if (acc != 0.0f) {
                        int l3[3];
                        l3[c] = lb[c] + a;
                        l3[pa] = lb[pa] + bp;
                        l3[qa] = lb[qa] + bq;
                        atomicAdd(&Jc[(l3[2] * G + l3[1]) * G + l3[0]], fix_of(fac * acc));
                    }
                }
            }
        }
    }
}

// Quadratic (TSC) shape: S(d) = 3/4 - d^2 (|d| <= 1/2), (3/2 - |d|)^2 / 2
// (1/2 <= |d| <= 3/2), 0 beyond
__device__ __forceinline__ float tsc(float d) {
    const float a = fabsf(d);
    const float b = 1.5f - a;
    return a <= 0.5f ? 0.75f - a * a : (a <= 1.5f ? 0.5f * b * b : 0.0f);
}

// TSC weights of one axis around the node nearest to s (staggering already
// removed): local index of the first of the three nodes and their weights
__device__ __forceinline__ void tsc_axis(float s, int o, int &l, float w[3]) {
    const float m = floorf(s + 0.5f);
    const float d = s - m;                 // in [-1/2, 1/2)
    l = (int)m - 1 - o;
    const float a = 0.5f - d, c = 0.5f + d;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - d * d;
    w[2] = 0.5f * c * c;
}

template <int F>
__device__ __forceinline__ float interp27(const float *__restrict__ f, int bx, int by, int bz, const float wx[3],
                                          const float wy[3], const float wz[3]) {
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float row = 0.0f;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float *r = f + ((bz + c) * F + by + b) * F + bx;
            row = fmaf(wy[b], fmaf(wx[2], r[2], fmaf(wx[1], r[1], wx[0] * r[0])), row);
        }
        acc = fmaf(wz[c], row, acc);
    }
    return acc;
}

// Esirkepov with the quadratic shape: per axis the 4-node window holding the
// old and new 3-node supports (base = the smaller nearest node, minus one),
// W as for CIC, prefix-summed over the window's 3 inner faces
template <int G>
__device__ __forceinline__ void deposit_quadratic(unsigned long long *__restrict__ sj, const float x0[3],
                                                  const float x1[3], const int o[3], float qw, const float jfac[3]) {
    constexpr int G3 = G * G * G;
    int lb[3];
    float S0[3][4], DS[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int m0 = (int)floorf(x0[a] + 0.5f), m1 = (int)floorf(x1[a] + 0.5f);
        const int gb = (m0 < m1 ? m0 : m1) - 1;
        lb[a] = gb - o[a];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            S0[a][k] = tsc(x0[a] - (float)(gb + k));
            DS[a][k] = tsc(x1[a] - (float)(gb + k)) - S0[a][k];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int pa = (c + 1) % 3, qa = (c + 2) % 3;
        const float fac = qw * jfac[c];
        unsigned long long *Jc = sj + c * G3;
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) {
            const float caq = fmaf(0.5f, DS[qa][bq], S0[qa][bq]);
            const float cbq = fmaf(1.0f / 3.0f, DS[qa][bq], 0.5f * S0[qa][bq]);
#pragma unroll
            for (int bp = 0; bp < 4; ++bp) {
                const float cross = fmaf(DS[pa][bp], cbq, S0[pa][bp] * caq);
                float acc = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc += DS[c][a] * cross;
                    if (acc != 0.0f) {
                        int l3[3];
                        l3[c] = lb[c] + a;
                        l3[pa] = lb[pa] + bp;
                        l3[qa] = lb[qa] + bq;
                        atomicAdd(&Jc[(l3[2] * G + l3[1]) * G + l3[0]], fix_of(fac * acc));
                    }
                }
            }
        }
    }
}

// One CTA per tile: stage E, B of the tile and a one-node halo, push every
// particle of every species, deposit its current into the tile's fixed-point
// frame, apply the stochastic events, write it back or send it to the
// migration buffer.  Particles that stay in their cell deposit at once;
// particles that crossed a cell face wait in a per-warp queue and are
// deposited 32 at a time with the full 3-node stencil, so that the long
// stencil runs with every lane of the warp busy.
template <int T, int ORDER>
__global__ void __launch_bounds__(PUSH_THREADS, 3) k_push_deposit(GridDev g, const float *__restrict__ E,
                                                                  const float *__restrict__ B,
                                                                  const SpDev *__restrict__ sps, int nsp,
                                                                  float *__restrict__ jscratch,
                                                                  int *__restrict__ jvalid, int *__restrict__ status,
                                                                  const long long *__restrict__ step_dev, QedDev qd) {
    constexpr int F = frame_F(T, ORDER), G = frame_G(T, ORDER);
    constexpr int F3 = F * F * F, G3 = G * G * G;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *sj = reinterpret_cast<unsigned long long *>(smraw);  // 3 current components, G^3 each
    float *sf = reinterpret_cast<float *>(smraw + align16(sizeof(unsigned long long) * 3 * G3));  // 6 x F^3
    float4 *queue = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(sf) + align16(sizeof(float) * 6 * F3));
    __shared__ int s_holes;
    __shared__ int s_qwmax[32];  // per warp: largest |q w| of the tile's particles (float bits)
    __shared__ int s_kfix;       // fixed-point exponent of the tile's current frame
    __shared__ double s_tal_e[NTALLY];
    __shared__ unsigned long long s_tal_n[NTALLY];
    __shared__ SpDev s_sp;       // the species being pushed (its descriptor read once per tile)
    const long long step = *step_dev;
    double tal_e[NTALLY] = {0.0, 0.0, 0.0};
    int tal_n[NTALLY] = {0, 0, 0};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *qa = queue + warp * 2 * PUSH_QCAP;  // (x0, q w) of queued particles
    float4 *qb = qa + PUSH_QCAP;                // (x1, -)

    const int t = blockIdx.x;
    // a tile without particles writes no frame: the reduction skips it
    int total = 0;
    for (int si = 0; si < nsp; ++si) total += min(sps[si].count[t], sps[si].cap);
    if (total == 0) {
        if (threadIdx.x < nsp) {
            sps[threadIdx.x].hole_count[t] = 0;
            sps[threadIdx.x].hole_used[t] = 0;
        }
        if (threadIdx.x == 0) jvalid[t] = 0;
        return;
    }
    // the largest |q w| in the tile bounds every frame sum (fixed-point scale)
    {
        float qwm = 0.0f;
        for (int si = 0; si < nsp; ++si) {
            const SpDev &sp = sps[si];
            const int n = min(sp.count[t], sp.cap);
            const long long base = (long long)t * sp.cap;
            for (int p = threadIdx.x; p < n; p += PUSH_THREADS) {
                const float qp = sp.zq ? sp.q * sp.zq[base + p] : sp.q;
                qwm = fmaxf(qwm, fabsf(qp * sp.w[base + p]));
            }
        }
        block_max_put(qwm, s_qwmax);
    }
    const int tx = t % g.nt[0], ty = (t / g.nt[0]) % g.nt[1], tz = t / (g.nt[0] * g.nt[1]);
    const int o[3] = {tx * T - ORDER, ty * T - ORDER, tz * T - ORDER};  // frame origin
    const long long N = g.N;

    for (int l = threadIdx.x; l < F3; l += PUSH_THREADS) {
        const int lx = l % F, ly = (l / F) % F, lz = l / (F * F);
        int gi[3] = {o[0] + lx, o[1] + ly, o[2] + lz};
        bool in = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (g.bc[a] == 0) {
                gi[a] = gi[a] < 0 ? gi[a] + g.n[a] : (gi[a] >= g.n[a] ? gi[a] - g.n[a] : gi[a]);
            } else if (gi[a] < 0 || gi[a] > g.n[a] - 1) {
                in = false;
            }
        }
        const long long c = in ? cidx(g, gi[0], gi[1], gi[2]) : 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            sf[q * F3 + l] = in ? E[q * N + c] : 0.0f;
            sf[(3 + q) * F3 + l] = in ? B[q * N + c] : 0.0f;
        }
    }
    for (int l = threadIdx.x; l < 3 * G3; l += PUSH_THREADS) sj[l] = 0ULL;
    if (threadIdx.x == 0) {
        s_holes = 0;
        for (int k = 0; k < NTALLY; ++k) {
            s_tal_e[k] = 0.0;
            s_tal_n[k] = 0;
        }
    }
    __syncthreads();

    const float dt = g.dt;
    const float inv_d[3] = {1.0f / g.d[0], 1.0f / g.d[1], 1.0f / g.d[2]};
    // current per unit q w of a face crossing: -1 / (dt dA_c), times the frame's
    // fixed-point scale 2^k (every Esirkepov weight is at most 1 in magnitude,
    // so a node's sum is at most total * max |q w| * max |jfac|)
    const float j0 = -1.0f / (dt * g.d[1] * g.d[2]), j1 = -1.0f / (dt * g.d[0] * g.d[2]),
                j2 = -1.0f / (dt * g.d[0] * g.d[1]);
    const int kfix = fix_exponent((double)total * (double)block_max_read(s_qwmax) *
                                  (double)fmaxf(fabsf(j0), fmaxf(fabsf(j1), fabsf(j2))));
    const float fscale = pow2f(kfix);
    const float jfac[3] = {j0 * fscale, j1 * fscale, j2 * fscale};
    if (threadIdx.x == 0) s_kfix = kfix;  // read back after the species loop's barriers
    const float *sEx = sf, *sEy = sf + F3, *sEz = sf + 2 * F3;
    const float *sBx = sf + 3 * F3, *sBy = sf + 4 * F3, *sBz = sf + 5 * F3;

    for (int si = 0; si < nsp; ++si) {
        {
            // the descriptor to shared memory: the loop reads it for every particle
            const int *src = reinterpret_cast<const int *>(sps + si);
            int *dst = reinterpret_cast<int *>(&s_sp);
            for (int w = threadIdx.x; w < (int)(sizeof(SpDev) / sizeof(int)); w += PUSH_THREADS) dst[w] = src[w];
            __syncthreads();
        }
        const SpDev &sp = s_sp;
        const int n = min(sp.count[t], sp.cap);
        const long long base = (long long)t * sp.cap;
        // times q_p below; photons (m = 0, q = 0) get no Lorentz force
        const float qm_half = sp.kind == 1 ? 0.0f : 0.5f * dt / sp.m;
        int qn = 0;  // entries in this warp's queue (warp-uniform)
        // the next particle's x, y, z, ux, uy, uz, w and charge state, loaded one
        // iteration ahead so that the loads overlap the current particle's work
        float pf[8];
        auto prefetch = [&](int pp) {
            if (pp < n) {
                const long long s2 = base + pp;
                pf[0] = sp.x[s2]; pf[1] = sp.y[s2]; pf[2] = sp.z[s2];
                pf[3] = sp.ux[s2]; pf[4] = sp.uy[s2]; pf[5] = sp.uz[s2];
                pf[6] = sp.w[s2];
                pf[7] = sp.zq ? sp.zq[s2] : 1.0f;
            }
        };
        prefetch(threadIdx.x);
        for (int p0 = 0; p0 < n; p0 += PUSH_THREADS) {
            const int p = p0 + threadIdx.x;
            bool act = p < n;
            const long long s = base + p;
            float x0[3] = {0.0f, 0.0f, 0.0f}, x1[3] = {0.0f, 0.0f, 0.0f}, u[3] = {0.0f, 0.0f, 0.0f};
            float e[3] = {0.0f, 0.0f, 0.0f}, b[3] = {0.0f, 0.0f, 0.0f};
            float wgt = 0.0f, q = 0.0f;
            if (act) {
                x0[0] = pf[0]; x0[1] = pf[1]; x0[2] = pf[2];
                u[0] = pf[3]; u[1] = pf[4]; u[2] = pf[5];
                wgt = pf[6];
                q = sp.q * pf[7];
            }
            prefetch(p + PUSH_THREADS);
            if (act) {
                // every shared-memory index below derives from a cell inside this
                // tile; anything else is flagged and left untouched
                bool inside = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int ci = (int)floorf(x0[a]);
                    if (g.bc[a] && ci == g.n[a] - 1 && x0[a] == (float)(g.n[a] - 1)) ci = g.n[a] - 2;
                    inside = inside && isfinite(x0[a]) && ci >= o[a] + ORDER && ci <= o[a] + ORDER + T - 1 &&
                             (g.bc[a] == 0 || ci <= g.n[a] - 2);
                }
                if (!inside) {
                    atomicOr(status, ST_BADPOS);
                    act = false;
                }
            }
            if (act) {
                // ---- gather E^n, B^n at x^n
                if constexpr (ORDER == 1) {
                    const AxisW ax = axis_weights(g, 0, x0[0], o[0]);
                    const AxisW ay = axis_weights(g, 1, x0[1], o[1]);
                    const AxisW az = axis_weights(g, 2, x0[2], o[2]);
                    e[0] = interp8<F>(sEx, ax.lh, ay.li, az.li, ax.fh, ay.fi, az.fi);
                    e[1] = interp8<F>(sEy, ax.li, ay.lh, az.li, ax.fi, ay.fh, az.fi);
                    e[2] = interp8<F>(sEz, ax.li, ay.li, az.lh, ax.fi, ay.fi, az.fh);
                    b[0] = interp8<F>(sBx, ax.li, ay.lh, az.lh, ax.fi, ay.fh, az.fh);
                    b[1] = interp8<F>(sBy, ax.lh, ay.li, az.lh, ax.fh, ay.fi, az.fh);
                    b[2] = interp8<F>(sBz, ax.lh, ay.lh, az.li, ax.fh, ay.fh, az.fi);
                } else {
                    // quadratic shape: integer (i) and half-integer (h) staggering per axis
                    int li[3], lh[3];
                    float wi[3][3], wh[3][3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        tsc_axis(x0[a], o[a], li[a], wi[a]);
                        tsc_axis(x0[a] - 0.5f, o[a], lh[a], wh[a]);
                    }
                    e[0] = interp27<F>(sEx, lh[0], li[1], li[2], wh[0], wi[1], wi[2]);
                    e[1] = interp27<F>(sEy, li[0], lh[1], li[2], wi[0], wh[1], wi[2]);
                    e[2] = interp27<F>(sEz, li[0], li[1], lh[2], wi[0], wi[1], wh[2]);
                    b[0] = interp27<F>(sBx, li[0], lh[1], lh[2], wi[0], wh[1], wh[2]);
                    b[1] = interp27<F>(sBy, lh[0], li[1], lh[2], wh[0], wi[1], wh[2]);
                    b[2] = interp27<F>(sBz, lh[0], lh[1], li[2], wh[0], wh[1], wi[2]);
                }

                // ---- momentum update (species-uniform choice: no divergence)
                const float h = q * qm_half;
                if (sp.pusher == HYB_PUSH_BORIS) boris_push(h, e, b, u);
                else if (sp.pusher == HYB_PUSH_VAY) vay_push(h, e, b, u);
                else higuera_cary_push(h, e, b, u);

                // ---- move (photons at c: velocity k / |k|), reflect at absorbing walls
                const float gam = sp.kind == 1 ? fmaxf(sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]), 1e-30f)
                                               : sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    x1[a] = x0[a] + u[a] * (dt / gam) * inv_d[a];
                    if (g.bc[a]) {
                        const float L = (float)(g.n[a] - 1);
                        if (x1[a] < 0.0f) { x1[a] = -x1[a]; u[a] = -u[a]; }
                        else if (x1[a] > L) { x1[a] = 2.0f * L - x1[a]; u[a] = -u[a]; }
                    }
                }
                bool finite = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) finite = finite && isfinite(x1[a]) && fabsf(x1[a] - x0[a]) < 1.0f;
                if (!finite) {
                    atomicOr(status, ST_BADPOS);
                    act = false;
                }
            }

            // ---- Esirkepov deposit into the shared frame: particles that stay
            // in their cell now, the others through the warp's queue
            bool same_cell = ORDER == 1;   // the quadratic stencil always takes the queue
#pragma unroll
            for (int a = 0; a < 3; ++a) same_cell = same_cell && floorf(x0[a]) == floorf(x1[a]);
            const bool dep = act && q != 0.0f;
            if (dep && same_cell) {
                const float qw = q * wgt;
                const float fac[3] = {qw * jfac[0], qw * jfac[1], qw * jfac[2]};
                deposit_same_cell<G>(sj, x0, x1, o, fac);
            }
            const unsigned cross = __ballot_sync(0xffffffffu, dep && !same_cell);
            if (dep && !same_cell) {
                const int pos = qn + __popc(cross & ((1u << lane) - 1u));
                qa[pos] = make_float4(x0[0], x0[1], x0[2], q * wgt);
                qb[pos] = make_float4(x1[0], x1[1], x1[2], 0.0f);
            }
            qn += __popc(cross);
            __syncwarp();
            if (qn >= 32) {
                const float4 A = qa[qn - 32 + lane], Bq = qb[qn - 32 + lane];
                const float y0[3] = {A.x, A.y, A.z}, y1[3] = {Bq.x, Bq.y, Bq.z};
                if constexpr (ORDER == 1) deposit_general<G>(sj, y0, y1, o, A.w, jfac);
                else deposit_quadratic<G>(sj, y0, y1, o, A.w, jfac);
                qn -= 32;
                __syncwarp();
            }

            if (act) {
                // ---- periodic image, tile membership, write back or migrate
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (g.bc[a] == 0) {
                        const float L = (float)g.n[a];
                        if (x1[a] < 0.0f) x1[a] += L;
                        else if (x1[a] >= L) x1[a] -= L;
                        if (x1[a] >= L) x1[a] = 0.0f;
                    }
                }
                const int nt = tile_index(g, x1[0], x1[1], x1[2]);

                // ---- stochastic events, after the deposit (this step's current
                // used the pre-event charge and momentum); new particles start at
                // x^{n+1} and enter their species through its migration buffer
                float zq_new = sp.zq ? sp.zq[s] : 0.0f;
                float tau = sp.tau ? sp.tau[s] : 0.0f;
                bool dead = false;
                const uint64_t pid = sp.id[s];
                if (sp.zmax > 0 && zq_new < (float)sp.zmax) {
                    // field ionization: at most one level per step; the electron
                    // takes the ion's u and weight
                    const int Z = (int)zq_new;
                    const float P = ion_probability(sp, Z, sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]));
                    const u32x4 r = philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)step, RNG_IONIZE,
                                                  g.seed, sp.sp_index);
                    if (u01f(r.v[0]) < P) {
                        zq_new = (float)(Z + 1);
                        tal_e[TALLY_IONIZE] += (double)wgt * sp.ip_mc2[Z];
                        tal_n[TALLY_IONIZE] += 1;
                        const SpDev &el = sps[sp.ion_into];
                        const uint64_t eid = (1ULL << 63) | (pid << 3) | (uint64_t)(Z + 1);
                        spawn(el, x1, u, wgt, eid, nt, step, g.seed, -1.0f, status);
                    }
                }
                if (sp.qed) {
                    // photon emission (radiation reaction), optical-depth method
                    const float gl = sqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                    const float chi = qed_chi(qd.kappa, e, b, u, gl);
                    tau -= qd.pref * qed_h(qd, chi) / gl * dt;
                    if (tau <= 0.0f) {
                        const u32x4 r = philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)step,
                                                      RNG_QED_EMIT, g.seed, sp.sp_index);
                        const float xi = qed_em_sample(qd, chi, u01f(r.v[0]));
                        tau = -logf(u01f(r.v[1]));
                        const float eps = fminf(xi * gl, gl - 1.0f);
                        const float g1 = gl - eps;
                        const float un = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                        const float u1 = sqrtf(fmaxf(g1 * g1 - 1.0f, 0.0f));
                        const float sc = un > 0.0f ? u1 / un : 0.0f;
                        float k[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            k[c] = un > 0.0f ? eps * u[c] / un : 0.0f;
                            u[c] *= sc;
                        }
                        tal_n[TALLY_EMIT] += 1;
                        if (eps >= sp.eps_min && sp.ph_species >= 0 && un > 0.0f) {
                            spawn(sps[sp.ph_species], x1, k, wgt, derived_id(pid, step, 2u), nt, step, g.seed,
                                  -logf(u01f(r.v[2])), status);
                        } else {
                            tal_e[TALLY_EMIT] += (double)wgt * eps;
                        }
                    }
                }
                if (sp.kind == 1 && sp.pair_e >= 0) {
                    // Breit-Wheeler pair creation by a photon (energy >= 2 m c^2)
                    const float eps = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                    if (eps >= 2.0f) {
                        const float chi = qed_chi(qd.kappa, e, b, u, eps);
                        tau -= qd.pref * qed_T(qd, chi) / eps * dt;
                        if (tau <= 0.0f) {
                            const u32x4 r = philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)step,
                                                          RNG_QED_PAIR, g.seed, sp.sp_index);
                            const float xi = qed_pair_sample(qd, chi, u01f(r.v[0]));
                            const float ee = xi * eps, ep = (1.0f - xi) * eps;
                            const float ue = ee > 1.0f ? sqrtf(ee * ee - 1.0f) : 0.0f;
                            const float up = ep > 1.0f ? sqrtf(ep * ep - 1.0f) : 0.0f;
                            if (ee < 1.0f) tal_e[TALLY_PAIR] += (double)wgt * (1.0f - ee);
                            if (ep < 1.0f) tal_e[TALLY_PAIR] += (double)wgt * (1.0f - ep);
                            tal_n[TALLY_PAIR] += 1;
                            float ve[3], vp[3];
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                ve[c] = ue * u[c] / eps;
                                vp[c] = up * u[c] / eps;
                            }
                            spawn(sps[sp.pair_e], x1, ve, wgt, derived_id(pid, step, 3u), nt, step, g.seed,
                                  -logf(u01f(r.v[1])), status);
                            spawn(sps[sp.pair_p], x1, vp, wgt, derived_id(pid, step, 5u), nt, step, g.seed,
                                  -logf(u01f(r.v[2])), status);
                            dead = true;
                        }
                    }
                }

                if (nt == t && !dead) {
                    sp.x[s] = x1[0]; sp.y[s] = x1[1]; sp.z[s] = x1[2];
                    sp.ux[s] = u[0]; sp.uy[s] = u[1]; sp.uz[s] = u[2];
                    if (sp.zmax > 0) sp.zq[s] = zq_new;
                    if (sp.tau) sp.tau[s] = tau;
                } else {
                    if (!dead) {
                        const int m = warp_append(sp.mig_count);
                        if (m < sp.mig_cap) {
                            sp.mx[m] = x1[0]; sp.my[m] = x1[1]; sp.mz[m] = x1[2];
                            sp.mux[m] = u[0]; sp.muy[m] = u[1]; sp.muz[m] = u[2];
                            sp.mw[m] = wgt;
                            if (sp.zq) sp.mzq[m] = zq_new;
                            if (sp.tau) sp.mtau[m] = tau;
                            sp.mid[m] = pid;
                            sp.mdest[m] = nt;
                        } else {
                            atomicOr(status, ST_OVERFLOW);
                        }
                    }
                    const int hslot = atomicAdd(&s_holes, 1);
                    sp.holes[base + hslot] = p;
                    sp.x[s] = -1.0f;
                }
            }
        }
        // the warp's queue holds fewer than 32 crossing particles: deposit them
        if (lane < qn) {
            const float4 A = qa[lane], Bq = qb[lane];
            const float y0[3] = {A.x, A.y, A.z}, y1[3] = {Bq.x, Bq.y, Bq.z};
            if constexpr (ORDER == 1) deposit_general<G>(sj, y0, y1, o, A.w, jfac);
            else deposit_quadratic<G>(sj, y0, y1, o, A.w, jfac);
        }
        __syncwarp();
        // per-tile tallies: warp sums, then shared accumulators, then one add per tile
#pragma unroll
        for (int k = 0; k < NTALLY; ++k) {
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                tal_e[k] += __shfl_down_sync(0xffffffffu, tal_e[k], o2);
                tal_n[k] += __shfl_down_sync(0xffffffffu, tal_n[k], o2);
            }
            if ((threadIdx.x & 31) == 0 && tal_n[k] > 0) {
                atomicAdd(&s_tal_e[k], tal_e[k]);
                atomicAdd(&s_tal_n[k], (unsigned long long)tal_n[k]);
            }
            tal_e[k] = 0.0;
            tal_n[k] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            sp.hole_count[t] = s_holes;
            sp.hole_used[t] = 0;
            s_holes = 0;
#pragma unroll
            for (int k = 0; k < NTALLY; ++k) {
                if (s_tal_n[k] > 0) {
                    sp.tal_e[(long long)t * NTALLY + k] += s_tal_e[k];
                    sp.tal_n[(long long)t * NTALLY + k] += s_tal_n[k];
                }
                s_tal_e[k] = 0.0;
                s_tal_n[k] = 0;
            }
        }
        __syncthreads();
    }

    float *dst = jscratch + (long long)t * 3 * G3;
    const float inv_scale = pow2f(-s_kfix);
    for (int l = threadIdx.x; l < 3 * G3; l += PUSH_THREADS) dst[l] = fix_to_float(sj[l], inv_scale);
    if (threadIdx.x == 0) jvalid[t] = 1;
}


// For every node: J = sum of the tile frames that cover it, in a fixed order.
__global__ void k_j_reduce(GridDev g, const float *__restrict__ jscratch, const int *__restrict__ jvalid,
                           float *__restrict__ J) {
    // grid (ceil(nx / blockDim.x), ny, nz)
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long c = ((long long)k * ny + j) * nx + i;
    float acc[3];
    frame_gather<3>(g, jscratch, jvalid, 3, g.order, i, j, k, acc);
    J[c] = acc[0];
    J[g.N + c] = acc[1];
    J[2 * g.N + c] = acc[2];
}

// Insert migrants: into a hole of the destination tile if one is free, else at
// its end.  Grid-stride over the migration buffer (its fill is read on device).
__global__ void k_rebin(SpDev sp, int *__restrict__ status) {
    const int nm = min(*sp.mig_count, sp.mig_cap);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += gridDim.x * blockDim.x) {
        const int t = sp.mdest[m];
        const int h = atomicAdd(&sp.hole_used[t], 1);
        int slot;
        if (h < sp.hole_count[t]) {
            slot = sp.holes[(long long)t * sp.cap + h];
        } else {
            slot = atomicAdd(&sp.count[t], 1);
            if (slot >= sp.cap) {
                atomicOr(status, ST_OVERFLOW);
                continue;
            }
        }
        const long long s = (long long)t * sp.cap + slot;
        sp.x[s] = sp.mx[m]; sp.y[s] = sp.my[m]; sp.z[s] = sp.mz[m];
        sp.ux[s] = sp.mux[m]; sp.uy[s] = sp.muy[m]; sp.uz[s] = sp.muz[m];
        sp.w[s] = sp.mw[m];
        if (sp.zq) sp.zq[s] = sp.mzq[m];
        sp.id[s] = sp.mid[m];
        if (sp.tau) sp.tau[s] = sp.mtau[m];
    }
}

// Close the holes no migrant filled: move live particles from the end of the
// tile into them and shrink the count.
__global__ void __launch_bounds__(32) k_compact(GridDev g, SpDev sp) {
    // one warp per tile: the holes below the new count (in hole-list order)
    // are filled with the live particles at or above it (in slot order), the
    // same pairing as a serial walk of both lists; FIFO queues of up to 64
    // entries in shared memory, refilled 32 candidates at a time
    __shared__ int hq[64], sq[64];
    const int t = blockIdx.x, lane = threadIdx.x;
    (void)g;
    const int hc = sp.hole_count[t], hu = sp.hole_used[t];
    const int n = min(sp.count[t], sp.cap);
    if (hu >= hc) {
        if (lane == 0) {
            sp.count[t] = n;  // an overflowing append left count above the capacity
            if (2 * n > sp.cap) atomicOr(sp.fill_flags, 1 << sp.sp_index);
        }
        return;
    }
    const long long base = (long long)t * sp.cap;
    const int new_n = n - (hc - hu);
    const unsigned below = (1u << lane) - 1u;
    int h = hu, src = new_n, hn = 0, sn = 0;
    for (;;) {
        while (hn < 32 && h < hc) {
            const int hh = h + lane;
            const int dst = hh < hc ? sp.holes[base + hh] : new_n;
            const bool ok = dst < new_n;  // holes at or above new_n vanish with the shrink
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) hq[hn + __popc(m & below)] = dst;
            hn += __popc(m);
            h += 32;
        }
        while (sn < 32 && src < n) {
            const int s0 = src + lane;
            const bool ok = s0 < n && !(sp.x[base + s0] < 0.0f);  // live slot (vacated slots hold x < 0)
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) sq[sn + __popc(m & below)] = s0;
            sn += __popc(m);
            src += 32;
        }
        __syncwarp();
        const int k = min(32, min(hn, sn));  // one pair per lane
        if (k == 0) break;
        if (lane < k) {
            const long long a = base + hq[lane], b = base + sq[lane];
            sp.x[a] = sp.x[b]; sp.y[a] = sp.y[b]; sp.z[a] = sp.z[b];
            sp.ux[a] = sp.ux[b]; sp.uy[a] = sp.uy[b]; sp.uz[a] = sp.uz[b];
            sp.w[a] = sp.w[b];
            if (sp.zq) sp.zq[a] = sp.zq[b];
            sp.id[a] = sp.id[b];
            if (sp.tau) sp.tau[a] = sp.tau[b];
        }
        // drop the k used entries of both queues
        const int h0 = lane + k < hn ? hq[lane + k] : 0, h1 = lane + 32 + k < hn ? hq[lane + 32 + k] : 0;
        const int q0 = lane + k < sn ? sq[lane + k] : 0, q1 = lane + 32 + k < sn ? sq[lane + 32 + k] : 0;
        __syncwarp();
        if (lane + k < hn) hq[lane] = h0;
        if (lane + 32 + k < hn) hq[lane + 32] = h1;
        if (lane + k < sn) sq[lane] = q0;
        if (lane + 32 + k < sn) sq[lane + 32] = q1;
        hn -= k;
        sn -= k;
        __syncwarp();
    }
    if (lane == 0) {
        sp.count[t] = new_n;
        sp.hole_count[t] = 0;
        sp.hole_used[t] = 0;
        if (2 * new_n > sp.cap) atomicOr(sp.fill_flags, 1 << sp.sp_index);
    }
}

// copy every tile's live slots into a species layout with a larger capacity
__global__ void k_regrid(SpDev from, SpDev to) {
    const int t = blockIdx.x;
    const int n = min(from.count[t], from.cap);
    const long long a = (long long)t * from.cap, b = (long long)t * to.cap;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        to.x[b + p] = from.x[a + p]; to.y[b + p] = from.y[a + p]; to.z[b + p] = from.z[a + p];
        to.ux[b + p] = from.ux[a + p]; to.uy[b + p] = from.uy[a + p]; to.uz[b + p] = from.uz[a + p];
        to.w[b + p] = from.w[a + p];
        if (from.zq) to.zq[b + p] = from.zq[a + p];
        if (from.tau) to.tau[b + p] = from.tau[a + p];
        to.id[b + p] = from.id[a + p];
    }
}

__global__ void k_count_tiles(GridDev g, long long n, const float *__restrict__ x, const float *__restrict__ y,
                              const float *__restrict__ z, int *__restrict__ counts) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        atomicAdd(&counts[tile_index(g, x[p], y[p], z[p])], 1);
}

__global__ void k_bin(GridDev g, SpDev sp, long long n, const float *__restrict__ x, const float *__restrict__ y,
                      const float *__restrict__ z, const float *__restrict__ ux, const float *__restrict__ uy,
                      const float *__restrict__ uz, const float *__restrict__ w, const float *__restrict__ zq,
                      const uint64_t *__restrict__ ids, const float *__restrict__ tau, int *__restrict__ status) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int t = tile_index(g, x[p], y[p], z[p]);
        const int slot = atomicAdd(&sp.count[t], 1);
        if (slot >= sp.cap) {
            atomicOr(status, ST_OVERFLOW);
            continue;
        }
        const long long s = (long long)t * sp.cap + slot;
        sp.x[s] = x[p]; sp.y[s] = y[p]; sp.z[s] = z[p];
        sp.ux[s] = ux[p]; sp.uy[s] = uy[p]; sp.uz[s] = uz[p];
        sp.w[s] = w[p];
        if (sp.zq) sp.zq[s] = zq ? zq[p] : 0.0f;
        sp.id[s] = ids ? ids[p] : (uint64_t)p;
        if (sp.tau) sp.tau[s] = tau ? tau[p] : tau_initial(sp.id[s], g.seed, sp.tau_index);
    }
}

// the live slots of every tile, tile after tile, into contiguous arrays
// (offsets: exclusive prefix sum of the tile counts); zq / tau / the outputs
// for them may be null
__global__ void k_tiles_to_arrays(SpDev sp, const long long *__restrict__ offsets, float *__restrict__ x,
                                  float *__restrict__ y, float *__restrict__ z, float *__restrict__ ux,
                                  float *__restrict__ uy, float *__restrict__ uz, float *__restrict__ w,
                                  float *__restrict__ zq, float *__restrict__ tau, uint64_t *__restrict__ ids) {
    const int t = blockIdx.x;
    const int n = min(sp.count[t], sp.cap);
    const long long a = (long long)t * sp.cap, b = offsets[t];
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        x[b + p] = sp.x[a + p]; y[b + p] = sp.y[a + p]; z[b + p] = sp.z[a + p];
        ux[b + p] = sp.ux[a + p]; uy[b + p] = sp.uy[a + p]; uz[b + p] = sp.uz[a + p];
        w[b + p] = sp.w[a + p];
        if (zq && sp.zq) zq[b + p] = sp.zq[a + p];
        if (tau && sp.tau) tau[b + p] = sp.tau[a + p];
        ids[b + p] = sp.id[a + p];
    }
}

static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

void launch_push_deposit(const GridDev &g, const float *E, const float *B, const SpDev *sps_dev, int nsp,
                         const QedDev &qd, float *jscratch, int *jvalid, int *status, const long long *step_dev,
                         cudaStream_t st) {
    const size_t smem = push_smem_bytes(g.T, g.order);
    // opt in to more than 48 KB of dynamic shared memory, once per instance
    static bool set[4] = {false, false, false, false};
    auto launch = [&](auto kern, int slot) {
        if (!set[slot]) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            set[slot] = true;
        }
        kern<<<g.ntiles, PUSH_THREADS, smem, st>>>(g, E, B, sps_dev, nsp, jscratch, jvalid, status, step_dev, qd);
    };
    if (g.order == 2) {
        if (g.T == 8) launch(k_push_deposit<8, 2>, 2);
        else launch(k_push_deposit<4, 2>, 3);
    } else {
        if (g.T == 8) launch(k_push_deposit<8, 1>, 0);
        else launch(k_push_deposit<4, 1>, 1);
    }
}

void launch_j_reduce(const GridDev &g, const float *jscratch, const int *jvalid, float *J, cudaStream_t st) {
    const int bx = g.n[0] >= 128 ? 128 : 32 * ((g.n[0] + 31) / 32);
    const dim3 grid((unsigned)((g.n[0] + bx - 1) / bx), (unsigned)g.n[1], (unsigned)g.n[2]);
    k_j_reduce<<<grid, bx, 0, st>>>(g, jscratch, jvalid, J);
}

void launch_rebin(const GridDev &g, const SpDev &s, int *status, cudaStream_t st) {
    (void)g;
    k_rebin<<<152 * 4, 256, 0, st>>>(s, status);
}

void launch_regrid(const GridDev &g, const SpDev &from, const SpDev &to, cudaStream_t st) {
    k_regrid<<<g.ntiles, 256, 0, st>>>(from, to);
}

void launch_compact(const GridDev &g, const SpDev &s, cudaStream_t st) {
    k_compact<<<g.ntiles, 32, 0, st>>>(g, s);
}

void launch_count_tiles(const GridDev &g, long long n, const float *x, const float *y, const float *z,
                        int *counts, cudaStream_t st) {
    if (n == 0) return;
    k_count_tiles<<<min(blocks_for(n, 256), 152u * 16u), 256, 0, st>>>(g, n, x, y, z, counts);
}

void launch_bin_particles(const GridDev &g, const SpDev &s, long long n, const float *x, const float *y,
                          const float *z, const float *ux, const float *uy, const float *uz, const float *w,
                          const float *zq, const uint64_t *ids, const float *tau, int *status, cudaStream_t st) {
    if (n == 0) return;
    k_bin<<<min(blocks_for(n, 256), 152u * 16u), 256, 0, st>>>(g, s, n, x, y, z, ux, uy, uz, w, zq, ids, tau,
                                                               status);
}

void launch_tiles_to_arrays(const GridDev &g, const SpDev &s, const long long *offsets, float *x, float *y, float *z,
                            float *ux, float *uy, float *uz, float *w, float *zq, float *tau, uint64_t *ids,
                            cudaStream_t st) {
    k_tiles_to_arrays<<<g.ntiles, 256, 0, st>>>(s, offsets, x, y, z, ux, uy, uz, w, zq, tau, ids);
}

}  // namespace hyb
