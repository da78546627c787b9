// Cold relativistic fluid on the nodes (arXiv 2510.11174, Methodology: fluid
// continuity and momentum equations with relativistic gamma factors for the
// bulk plasma in stable regions; clamping against numerical instability).
//
//   dn/dt + div(n v) = 0,   d(n u)/dt + div(n u v) = (q/m) n (E + v x B)
//
// Two kernels per fluid and step:
//  1. k_fluid_lorentz: at every node, E and B averaged from their Yee
//     positions, u* = Boris(u; E, B); a warm fluid (p = K n^Gamma) also takes
//     u* -= dt (P(i+1/2) - P(i-1/2)) / (d m n) per axis, P the mean of the two
//     nodes' p on inner faces and the node's own p on the outer face of an
//     absorbing axis; u* and a copy of n go to scratch.
//  2. k_fluid_update: donor-cell transport on the node control volumes; the
//     flux through the face between nodes i and i+1 along axis a uses the
//     mean face velocity s = (v*_a(i) + v*_a(i+1))/2 and the upwind node:
//       F = max(s,0) n_i + min(s,0) n_{i+1},  G = the same with n u*,
//     n^{n+1} = n - dt sum (F+ - F-)/d,  (n u)^{n+1} = n u* - dt sum (G+ - G-)/d;
//     each node adds q F of its upper faces to J (the face of the node control
//     volume is the Yee edge of E_a, so continuity holds exactly with rho = q n);
//     negative densities are clamped to 0 and counted, u = 0 below n_floor.
// Outer faces of absorbing axes carry no flux.
#include "hyb_internal.cuh"

namespace hyb {

// all fluids of a context in one launch (they share E, B and J)
struct FluidSet {
    FluidDev f[HYB_MAX_FLUIDS];
    int n;
};

// index of the lower neighbour along an axis: wrapped on periodic axes, -1
// (outside: zero field, closed face) on absorbing ones
__device__ __forceinline__ int lower_nb(int i, int n, int periodic) { return i > 0 ? i - 1 : (periodic ? n - 1 : -1); }
__device__ __forceinline__ int upper_nb(int i, int n, int periodic) { return i < n - 1 ? i + 1 : (periodic ? 0 : -1); }

// node plane i outside the x-range [xr[0], xr[1]) that a classification with a
// reach set (xr[1] <= xr[0]: every plane counts as inside).  Outside it every
// fluid is empty (n = 0, u = 0) and stays so until the range lapses: each face
// there joins two empty nodes and carries no flux whatever their u*
__device__ __forceinline__ bool outside_range(const int *__restrict__ xr, int i) {
    const int lo = __ldg(xr), hi = __ldg(xr + 1);
    return hi > lo && (i < lo || i >= hi);
}

// grid: (ceil(nx / blockDim.x), ny, nz); one thread per node
__global__ void __launch_bounds__(128) k_fluid_lorentz(GridDev g, const float *__restrict__ E,
                                                       const float *__restrict__ B, FluidSet fs,
                                                       const int *__restrict__ xr) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx || outside_range(xr, i)) return;
    const int im = lower_nb(i, nx, g.bc[0] == 0), jm = lower_nb(j, ny, g.bc[1] == 0),
              km = lower_nb(k, nz, g.bc[2] == 0);
    const long long N = g.N;
    auto at = [&](const float *F, int a, int b, int c) -> float {
        return (a < 0 || b < 0 || c < 0) ? 0.0f : __ldg(F + ((long long)c * ny + b) * nx + a);
    };
    const float *Ex = E, *Ey = E + N, *Ez = E + 2 * N, *Bx = B, *By = B + N, *Bz = B + 2 * N;
    float e[3], b[3];
    e[0] = 0.5f * (at(Ex, im, j, k) + at(Ex, i, j, k));
    e[1] = 0.5f * (at(Ey, i, jm, k) + at(Ey, i, j, k));
    e[2] = 0.5f * (at(Ez, i, j, km) + at(Ez, i, j, k));
    b[0] = 0.25f * (at(Bx, i, jm, km) + at(Bx, i, j, km) + at(Bx, i, jm, k) + at(Bx, i, j, k));
    b[1] = 0.25f * (at(By, im, j, km) + at(By, i, j, km) + at(By, im, j, k) + at(By, i, j, k));
    b[2] = 0.25f * (at(Bz, im, jm, k) + at(Bz, i, jm, k) + at(Bz, im, j, k) + at(Bz, i, j, k));
    const long long c = ((long long)k * ny + j) * nx + i;
    for (int q = 0; q < fs.n; ++q) {
        const FluidDev &f = fs.f[q];
        const float h = f.q * 0.5f * g.dt / f.m;
        float um[3], tt[3], ss[3], ud[3];
        const float u0[3] = {f.ux[c], f.uy[c], f.uz[c]};
#pragma unroll
        for (int a = 0; a < 3; ++a) um[a] = u0[a] + h * e[a];
        const float gm = sqrtf(1.0f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) tt[a] = h * b[a] * (1.0f / gm);
        const float t2 = tt[0] * tt[0] + tt[1] * tt[1] + tt[2] * tt[2];
        const float s2 = 2.0f / (1.0f + t2);
#pragma unroll
        for (int a = 0; a < 3; ++a) ss[a] = tt[a] * s2;
        ud[0] = um[0] + (um[1] * tt[2] - um[2] * tt[1]);
        ud[1] = um[1] + (um[2] * tt[0] - um[0] * tt[2]);
        ud[2] = um[2] + (um[0] * tt[1] - um[1] * tt[0]);
        float us[3] = {um[0] + (ud[1] * ss[2] - ud[2] * ss[1]) + h * e[0],
                       um[1] + (ud[2] * ss[0] - ud[0] * ss[2]) + h * e[1],
                       um[2] + (ud[0] * ss[1] - ud[1] * ss[0]) + h * e[2]};
        const float nc = f.n[c];
        if (f.pK > 0.0f && nc > f.n_floor) {
            // adiabatic pressure force, central face pressures, walls reflect
            auto pr = [&](float n) { return n > 0.0f ? f.pK * powf(n, f.pgam) : 0.0f; };
            const float pc = pr(nc);
            const int lo[3] = {im, jm, km};
            const int hi[3] = {upper_nb(i, nx, g.bc[0] == 0), upper_nb(j, ny, g.bc[1] == 0),
                               upper_nb(k, nz, g.bc[2] == 0)};
            const long long st[3] = {1, nx, (long long)nx * ny};
            const int idx[3] = {i, j, k};
            const float coef = g.dt / (f.m * nc);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float plo = lo[a] < 0 ? pc : 0.5f * (pc + pr(f.n[c + (lo[a] - idx[a]) * st[a]]));
                const float phi = hi[a] < 0 ? pc : 0.5f * (pc + pr(f.n[c + (hi[a] - idx[a]) * st[a]]));
                us[a] -= coef * (phi - plo) / g.d[a];
            }
        }
        f.usx[c] = us[0];
        f.usy[c] = us[1];
        f.usz[c] = us[2];
        f.ns[c] = nc;
    }
}

__global__ void __launch_bounds__(128) k_fluid_update(GridDev g, FluidSet fs, float *__restrict__ J,
                                                      const int *__restrict__ xr) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx || outside_range(xr, i)) return;
    const int idx[3] = {i, j, k};
    // neighbour nodes (lower, upper) per axis; -1 = closed outer face
    int nbi[3][2];
    nbi[0][0] = lower_nb(i, nx, g.bc[0] == 0);
    nbi[0][1] = upper_nb(i, nx, g.bc[0] == 0);
    nbi[1][0] = lower_nb(j, ny, g.bc[1] == 0);
    nbi[1][1] = upper_nb(j, ny, g.bc[1] == 0);
    nbi[2][0] = lower_nb(k, nz, g.bc[2] == 0);
    nbi[2][1] = upper_nb(k, nz, g.bc[2] == 0);
    const long long c = ((long long)k * ny + j) * nx + i;
    const float inv_d[3] = {1.0f / g.d[0], 1.0f / g.d[1], 1.0f / g.d[2]};
    float jf[3] = {0.0f, 0.0f, 0.0f};
    for (int q = 0; q < fs.n; ++q) {
        const FluidDev &f = fs.f[q];
        const float n0 = f.ns[c];
        const float u0[3] = {f.usx[c], f.usy[c], f.usz[c]};
        const float ig0 = rsqrtf(1.0f + u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2]);  // 1 / gamma
        float dn = 0.0f, dm[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ida = inv_d[a];
            // upper face (c, c+1) and lower face (c-1, c)
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int nbv = nbi[a][side == 0 ? 1 : 0];
                if (nbv < 0) continue;  // closed outer face
                int nb[3] = {idx[0], idx[1], idx[2]};
                nb[a] = nbv;
                const long long c1 = ((long long)nb[2] * ny + nb[1]) * nx + nb[0];
                const float n1 = f.ns[c1];
                const float u1[3] = {f.usx[c1], f.usy[c1], f.usz[c1]};
                const float ig1 = rsqrtf(1.0f + u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
                // nodes (lo, hi) of the face, in increasing index order
                const float nlo = side == 0 ? n0 : n1, nhi = side == 0 ? n1 : n0;
                const float v0 = u0[a] * ig0, v1 = u1[a] * ig1;
                const float vlo = side == 0 ? v0 : v1, vhi = side == 0 ? v1 : v0;
                const float s = 0.5f * (vlo + vhi);
                const float sp = fmaxf(s, 0.0f), sm = fminf(s, 0.0f);
                const float F = sp * nlo + sm * nhi;
                const float sgn = side == 0 ? -1.0f : 1.0f;  // out through the upper face, in through the lower
                dn += sgn * F * ida;
#pragma unroll
                for (int b2 = 0; b2 < 3; ++b2) {
                    const float ulo = side == 0 ? u0[b2] : u1[b2], uhi = side == 0 ? u1[b2] : u0[b2];
                    dm[b2] += sgn * (sp * nlo * ulo + sm * nhi * uhi) * ida;
                }
                if (side == 0) jf[a] += f.q * F;
            }
        }
        const float n1 = n0 + g.dt * dn;
        float mom[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) mom[a] = n0 * u0[a] + g.dt * dm[a];
        if (n1 < 0.0f) atomicAdd(f.clamped, 1ULL);
        f.n[c] = fmaxf(n1, 0.0f);
        const bool keep = n1 > f.n_floor;
        const float in1 = keep ? 1.0f / n1 : 0.0f;
        f.ux[c] = mom[0] * in1;
        f.uy[c] = mom[1] * in1;
        f.uz[c] = mom[2] * in1;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (fs.n > 0) J[(long long)a * g.N + c] += jf[a];
}

static constexpr int FB = 256;

__global__ void __launch_bounds__(FB) k_fluid_energy(GridDev g, FluidDev f, double *__restrict__ p_w,
                                                     double *__restrict__ p_n, int nblocks) {
    __shared__ double sh[FB];
    // double-float sums of n (gamma - 1) and n; m and dV applied to the block sums
    ff sw = {0.0f, 0.0f}, sn = {0.0f, 0.0f};
    for (long long c = blockIdx.x * (long long)FB + threadIdx.x; c < g.N; c += (long long)nblocks * FB) {
        const float n = f.n[c];
        sw = ff_add(sw, ff_mulf(ff_gamma_minus_one(ff_u2(f.ux[c], f.uy[c], f.uz[c])), n));
        sn = ff_add(sn, ff{n, 0.0f});
    }
    const double aw = ff_to_double(sw), an = ff_to_double(sn);
    const double dV = g.dd[0] * g.dd[1] * g.dd[2];
    for (int q = 0; q < 2; ++q) {
        sh[threadIdx.x] = q == 0 ? aw : an;
        __syncthreads();
        for (int s = FB / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) (q == 0 ? p_w : p_n)[blockIdx.x] = q == 0 ? sh[0] * f.m_d * dV : sh[0] * dV;
        __syncthreads();
    }
}

void launch_fluids(const GridDev &g, const float *E, const float *B, const FluidDev *f, int nf, float *J,
                   const int *xr, cudaStream_t st) {
    FluidSet fs;
    memset(&fs, 0, sizeof(fs));
    fs.n = nf < HYB_MAX_FLUIDS ? nf : HYB_MAX_FLUIDS;
    for (int q = 0; q < fs.n; ++q) fs.f[q] = f[q];
    const int bx = g.n[0] >= 128 ? 128 : 32 * ((g.n[0] + 31) / 32);
    const dim3 grid((unsigned)((g.n[0] + bx - 1) / bx), (unsigned)g.n[1], (unsigned)g.n[2]);
    k_fluid_lorentz<<<grid, bx, 0, st>>>(g, E, B, fs, xr);
    k_fluid_update<<<grid, bx, 0, st>>>(g, fs, J, xr);
}

void launch_fluid_energy(const GridDev &g, const FluidDev &f, double *p_w, double *p_n, int nblocks,
                         cudaStream_t st) {
    k_fluid_energy<<<nblocks, FB, 0, st>>>(g, f, p_w, p_n, nblocks);
}

}  // namespace hyb
