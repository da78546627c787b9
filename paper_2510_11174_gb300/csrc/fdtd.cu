// Yee FDTD field update, first-order Mur absorbing faces and the Gaussian soft
// laser source (arXiv 2510.11174, Methodology: explicit FDTD solution of
// Maxwell's equations on a uniform grid with a constant Courant-limited dt;
// first-order Mur absorbers storing past boundary values with coefficient
// (c dt - d)/(c dt + d); a Gaussian pulse whose field components get
// temporal and spatial envelopes).
//
// The magnetic update is split into two half steps, so E^n and B^n are
// co-temporal when particles gather them:
//   B^{n+1/2} = B^n - dt/2 curl E^n
//   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2})
//   B^{n+1}   = B^{n+1/2} - dt/2 curl E^{n+1}
// A value at a half-integer position along a non-periodic axis exists for
// index <= n-2 and stays zero otherwise.  Tangential E on a Mur boundary plane
// is set by Mur from the value one node inwards:
//   E_0^{n+1} = E_1^n + ((dt - d)/(dt + d)) (E_1^{n+1} - E_0^n);
// a node on the boundary of two axes (an edge) uses the lower axis and is set
// after the faces, so its inward neighbour is already final.
#include "hyb_internal.cuh"

namespace hyb {

__device__ __forceinline__ bool half_ok(const GridDev &g, int a, int i) {
    return g.bc[a] == 0 || i <= g.n[a] - 2;
}

// bit a set when node (i,j,k) lies on a boundary plane of non-periodic axis a != comp
__device__ __forceinline__ int e_bmask(const GridDev &g, int comp, int i, int j, int k) {
    int m = 0;
    if (comp != 0 && g.bc[0] && (i == 0 || i == g.n[0] - 1)) m |= 1;
    if (comp != 1 && g.bc[1] && (j == 0 || j == g.n[1] - 1)) m |= 2;
    if (comp != 2 && g.bc[2] && (k == 0 || k == g.n[2] - 1)) m |= 4;
    return m;
}

// grid (ceil(nx / blockDim.x), ny, nz): node (i, j, k) from the block and
// thread indices, neighbours as offsets of the linear index (no divisions)
__global__ void k_b_half(GridDev g, const float *__restrict__ E, float *__restrict__ B) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long c = k * sz + j * sy + i;
    const long long oxp = i + 1 == nx ? 1 - nx : 1, oyp = j + 1 == ny ? (1 - ny) * sy : sy,
                    ozp = k + 1 == nz ? (1 - nz) * sz : sz;
    const long long N = g.N;
    const float h = 0.5f * g.dt;
    const float idx = 1.0f / g.d[0], idy = 1.0f / g.d[1], idz = 1.0f / g.d[2];
    const float *Ex = E, *Ey = E + N, *Ez = E + 2 * N;
    const float ex = Ex[c], ey = Ey[c], ez = Ez[c];
    if (half_ok(g, 1, j) && half_ok(g, 2, k)) {
        float cx = (Ez[c + oyp] - ez) * idy - (Ey[c + ozp] - ey) * idz;
        B[c] -= h * cx;
    }
    if (half_ok(g, 0, i) && half_ok(g, 2, k)) {
        float cy = (Ex[c + ozp] - ex) * idz - (Ez[c + oxp] - ez) * idx;
        B[N + c] -= h * cy;
    }
    if (half_ok(g, 0, i) && half_ok(g, 1, j)) {
        float cz = (Ey[c + oxp] - ey) * idx - (Ex[c + oyp] - ex) * idy;
        B[2 * N + c] -= h * cz;
    }
}

__global__ void k_e_yee(GridDev g, float *__restrict__ E, const float *__restrict__ B,
                        const float *__restrict__ J) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long c = k * sz + j * sy + i;
    const long long oxm = i == 0 ? nx - 1 : -1, oym = j == 0 ? (ny - 1) * sy : -sy,
                    ozm = k == 0 ? (nz - 1) * sz : -sz;
    const long long N = g.N;
    const float dt = g.dt;
    const float idx = 1.0f / g.d[0], idy = 1.0f / g.d[1], idz = 1.0f / g.d[2];
    const float *Bx = B, *By = B + N, *Bz = B + 2 * N;
    const float bx = Bx[c], by = By[c], bz = Bz[c];
    if (half_ok(g, 0, i) && e_bmask(g, 0, i, j, k) == 0) {
        float cx = (bz - Bz[c + oym]) * idy - (by - By[c + ozm]) * idz;
        E[c] += dt * (cx - J[c]);
    }
    if (half_ok(g, 1, j) && e_bmask(g, 1, i, j, k) == 0) {
        float cy = (bx - Bx[c + ozm]) * idz - (bz - Bz[c + oxm]) * idx;
        E[N + c] += dt * (cy - J[N + c]);
    }
    if (half_ok(g, 2, k) && e_bmask(g, 2, i, j, k) == 0) {
        float cz = (by - By[c + oxm]) * idx - (bx - Bx[c + oym]) * idy;
        E[2 * N + c] += dt * (cz - J[2 * N + c]);
    }
}

// Mur storage: for axis a, side s (0 low, 1 high), plane p (0 boundary, 1 one node
// inwards), tangential slot cs (the two components != a in increasing order),
// position (u, v) over the two other axes in increasing order.
__device__ __forceinline__ long long mur_slot(int a, int s, int p, int cs, long long plane) {
    return ((((long long)a * 2 + s) * 2 + p) * 2 + cs) * plane;
}

// thread -> (axis, side, slot, u, v) over all Mur planes; returns false if idle
__device__ __forceinline__ bool mur_decode(const GridDev &g, long long t, long long plane, int &a, int &s,
                                           int &cs, int &u, int &v) {
    for (a = 0; a < 3; ++a) {
        if (!g.bc[a]) continue;
        const int au = a == 0 ? 1 : 0, av = a == 2 ? 1 : 2;
        const long long psz = (long long)g.n[au] * g.n[av];
        const long long tot = 4 * psz;
        if (t < tot) {
            s = (int)(t / (2 * psz));
            cs = (int)((t / psz) % 2);
            long long r = t % psz;
            u = (int)(r % g.n[au]);
            v = (int)(r / g.n[au]);
            return true;
        }
        t -= tot;
    }
    (void)plane;
    return false;
}

__global__ void k_mur(GridDev g, float *__restrict__ E, const float *__restrict__ old, long long plane,
                      int phase, long long total) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int a, s, cs, u, v;
    if (!mur_decode(g, t, plane, a, s, cs, u, v)) return;
    const int au = a == 0 ? 1 : 0, av = a == 2 ? 1 : 2;
    const int comp = cs == 0 ? au : av;
    int idx[3];
    idx[a] = s == 0 ? 0 : g.n[a] - 1;
    idx[au] = u;
    idx[av] = v;
    if (!half_ok(g, comp, idx[comp])) return;
    const int m = e_bmask(g, comp, idx[0], idx[1], idx[2]);
    if (__popc(m) != phase) return;
    const int amin = (m & 1) ? 0 : ((m & 2) ? 1 : 2);
    if (amin != a) return;
    int nb[3] = {idx[0], idx[1], idx[2]};
    nb[a] = s == 0 ? 1 : g.n[a] - 2;
    const long long c0 = cidx(g, idx[0], idx[1], idx[2]), c1 = cidx(g, nb[0], nb[1], nb[2]);
    const long long pos = (long long)u + (long long)g.n[au] * v;
    const float e0_old = old[mur_slot(a, s, 0, cs, plane) + pos];
    const float e1_old = old[mur_slot(a, s, 1, cs, plane) + pos];
    const float da = g.d[a];
    const float coef = (g.dt - da) / (g.dt + da);
    float *Ec = E + (long long)comp * g.N;
    Ec[c0] = e1_old + coef * (Ec[c1] - e0_old);
}

__global__ void k_mur_save(GridDev g, const float *__restrict__ E, float *__restrict__ old, long long plane,
                           long long total) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int a, s, cs, u, v;
    if (!mur_decode(g, t, plane, a, s, cs, u, v)) return;
    const int au = a == 0 ? 1 : 0, av = a == 2 ? 1 : 2;
    const int comp = cs == 0 ? au : av;
    const float *Ec = E + (long long)comp * g.N;
    const long long pos = (long long)u + (long long)g.n[au] * v;
    for (int p = 0; p < 2; ++p) {
        int idx[3];
        idx[a] = s == 0 ? p : g.n[a] - 1 - p;
        idx[au] = u;
        idx[av] = v;
        old[mur_slot(a, s, p, cs, plane) + pos] = Ec[cidx(g, idx[0], idx[1], idx[2])];
    }
}

static long long mur_threads(const GridDev &g) {
    long long t = 0;
    for (int a = 0; a < 3; ++a) {
        if (!g.bc[a]) continue;
        const int au = a == 0 ? 1 : 0, av = a == 2 ? 1 : 2;
        t += 4LL * g.n[au] * g.n[av];
    }
    return t;
}

// Soft source: a current sheet J_pol = -2 A(t) f(y, z) / dx on the plane
// x = x_src radiates E_pol = A(t) f towards both sides (normalised units,
// c = 1).  A(t) = a0 exp(-2 ln2 (t - t_peak)^2 / tau^2) sin(t - t_peak) at
// t = (n + 1/2) dt (w0 = 1); tau is the intensity FWHM.  The temporal factor
// is evaluated in FP64, the transverse profile f was built in FP64 on the host.
__global__ void k_laser_source(GridDev g, int x_src, int pol, double a0, double tau, double t_peak,
                               const long long *__restrict__ step_dev, const float *__restrict__ profile,
                               float *__restrict__ J) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int ny = g.n[1], nz = g.n[2];
    if (t >= ny * nz) return;
    const int j = t % ny, k = t / ny;
    if (pol == 1 && !(g.bc[1] == 0 || j <= ny - 2)) return;
    if (pol == 2 && !(g.bc[2] == 0 || k <= nz - 2)) return;
    const double tt = ((double)(*step_dev) + 0.5) * g.dt_d - t_peak;
    const double A = a0 * exp(-2.0 * 0.69314718055994530942 * tt * tt / (tau * tau)) * sin(tt);
    const float val = (float)(-2.0 * A / (double)g.d[0]) * profile[t];
    J[(long long)pol * g.N + cidx(g, x_src, j, k)] += val;
}

static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

void launch_fdtd_b_half(const GridDev &g, const float *E, float *B, cudaStream_t st) {
    k_b_half<<<node_grid(g), node_block(g), 0, st>>>(g, E, B);
}

void launch_fdtd_e(const GridDev &g, float *E, const float *B, const float *J, cudaStream_t st) {
    k_e_yee<<<node_grid(g), node_block(g), 0, st>>>(g, E, B, J);
}

void launch_mur(const GridDev &g, float *E, float *mur_old, long long plane, cudaStream_t st) {
    const long long tot = mur_threads(g);
    if (tot == 0) return;
    k_mur<<<blocks_for(tot, 256), 256, 0, st>>>(g, E, mur_old, plane, 1, tot);
    k_mur<<<blocks_for(tot, 256), 256, 0, st>>>(g, E, mur_old, plane, 2, tot);
    k_mur_save<<<blocks_for(tot, 256), 256, 0, st>>>(g, E, mur_old, plane, tot);
}

void launch_mur_save(const GridDev &g, const float *E, float *mur_old, long long plane, cudaStream_t st) {
    const long long tot = mur_threads(g);
    if (tot == 0) return;
    k_mur_save<<<blocks_for(tot, 256), 256, 0, st>>>(g, E, mur_old, plane, tot);
}

void launch_laser_source(const GridDev &g, const hyb_grid_desc &d, const float *profile,
                         const long long *step_dev, float *J, cudaStream_t st) {
    const int n = g.n[1] * g.n[2];
    k_laser_source<<<blocks_for(n, 256), 256, 0, st>>>(g, d.x_src, d.pol, d.a0, d.tau_fwhm, d.t_peak, step_dev,
                                                        profile, J);
}

}  // namespace hyb

namespace hyb {
__global__ void k_step_inc(long long *step_dev) { *step_dev += 1; }
void launch_step_inc(long long *step_dev, cudaStream_t st) { k_step_inc<<<1, 1, 0, st>>>(step_dev); }
}  // namespace hyb
