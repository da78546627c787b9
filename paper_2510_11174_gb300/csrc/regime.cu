// Regime switching: the physics criterion (or the classifier's decision), the
// dilated mask, and the charge-exact fluid <-> particle conversions
// (arXiv 2510.11174, Methodology: fluid models in stable regions, PIC where
// the learned switch flags instability; charge and energy checked during
// regime switches).  The paper does not define the criterion; the reading is
// stated with hyb_regime_desc in include/hyb.h.
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

// electron density from the macro-particles (CIC, node arrays)
__global__ void k_density(GridDev g, SpDev sp, float scale, float *__restrict__ ne) {
    const int t = blockIdx.x;
    const int n = min(sp.count[t], sp.cap);
    const long long base = (long long)t * sp.cap;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const float pos[3] = {sp.x[base + p], sp.y[base + p], sp.z[base + p]};
        const float val = scale * sp.w[base + p];
        int b[3];
        float f[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floorf(pos[a]);
            if (g.bc[a] && i > g.n[a] - 2) i = g.n[a] - 2;
            b[a] = i;
            f[a] = pos[a] - (float)i;
        }
        for (int c = 0; c < 8; ++c) {
            int q[3] = {b[0] + (c & 1), b[1] + ((c >> 1) & 1), b[2] + (c >> 2)};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                if (g.bc[a] == 0) q[a] = q[a] >= g.n[a] ? q[a] - g.n[a] : q[a];
                else if (q[a] > g.n[a] - 1) ok = false;
            }
            if (!ok) continue;
            const float wgt = ((c & 1) ? f[0] : 1.0f - f[0]) * (((c >> 1) & 1) ? f[1] : 1.0f - f[1]) *
                              ((c >> 2) ? f[2] : 1.0f - f[2]);
            atomicAdd(&ne[cidx(g, q[0], q[1], q[2])], wgt * val);
        }
    }
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
    uint8_t m = 0;
    for (int d = -r; d <= r && !m; ++d) {
        int q = i0 + d;
        if (g.bc[a] == 0) q = r < n ? (q < 0 ? q + n : (q >= n ? q - n : q)) : ((q % n) + n) % n;
        else if (q < 0 || q > n - 1) continue;
        m = in[c + (q - i0) * st];
    }
    out[c] = m;
}

// fluid -> particles at kinetic nodes; rho_bg takes (removed fluid charge) -
// (CIC charge of the new particles)
__global__ void k_fluid_to_particles(GridDev g, const uint8_t *__restrict__ mask, const uint8_t *__restrict__ prev,
                                     FluidDev f, SpDev dst, int ppc, uint32_t epoch, float *__restrict__ rho_bg,
                                     int *__restrict__ status) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    // only nodes that switch to kinetic now: fluid that flows into a node
    // that was kinetic already stays fluid there
    if (!mask[c] || prev[c] || !(f.n[c] > f.n_floor)) return;
    const int nx = g.n[0], ny = g.n[1];
    const int idx[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
    const float dV = g.d[0] * g.d[1] * g.d[2];
    const float n = f.n[c];
    const float w = n * dV / (float)ppc;
    atomicAdd(&rho_bg[c], f.q * n);
    const float u[3] = {f.ux[c], f.uy[c], f.uz[c]};
    for (int p = 0; p < ppc; ++p) {
        const u32x4 r = philox4x32_10((uint32_t)c, epoch, (uint32_t)p, 6u, g.seed, dst.sp_index);
        float pos[3];
        for (int a = 0; a < 3; ++a) {
            float lo = (float)idx[a] - 0.5f, hi = (float)idx[a] + 0.5f;
            if (g.bc[a]) {
                lo = fmaxf(lo, 0.0f);
                hi = fminf(hi, (float)(g.n[a] - 1));
            }
            pos[a] = lo + (hi - lo) * u01f(r.v[a]);
            if (g.bc[a] == 0) {
                if (pos[a] < 0.0f) pos[a] += (float)g.n[a];
                if (pos[a] >= (float)g.n[a]) pos[a] -= (float)g.n[a];
                if (pos[a] >= (float)g.n[a]) pos[a] = 0.0f;
            }
        }
        // CIC charge of the new particle leaves rho_bg
        int b[3];
        float fr[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floorf(pos[a]);
            if (g.bc[a] && i > g.n[a] - 2) i = g.n[a] - 2;
            b[a] = i;
            fr[a] = pos[a] - (float)i;
        }
        for (int k8 = 0; k8 < 8; ++k8) {
            int q[3] = {b[0] + (k8 & 1), b[1] + ((k8 >> 1) & 1), b[2] + (k8 >> 2)};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                if (g.bc[a] == 0) q[a] = q[a] >= g.n[a] ? q[a] - g.n[a] : q[a];
                else if (q[a] > g.n[a] - 1) ok = false;
            }
            if (!ok) continue;
            const float wgt = ((k8 & 1) ? fr[0] : 1.0f - fr[0]) * (((k8 >> 1) & 1) ? fr[1] : 1.0f - fr[1]) *
                              ((k8 >> 2) ? fr[2] : 1.0f - fr[2]);
            atomicAdd(&rho_bg[cidx(g, q[0], q[1], q[2])], -dst.q * w / dV * wgt);
        }
        const uint64_t id = (1ULL << 62) | (derived_id((uint64_t)c | ((uint64_t)epoch << 40), p, 6u) >> 2);
        const float tau = dst.tau ? tau_initial(id, g.seed, dst.tau_index) : 0.0f;
        tile_put(dst, tile_index(g, pos[0], pos[1], pos[2]), pos, u, w, id, tau, status);
    }
    f.n[c] = 0.0f;
    f.ux[c] = f.uy[c] = f.uz[c] = 0.0f;
}

__global__ void k_mom_init(long long N, FluidDev f) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    f.usx[c] = f.n[c] * f.ux[c];
    f.usy[c] = f.n[c] * f.uy[c];
    f.usz[c] = f.n[c] * f.uz[c];
}

// particles whose nearest node is fluid: CIC-deposit n and n u, then remove
__global__ void k_particles_to_fluid(GridDev g, const uint8_t *__restrict__ mask, SpDev sp, FluidDev f) {
    __shared__ int s_holes;
    const int t = blockIdx.x;
    if (threadIdx.x == 0) s_holes = 0;
    __syncthreads();
    const int n = min(sp.count[t], sp.cap);
    const long long base = (long long)t * sp.cap;
    const float idV = 1.0f / (g.d[0] * g.d[1] * g.d[2]);
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const long long s = base + p;
        const float pos[3] = {sp.x[s], sp.y[s], sp.z[s]};
        int nd[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floorf(pos[a] + 0.5f);
            if (g.bc[a] == 0) i = i >= g.n[a] ? i - g.n[a] : i;
            else if (i > g.n[a] - 1) i = g.n[a] - 1;
            nd[a] = i;
        }
        if (mask[cidx(g, nd[0], nd[1], nd[2])]) continue;
        const float wn = sp.w[s] * idV;
        const float u[3] = {sp.ux[s], sp.uy[s], sp.uz[s]};
        int b[3];
        float fr[3];
        for (int a = 0; a < 3; ++a) {
            int i = (int)floorf(pos[a]);
            if (g.bc[a] && i > g.n[a] - 2) i = g.n[a] - 2;
            b[a] = i;
            fr[a] = pos[a] - (float)i;
        }
        for (int k8 = 0; k8 < 8; ++k8) {
            int q[3] = {b[0] + (k8 & 1), b[1] + ((k8 >> 1) & 1), b[2] + (k8 >> 2)};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                if (g.bc[a] == 0) q[a] = q[a] >= g.n[a] ? q[a] - g.n[a] : q[a];
                else if (q[a] > g.n[a] - 1) ok = false;
            }
            if (!ok) continue;
            const float wgt = ((k8 & 1) ? fr[0] : 1.0f - fr[0]) * (((k8 >> 1) & 1) ? fr[1] : 1.0f - fr[1]) *
                              ((k8 >> 2) ? fr[2] : 1.0f - fr[2]);
            const long long cc = cidx(g, q[0], q[1], q[2]);
            atomicAdd(&f.n[cc], wgt * wn);
            atomicAdd(&f.usx[cc], wgt * wn * u[0]);
            atomicAdd(&f.usy[cc], wgt * wn * u[1]);
            atomicAdd(&f.usz[cc], wgt * wn * u[2]);
        }
        const int h = atomicAdd(&s_holes, 1);
        sp.holes[base + h] = p;
        sp.x[s] = -1.0f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sp.hole_count[t] = s_holes;
        sp.hole_used[t] = 0;
    }
}

__global__ void k_mom_final(long long N, FluidDev f) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const float n = f.n[c];
    const bool keep = n > f.n_floor;
    f.ux[c] = keep ? f.usx[c] / n : 0.0f;
    f.uy[c] = keep ? f.usy[c] / n : 0.0f;
    f.uz[c] = keep ? f.usz[c] / n : 0.0f;
}

static inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

// Criterion (or classifier decision) -> dilated mask -> conversions.
hyb_status regime_update(hyb_ctx *c, const float *pm, const float *ps) {
    const GridDev &g = c->g;
    cudaStream_t st = c->stream;
    const hyb_regime_desc &rd = c->regime;
    uint8_t *raw = c->mask_tmp, *mask = c->mask;
    cudaMemcpyAsync(c->mask_prev, mask, (size_t)g.N, cudaMemcpyDeviceToDevice, st);
    const bool all = rd.policy == HYB_REGIME_ALL_KINETIC;
    const bool physics = !all && (!pm || rd.policy == HYB_REGIME_UNION);
    long long launches = 0;
    if (all) cudaMemsetAsync(raw, 1, (size_t)g.N, st);
    if (physics) {
        cudaMemsetAsync(c->ne, 0, sizeof(float) * g.N, st);
        for (const Species &s : c->sp)
            if (s.dev.kind == 0 && s.q < 0.0 && !s.has_zq && ++launches)
                k_density<<<g.ntiles, 256, 0, st>>>(g, s.dev, (float)(-s.q / (g.dd[0] * g.dd[1] * g.dd[2])), c->ne);
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
    k_dilate<<<dg, db, 0, st>>>(g, 0, rd.dilate, raw, mask);
    k_dilate<<<dg, db, 0, st>>>(g, 1, rd.dilate, mask, raw);
    k_dilate<<<dg, db, 0, st>>>(g, 2, rd.dilate, raw, mask);
    launches += 3;
    // conversions
    for (size_t f = 0; f < c->fluids.size(); ++f) {
        const int sid = rd.to_species[f];
        if (sid < 0 || sid >= (int)c->sp.size()) continue;
        const SpDev &dst = c->sp[sid].dev;
        // the tiles are compact between steps: new particles go straight into them
        k_fluid_to_particles<<<nblk(g.N), 256, 0, st>>>(g, mask, c->mask_prev, c->fluids[f], dst,
                                                        rd.ppc > 0 ? rd.ppc : 8, c->epoch, c->rho_bg, c->status);
        k_clamp_counts<<<(g.ntiles + 255) / 256, 256, 0, st>>>(g.ntiles, dst);
        k_mom_init<<<nblk(g.N), 256, 0, st>>>(g.N, c->fluids[f]);
        k_particles_to_fluid<<<g.ntiles, 256, 0, st>>>(g, mask, dst, c->fluids[f]);
        k_mom_final<<<nblk(g.N), 256, 0, st>>>(g.N, c->fluids[f]);
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
