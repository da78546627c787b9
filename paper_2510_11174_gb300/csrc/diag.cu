// FP64 energy reductions (arXiv 2510.11174, Methodology: total energy from
// electromagnetic, kinetic and thermal components; conservation checks during
// steps).  Field energy (1/2) sum (E^2 + B^2) dV and particle kinetic energy
// sum w m (gamma - 1), both in units m_e c^2 n_c (c/w0)^3.
//
// Deterministic two-pass reduction: a fixed grid of blocks accumulates FP64
// per-thread sums in a fixed grid-stride order, reduces them with a fixed
// shared-memory tree and writes one partial per block into a scratch array;
// a single block then sums the partials of each quantity in block order.
#include "hyb_internal.cuh"

namespace hyb {

static constexpr int RB = 256;  // threads per reduction block

__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(RB) k_energy_fields(GridDev g, const float *__restrict__ E,
                                                      const float *__restrict__ B, double *__restrict__ partials,
                                                      int nblocks, int *__restrict__ status) {
    __shared__ double sh[RB];
    // each square is exact, the sums double-float; four independent sums per
    // thread keep four loads of each array in flight
    ff se[4], sb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) se[k] = sb[k] = ff{0.0f, 0.0f};
    bool finite = true;
    const long long n3 = 3 * g.N, stride = (long long)nblocks * RB;
    long long c = blockIdx.x * (long long)RB + threadIdx.x;
    for (; c + 3 * stride < n3; c += 4 * stride) {
        float e[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            e[k] = E[c + k * stride];
            b[k] = B[c + k * stride];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            finite = finite && isfinite(e[k]) && isfinite(b[k]);
            se[k] = ff_add(se[k], ff_two_prod(e[k], e[k]));
            sb[k] = ff_add(sb[k], ff_two_prod(b[k], b[k]));
        }
    }
    for (; c < n3; c += stride) {
        const float e = E[c], b = B[c];
        finite = finite && isfinite(e) && isfinite(b);
        se[0] = ff_add(se[0], ff_two_prod(e, e));
        sb[0] = ff_add(sb[0], ff_two_prod(b, b));
    }
    const ff se_t = ff_add(ff_add(se[0], se[1]), ff_add(se[2], se[3]));
    const ff sb_t = ff_add(ff_add(sb[0], sb[1]), ff_add(sb[2], sb[3]));
    if (!finite) atomicOr(status, ST_NAN);
    const double te = block_sum(ff_to_double(se_t), sh);
    const double tb = block_sum(ff_to_double(sb_t), sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = te;
        partials[nblocks + blockIdx.x] = tb;
    }
}

// sum over particles of w (gamma - 1) (massive; times m per block) or w |u| (photons)
__global__ void __launch_bounds__(RB) k_energy_species(GridDev g, SpDev sp, double *__restrict__ partials,
                                                       int nblocks) {
    __shared__ double sh[RB];
    // work items are (chunk of LCH slots, tile), chunk-major: item i goes to
    // warp i mod W (W = nblocks x 8 warps), its lanes take the chunk's
    // particles -- a fixed assignment (fixed sum order) that spreads dense
    // tiles over many warps; chunks past a tile's count end at once.  The
    // item is stepped by W with a carry, not divided out.
    constexpr int NW = RB / 32, LCH = 256;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = (sp.cap + LCH - 1) / LCH, nt = g.ntiles;
    const int W = nblocks * NW, w = blockIdx.x * NW + warp;
    const int dt = W % nt, dch = W / nt;
    int t = w % nt, ch = w / nt;
    ff acc = {0.0f, 0.0f};
    while (ch < nch) {
        const int n = min(sp.count[t], sp.cap), p0 = ch * LCH;
        if (p0 < n) {
            const int p1 = min(n, p0 + LCH);
            const long long base = (long long)t * sp.cap;
#pragma unroll 4
            for (int p = p0 + lane; p < p1; p += 32) {
                const ff u2 = ff_u2(sp.ux[base + p], sp.uy[base + p], sp.uz[base + p]);
                const ff term = sp.kind == 1 ? ff_norm(u2) : ff_gamma_minus_one(u2);
                acc = ff_add(acc, ff_mulf(term, sp.w[base + p]));
            }
        }
        t += dt;
        ch += dch;
        if (t >= nt) {
            t -= nt;
            ++ch;
        }
    }
    const double tot = block_sum(ff_to_double(acc), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = sp.kind == 1 ? tot : tot * sp.m_d;
}

__global__ void __launch_bounds__(RB) k_final(const double *__restrict__ partials, int nq, int nblocks,
                                              double dvol_half, double *__restrict__ out) {
    __shared__ double sh[RB];
    for (int q = 0; q < nq; ++q) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += RB) acc += partials[(long long)q * nblocks + b];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) out[q] = q < 2 ? acc * dvol_half : acc;
    }
}

// block s < set.n: particle count and event tallies of species s, summed
// over the tiles in a fixed order (thread-strided, then a shared-memory
// tree); block set.n: the reduction results, clamp counters and status word
__global__ void __launch_bounds__(RB) k_diag_summary(SpSet set, int ntiles, const double *__restrict__ red, int nred,
                                                     ClampPtrs cl, const int *__restrict__ status,
                                                     DiagSummary *__restrict__ out) {
    __shared__ double sh[RB];
    const int b = blockIdx.x;
    if (b < set.n) {
        const SpDev &sp = set.s[b];
        double cnt = 0.0, te[NTALLY] = {0.0, 0.0, 0.0}, tn[NTALLY] = {0.0, 0.0, 0.0};  // exact below 2^53
#pragma unroll 4
        for (int t = threadIdx.x; t < ntiles; t += RB) {
            cnt += (double)min(sp.count[t], sp.cap);
#pragma unroll
            for (int k = 0; k < NTALLY; ++k) {
                te[k] += sp.tal_e[(long long)t * NTALLY + k];
                tn[k] += (double)sp.tal_n[(long long)t * NTALLY + k];
            }
        }
        const double c = block_sum(cnt, sh);
        if (threadIdx.x == 0) out->count[b] = (long long)c;
#pragma unroll
        for (int k = 0; k < NTALLY; ++k) {
            const double e = block_sum(te[k], sh), n = block_sum(tn[k], sh);
            if (threadIdx.x == 0) {
                out->tal_e[b][k] = e;
                out->tal_n[b][k] = (unsigned long long)n;
            }
        }
    } else {
        for (int i = threadIdx.x; i < nred; i += RB) out->red[i] = red[i];
        if (threadIdx.x < cl.n) out->clamped[threadIdx.x] = *cl.p[threadIdx.x];
        if (threadIdx.x == 0) out->status = *status;
    }
}

void launch_diag_summary(const SpSet &set, int ntiles, const double *red, int nred, const ClampPtrs &cl,
                         const int *status, DiagSummary *out, cudaStream_t st) {
    k_diag_summary<<<set.n + 1, RB, 0, st>>>(set, ntiles, red, nred, cl, status, out);
}

void launch_energy(const GridDev &g, const float *E, const float *B, const SpSet &set, double *partials,
                   int nblocks, double *out, int *status, cudaStream_t st, int n_extra) {
    k_energy_fields<<<nblocks, RB, 0, st>>>(g, E, B, partials, nblocks, status);
    for (int s = 0; s < set.n; ++s)
        k_energy_species<<<nblocks, RB, 0, st>>>(g, set.s[s], partials + (long long)(2 + s) * nblocks, nblocks);
    const double dvol_half = 0.5 * g.dd[0] * g.dd[1] * g.dd[2];
    // quantities 2 + set.n .. are partials the caller filled before (already in final units)
    k_final<<<1, RB, 0, st>>>(partials, 2 + set.n + n_extra, nblocks, dvol_half, out);
}

}  // namespace hyb
