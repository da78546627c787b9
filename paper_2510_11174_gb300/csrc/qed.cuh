// Device-side LCFA QED tables and their lookups (arXiv 2510.11174, Methodology:
// radiation reaction and pair production from Airy-function rates with the
// local field).  Built in FP64 by qed.cu; looked up in FP32 by the step.
//
//   chi_e = kappa sqrt((gamma E + u x B)^2 - (u.E)^2),  kappa = hbar w0 / m c^2
//   chi_g = kappa sqrt((eps E + k x B)^2 - (k.E)^2)
//   photon emission rate  (alpha/kappa) h(chi) / gamma,  spectrum F_em(chi, xi)
//   pair creation rate    (alpha/kappa) T(chi) / eps,    spectrum F_pair(chi, xi)
// Emission spectra are tabulated over mu = ln(xi/(1-xi)) - ln chi in
// [-30, 5] (the whole spectrum for every chi), pair spectra over xi in [0, 1].
#pragma once
#include "hyb_internal.cuh"

namespace hyb {

// rate tables: uniform in log2 chi (emission 2^-20 .. 2^10, pairs 2^-7 .. 2^10)
static constexpr int QED_EM_E0 = -20, QED_EM_E1 = 10, QED_EM_NPO = 256;
static constexpr int QED_EM_NH = (QED_EM_E1 - QED_EM_E0) * QED_EM_NPO + 1;
static constexpr int QED_PAIR_E0 = -7, QED_PAIR_E1 = 10, QED_PAIR_NPO = 1024;
static constexpr int QED_PAIR_NH = (QED_PAIR_E1 - QED_PAIR_E0) * QED_PAIR_NPO + 1;
// Spectrum tables: rows uniform in ln chi, blended linearly between rows; the
// blend's error, about (d ln chi)^2 / 8 times the curvature of the cumulative
// spectrum in ln chi, sets the sampler's accuracy (d ln chi = 0.02 here)
static constexpr int QED_NROW = 1024;  // spectrum table rows (ln chi)
static constexpr int QED_NCOL = 2048;  // spectrum table columns
static constexpr double QED_EM_CHI0 = 1e-6, QED_EM_CHI1 = 1e3;
static constexpr double QED_PAIR_CHI0 = 1e-2, QED_PAIR_CHI1 = 1e3;
static constexpr double QED_MU0 = -30.0, QED_MU1 = 5.0;

// linear interpolation of a log-log rate table on a log2 grid; below the grid:
//   emission: h ~ chi (slope 1); pairs: 0 (rate ~ exp(-8/3chi))
__device__ __forceinline__ float qed_rate(const float *lnt, float chi, int e0, int npo, int nh, bool emission) {
    if (!(chi > 0.0f)) return 0.0f;
    int i;
    float f;
    log2_grid(chi, e0, npo, i, f);
    if (i < 0) return emission ? expf(lnt[0]) * chi * exp2f((float)-e0) : 0.0f;
    if (i >= nh - 1) {
        i = nh - 2;
        f = 1.0f;
    }
    return expf(lnt[i] + f * (lnt[i + 1] - lnt[i]));
}

__device__ __forceinline__ float qed_h(const QedDev &q, float chi) {
    return qed_rate(q.em_lnh, chi, QED_EM_E0, QED_EM_NPO, QED_EM_NH, true);
}
__device__ __forceinline__ float qed_T(const QedDev &q, float chi) {
    return qed_rate(q.pair_lnT, chi, QED_PAIR_E0, QED_PAIR_NPO, QED_PAIR_NH, false);
}

// invert a cumulative row pair (rows i, i+1 blended with weight f) at r:
// returns the fractional column position
static __device__ __noinline__ float qed_invert(const float *cdf, int i, float f, float r) {
    const float *a = cdf + (long long)i * QED_NCOL, *b = a + QED_NCOL;
    int lo = 0, hi = QED_NCOL - 1;  // smallest k with C(k) >= r
    if (r <= (1.0f - f) * a[0] + f * b[0]) return -1.0f;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        const float c = (1.0f - f) * a[mid] + f * b[mid];
        if (c >= r) hi = mid; else lo = mid;
    }
    const float clo = (1.0f - f) * a[lo] + f * b[lo], chi_ = (1.0f - f) * a[hi] + f * b[hi];
    const float t = chi_ > clo ? (r - clo) / (chi_ - clo) : 0.5f;
    return (float)lo + fminf(fmaxf(t, 0.0f), 1.0f);
}

__device__ __forceinline__ void qed_row(float chi, double c0, double c1, int &i, float &f) {
    const float l0 = (float)log(c0), l1 = (float)log(c1);
    float y = (logf(chi) - l0) * ((float)(QED_NROW - 1) / (l1 - l0));
    y = fminf(fmaxf(y, 0.0f), (float)(QED_NROW - 1) - 1e-3f);
    i = (int)y;
    f = y - (float)i;
}

// photon energy fraction for an emission at chi with uniform r
__device__ __forceinline__ float qed_em_sample(const QedDev &q, float chi, float r) {
    int i;
    float f;
    qed_row(chi, QED_EM_CHI0, QED_EM_CHI1, i, f);
    const float dmu = (float)((QED_MU1 - QED_MU0) / (QED_NCOL - 1));
    const float k = qed_invert(q.em_cdf, i, f, r);
    if (k < 0.0f) {
        // below the first column the cumulative spectrum grows as xi^{1/3}
        const float c0 = (1.0f - f) * q.em_cdf[(long long)i * QED_NCOL] + f * q.em_cdf[(long long)(i + 1) * QED_NCOL];
        const float e = chi * expf((float)QED_MU0);
        const float xi0 = e / (1.0f + e);
        const float s = r / c0;
        return xi0 * s * s * s;
    }
    const float e = chi * expf((float)QED_MU0 + k * dmu);
    return e / (1.0f + e);
}

// electron energy fraction for a pair created at chi with uniform r
__device__ __forceinline__ float qed_pair_sample(const QedDev &q, float chi, float r) {
    int i;
    float f;
    qed_row(chi, QED_PAIR_CHI0, QED_PAIR_CHI1, i, f);
    const float k = qed_invert(q.pair_cdf, i, f, r);
    return fminf(fmaxf(k, 0.0f), (float)(QED_NCOL - 1)) / (float)(QED_NCOL - 1);
}

__device__ __forceinline__ float qed_chi(float kappa, const float e[3], const float b[3], const float u[3], float g) {
    const float f0 = g * e[0] + (u[1] * b[2] - u[2] * b[1]);
    const float f1 = g * e[1] + (u[2] * b[0] - u[0] * b[2]);
    const float f2 = g * e[2] + (u[0] * b[1] - u[1] * b[0]);
    const float ue = u[0] * e[0] + u[1] * e[1] + u[2] * e[2];
    const float s = f0 * f0 + f1 * f1 + f2 * f2 - ue * ue;
    return kappa * sqrtf(fmaxf(s, 0.0f));
}

// splitmix64 (Vigna): ids of particles created by an event
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t derived_id(uint64_t id, long long step, unsigned tag) {
    return splitmix64(id ^ splitmix64(((uint64_t)step << 8) | tag));
}

}  // namespace hyb
