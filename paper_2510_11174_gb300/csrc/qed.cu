// FP64 construction of the LCFA QED tables on the device (arXiv 2510.11174,
// Methodology: radiation reaction and pair production from Airy-function rates
// with the local field), and the table-evaluation entry.
//
// Airy functions are tabulated on z in [0, 16] with spacing 1/1024:
//  * z <= 1: Maclaurin series of the two solutions of y'' = z y
//    (Abramowitz & Stegun 10.4.2-10.4.5), Ai = Ai(0) f + Ai'(0) g, and the
//    termwise integral for int_0^z Ai, so int_z^inf Ai = 1/3 - int_0^z Ai;
//  * 1 < z <= 16: the system (Ai, Ai', int_z^inf Ai)' = (Ai', z Ai, -Ai)
//    integrated with classical RK4 from z = 16 downwards (the direction in
//    which Ai grows, so the integration is stable), started from the
//    asymptotic expansions (A&S 10.4.59, 10.4.61):
//      Ai(z)  ~ e^{-zeta} / (2 sqrt(pi) z^{1/4}) sum (-1)^k u_k zeta^{-k}
//      Ai'(z) ~ -z^{1/4} e^{-zeta} / (2 sqrt(pi)) sum (-1)^k v_k zeta^{-k}
//      u_k = Gamma(3k+1/2) / (54^k k! Gamma(k+1/2)),  v_k = -(6k+1)/(6k-1) u_k
//    and int_z^inf Ai ~ (-Ai'(z)/z - Ai(z)/z^2) / (1 - 2/z^3) (integration by
//    parts of Ai = Ai''/z);
//  * z > 16: every spectrum term is below e^{-42} and is taken as zero.
// Values between nodes are cubic Hermite interpolants (the derivatives are
// known: Ai' , z Ai, -Ai).
//
// Spectra and rates (see qed.cuh for the definitions):
//   F_em(chi, xi)   = -[Ai_1(z) + ((1-xi) + 1/(1-xi)) Ai'(z)/z],  z = (xi/(chi(1-xi)))^{2/3}
//   F_pair(chi, xi) = Ai_1(z) - (xi/(1-xi) + (1-xi)/xi) Ai'(z)/z, z = (1/(chi xi(1-xi)))^{2/3}
// h(chi) = int F_em dxi is integrated in mu = ln(xi/(1-xi)) - ln chi over
// [-30, 5] (z = e^{2mu/3}) by composite Simpson with step 1/128, plus the
// closed-form integral of the small-xi limit 2|Ai'(0)|/z below mu = -30;
// T(chi) = int F_pair dxi by composite Simpson in t = ln(xi/(1-xi)) over
// [-30, 30] with 8192 intervals.
// The spectrum rows are the running integrals of the same integrands,
// normalised to 1 at the end of the row.
#include <cmath>

#include "qed.cuh"

namespace hyb {

static constexpr int AIRY_NZ = 16384;              // intervals on [0, 16]
static constexpr double AIRY_DZ = 16.0 / AIRY_NZ;  // 1/1024

struct AiryTab {
    const double *ai, *aip, *aint;
};

__device__ void airy_series(double z, double ai0, double aip0, double *ai, double *aip, double *aint) {
    // f = sum a_m z^{3m}, a_m = a_{m-1} / ((3m)(3m-1));  g = sum b_m z^{3m+1}, b_m = b_{m-1} / ((3m+1)(3m))
    double f = 0, fp = 0, fi = 0, gg = 0, gp = 0, gi = 0;
    double a = 1.0, b = 1.0;
    const double z3 = z * z * z;
    double zp = 1.0, zprev = 1.0;  // z^{3m}, z^{3(m-1)}
    for (int m = 0; m < 40; ++m) {
        if (m > 0) {
            a /= (3.0 * m) * (3.0 * m - 1.0);
            b /= (3.0 * m + 1.0) * (3.0 * m);
            zprev = zp;
            zp *= z3;
        }
        f += a * zp;
        fp += m > 0 ? a * 3.0 * m * zprev * z * z : 0.0;  // d/dz z^{3m} = 3m z^{3m-1}
        fi += a * zp * z / (3.0 * m + 1.0);
        gg += b * zp * z;
        gp += b * (3.0 * m + 1.0) * zp;
        gi += b * zp * z * z / (3.0 * m + 2.0);
        if (a * zp < 1e-20 && b * zp < 1e-20) break;
    }
    *ai = ai0 * f + aip0 * gg;
    *aip = ai0 * fp + aip0 * gp;
    *aint = 1.0 / 3.0 - (ai0 * fi + aip0 * gi);
}

// one thread: fills the whole table
__global__ void k_airy_table(double *ai, double *aip, double *aint) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double PI = 3.14159265358979323846;
    const double ai0 = 1.0 / (pow(3.0, 2.0 / 3.0) * tgamma(2.0 / 3.0));
    const double aip0 = -1.0 / (pow(3.0, 1.0 / 3.0) * tgamma(1.0 / 3.0));
    const int k1 = (int)(1.0 / AIRY_DZ);
    for (int k = 0; k <= k1; ++k) airy_series(k * AIRY_DZ, ai0, aip0, &ai[k], &aip[k], &aint[k]);
    // asymptotic start at z = 16
    double z = 16.0;
    const double zeta = 2.0 / 3.0 * z * sqrt(z);
    double su = 0.0, sv = 0.0, u = 1.0, zk = 1.0;
    for (int k = 0; k <= 12; ++k) {
        if (k > 0) {
            u *= (3.0 * k - 0.5) * (3.0 * k - 1.5) * (3.0 * k - 2.5) / (54.0 * k * (k - 0.5));
            zk /= zeta;
        }
        const double v = k == 0 ? 1.0 : -(6.0 * k + 1.0) / (6.0 * k - 1.0) * u;
        const double sg = (k & 1) ? -1.0 : 1.0;
        su += sg * u * zk;
        sv += sg * v * zk;
    }
    const double pre = exp(-zeta) / (2.0 * sqrt(PI));
    double y0 = pre * pow(z, -0.25) * su;   // Ai
    double y1 = -pre * pow(z, 0.25) * sv;   // Ai'
    double y2 = (-y1 / z - y0 / (z * z)) / (1.0 - 2.0 / (z * z * z));  // int_z^inf Ai
    ai[AIRY_NZ] = y0;
    aip[AIRY_NZ] = y1;
    aint[AIRY_NZ] = y2;
    const int sub = 8;
    const double h = -AIRY_DZ / sub;
    for (int k = AIRY_NZ - 1; k > k1; --k) {
        for (int s = 0; s < sub; ++s) {
            // RK4 on y' = (y1, z y0, -y0)
            const double a0 = y1, a1 = z * y0, a2 = -y0;
            const double zm = z + 0.5 * h;
            const double b0 = y1 + 0.5 * h * a1, b1 = zm * (y0 + 0.5 * h * a0), b2 = -(y0 + 0.5 * h * a0);
            const double c0 = y1 + 0.5 * h * b1, c1 = zm * (y0 + 0.5 * h * b0), c2 = -(y0 + 0.5 * h * b0);
            const double ze = z + h;
            const double d0 = y1 + h * c1, d1 = ze * (y0 + h * c0), d2 = -(y0 + h * c0);
            y0 += h / 6.0 * (a0 + 2.0 * b0 + 2.0 * c0 + d0);
            y1 += h / 6.0 * (a1 + 2.0 * b1 + 2.0 * c1 + d1);
            y2 += h / 6.0 * (a2 + 2.0 * b2 + 2.0 * c2 + d2);
            z = ze;
        }
        z = k * AIRY_DZ;  // remove the drift of the running sum of h
        ai[k] = y0;
        aip[k] = y1;
        aint[k] = y2;
    }
}

// cubic Hermite interpolation of the tabulated functions; zero beyond z = 16
__device__ void airy_eval(const AiryTab &T, double z, double *ai, double *aip, double *aint) {
    if (z >= 16.0) {
        *ai = *aip = *aint = 0.0;
        return;
    }
    const double x = z / AIRY_DZ;
    int k = (int)x;
    if (k >= AIRY_NZ) k = AIRY_NZ - 1;
    const double t = x - k, t2 = t * t, t3 = t2 * t;
    const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
    const double za = k * AIRY_DZ, zb = (k + 1) * AIRY_DZ, d = AIRY_DZ;
    const double A0 = T.ai[k], A1 = T.ai[k + 1], P0 = T.aip[k], P1 = T.aip[k + 1];
    const double I0 = T.aint[k], I1 = T.aint[k + 1];
    *ai = h00 * A0 + h10 * d * P0 + h01 * A1 + h11 * d * P1;
    *aip = h00 * P0 + h10 * d * za * A0 + h01 * P1 + h11 * d * zb * A1;
    *aint = h00 * I0 - h10 * d * A0 + h01 * I1 - h11 * d * A1;
}

// emission integrand in mu (number spectrum times dxi/dmu)
__device__ double em_mu(const AiryTab &T, double chi, double mu) {
    const double e = chi * exp(mu);
    const double xi = e / (1.0 + e), omx = 1.0 / (1.0 + e);
    const double z = exp(2.0 * mu / 3.0);
    double ai, aip, aint;
    airy_eval(T, z, &ai, &aip, &aint);
    return -(aint + (omx + 1.0 / omx) * aip / z) * xi * omx;
}

__device__ double pair_xi(const AiryTab &T, double chi, double xi) {
    if (xi <= 0.0 || xi >= 1.0) return 0.0;
    const double z = pow(1.0 / (chi * xi * (1.0 - xi)), 2.0 / 3.0);
    if (z >= 16.0) return 0.0;
    double ai, aip, aint;
    airy_eval(T, z, &ai, &aip, &aint);
    return aint - (xi / (1.0 - xi) + (1.0 - xi) / xi) * aip / z;
}

// integral of the small-xi limit 2|Ai'(0)|/z over xi < xi(mu0)
__device__ double em_tail(double chi, double aip0) {
    const double e = chi * exp(QED_MU0);
    const double xa = e / (1.0 + e);
    return -2.0 * aip0 * pow(chi, 2.0 / 3.0) * 3.0 * cbrt(xa);
}

__global__ void k_em_rates(AiryTab T, float *lnh, double aip0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= QED_EM_NH) return;
    const double chi = exp2((double)QED_EM_E0 + (double)j / QED_EM_NPO);
    const int N = 35 * 128;  // Simpson intervals over [mu0, mu1]
    const double h = (QED_MU1 - QED_MU0) / N;
    double s = em_mu(T, chi, QED_MU0) + em_mu(T, chi, QED_MU1);
    for (int i = 1; i < N; ++i) s += (i & 1 ? 4.0 : 2.0) * em_mu(T, chi, QED_MU0 + i * h);
    lnh[j] = (float)log(s * h / 3.0 + em_tail(chi, aip0));
}

__global__ void k_em_cdf(AiryTab T, float *cdf, double aip0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= QED_NROW) return;
    const double l0 = log(QED_EM_CHI0), l1 = log(QED_EM_CHI1);
    const double chi = exp(l0 + (l1 - l0) * i / (QED_NROW - 1));
    const double dm = (QED_MU1 - QED_MU0) / (QED_NCOL - 1);
    const int sub = 4;  // Simpson panels per column (step dm / 4)
    const double h = dm / sub;
    // pass 0: the row total; pass 1: the normalised running integral
    double total = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        double acc = em_tail(chi, aip0);
        if (pass) cdf[(long long)i * QED_NCOL] = (float)(acc / total);
        for (int k = 1; k < QED_NCOL; ++k) {
            const double a = QED_MU0 + (k - 1) * dm;
            double s = em_mu(T, chi, a) + em_mu(T, chi, a + dm);
            for (int q = 1; q < sub; ++q) s += (q & 1 ? 4.0 : 2.0) * em_mu(T, chi, a + q * h);
            acc += s * h / 3.0;
            if (pass) cdf[(long long)i * QED_NCOL + k] = (float)(acc / total);
        }
        total = acc;
    }
}

__global__ void k_pair_rates(AiryTab T, float *lnT) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= QED_PAIR_NH) return;
    const double chi = exp2((double)QED_PAIR_E0 + (double)j / QED_PAIR_NPO);
    // Simpson in t = ln(xi/(1-xi)) over [-30, 30]: resolves the spectrum both at
    // xi ~ 1/2 (chi << 1) and down to xi ~ 1/chi (chi >> 1)
    const int N = 8192;
    const double h = 60.0 / N;
    double s = 0.0;  // both end points vanish
    for (int i = 1; i < N; ++i) {
        const double t = -30.0 + i * h;
        const double xi = 1.0 / (1.0 + exp(-t));
        s += (i & 1 ? 4.0 : 2.0) * pair_xi(T, chi, xi) * xi * (1.0 - xi);
    }
    const double v = s * h / 3.0;
    lnT[j] = (float)(v > 0.0 ? log(v) : -1e30);
}

__global__ void k_pair_cdf(AiryTab T, float *cdf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= QED_NROW) return;
    const double l0 = log(QED_PAIR_CHI0), l1 = log(QED_PAIR_CHI1);
    const double chi = exp(l0 + (l1 - l0) * i / (QED_NROW - 1));
    const double dx = 1.0 / (QED_NCOL - 1);
    const int sub = 4;  // Simpson panels per column (step dx / 4)
    const double h = dx / sub;
    double total = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        double acc = 0.0;
        if (pass) cdf[(long long)i * QED_NCOL] = 0.0f;
        for (int k = 1; k < QED_NCOL; ++k) {
            const double a = (k - 1) * dx;
            double s = pair_xi(T, chi, a) + pair_xi(T, chi, a + dx);
            for (int q = 1; q < sub; ++q) s += (q & 1 ? 4.0 : 2.0) * pair_xi(T, chi, a + q * h);
            acc += s * h / 3.0;
            if (pass) cdf[(long long)i * QED_NCOL + k] = (float)(total > 0.0 ? acc / total : 0.0);
        }
        total = acc;
    }
}

__global__ void k_eval_qed(QedDev q, AiryTab T, int what, const float *__restrict__ chi, const float *__restrict__ r,
                           int n, float *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    switch (what) {
        case HYB_QED_H: out[t] = qed_h(q, chi[t]); break;
        case HYB_QED_T: out[t] = qed_T(q, chi[t]); break;
        case HYB_QED_EM_SAMPLE: out[t] = qed_em_sample(q, chi[t], r[t]); break;
        case HYB_QED_PAIR_SAMPLE: out[t] = qed_pair_sample(q, chi[t], r[t]); break;
        default: {
            // 100 + j: the FP64 Airy table (j = 0 Ai, 1 Ai', 2 int Ai) at z = chi[t]
            double ai, aip, aint;
            airy_eval(T, chi[t], &ai, &aip, &aint);
            out[t] = (float)(what == 100 ? ai : (what == 101 ? aip : aint));
        }
    }
}

// physical constants (CODATA 2018)
static constexpr double QHBAR = 1.054571817e-34, QME = 9.1093837015e-31, QC = 299792458.0;
static constexpr double QALPHA = 7.2973525693e-3;

hyb_status setup_qed(hyb_ctx *c) {
    if (c->qed_ready) return HYB_OK;
    const double lambda = c->desc.lambda_um * 1e-6;
    if (!(lambda > 0.0)) return set_error(HYB_EINVAL, "QED needs lambda_um > 0");
    const double kappa = QHBAR * 2.0 * M_PI * QC / lambda / (QME * QC * QC);
    float *em_lnh = nullptr, *em_cdf = nullptr, *pair_lnT = nullptr, *pair_cdf = nullptr;
    if (ctx_alloc(c, (void **)&em_lnh, sizeof(float) * QED_EM_NH) ||
        ctx_alloc(c, (void **)&pair_lnT, sizeof(float) * QED_PAIR_NH) ||
        ctx_alloc(c, (void **)&em_cdf, sizeof(float) * QED_NROW * QED_NCOL) ||
        ctx_alloc(c, (void **)&pair_cdf, sizeof(float) * QED_NROW * QED_NCOL) ||
        ctx_alloc(c, (void **)&c->airy_ai, sizeof(double) * (AIRY_NZ + 1)) ||
        ctx_alloc(c, (void **)&c->airy_aip, sizeof(double) * (AIRY_NZ + 1)) ||
        ctx_alloc(c, (void **)&c->airy_aint, sizeof(double) * (AIRY_NZ + 1)))
        return set_error(HYB_ENOMEM, "QED table allocation failed");
    cudaStream_t st = c->stream;
    k_airy_table<<<1, 1, 0, st>>>(c->airy_ai, c->airy_aip, c->airy_aint);
    AiryTab T{c->airy_ai, c->airy_aip, c->airy_aint};
    const double aip0 = -1.0 / (std::pow(3.0, 1.0 / 3.0) * std::tgamma(1.0 / 3.0));
    k_em_rates<<<(QED_EM_NH + 127) / 128, 128, 0, st>>>(T, em_lnh, aip0);
    k_em_cdf<<<(QED_NROW + 31) / 32, 32, 0, st>>>(T, em_cdf, aip0);
    k_pair_rates<<<(QED_PAIR_NH + 127) / 128, 128, 0, st>>>(T, pair_lnT);
    k_pair_cdf<<<(QED_NROW + 31) / 32, 32, 0, st>>>(T, pair_cdf);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("QED tables: ") + cudaGetErrorString(e));
    c->qed.em_lnh = em_lnh;
    c->qed.em_cdf = em_cdf;
    c->qed.pair_lnT = pair_lnT;
    c->qed.pair_cdf = pair_cdf;
    c->qed.kappa = (float)kappa;
    c->qed.pref = (float)(QALPHA / kappa);
    c->qed_ready = true;
    return HYB_OK;
}

hyb_status eval_qed(hyb_ctx *c, int what, const float *chi, const float *r, int n, float *out) {
    hyb_status s = setup_qed(c);
    if (s != HYB_OK) return s;
    const bool sampler = what == HYB_QED_EM_SAMPLE || what == HYB_QED_PAIR_SAMPLE;
    if (!(what == HYB_QED_H || what == HYB_QED_T || sampler || (what >= 100 && what <= 102)))
        return set_error(HYB_EINVAL, "unknown QED table");
    if (sampler && !r) return set_error(HYB_EINVAL, "samplers need r");
    float *dc = nullptr, *dr = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, sizeof(float) * n) != cudaSuccess || cudaMalloc(&dr, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&dout, sizeof(float) * n) != cudaSuccess) {
        cudaFree(dc);
        cudaFree(dr);
        return set_error(HYB_ENOMEM, "eval staging failed");
    }
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(dc, chi, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (r) cudaMemcpyAsync(dr, r, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    AiryTab T{c->airy_ai, c->airy_aip, c->airy_aint};
    k_eval_qed<<<(n + 255) / 256, 256, 0, st>>>(c->qed, T, what, dc, dr, n, dout);
    cudaMemcpyAsync(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(dc);
    cudaFree(dr);
    cudaFree(dout);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("eval: ") + cudaGetErrorString(e));
    return HYB_OK;
}

}  // namespace hyb
