// FP64 construction of the ionization rate tables on the device, and the
// table-evaluation entry used by hyb_eval_rate_table.
//
// Rates (atomic units), for the removal of an electron with orbital quantum
// number l (m = 0) from charge state Z (charge after ionization Zc = Z + 1):
//   ADK (Ammosov, Delone, Krainov 1986):
//     n* = Zc / sqrt(2 Ip), l* = n* - 1, k = (2 Ip)^{3/2},
//     ln C^2 = 2 n* ln 2 - ln n* - lnGamma(n* + l* + 1) - lnGamma(n* - l*),
//     ln w_ADK = ln C^2 + ln((2l+1) Ip) + (2n* - 1) ln(2k/F) - 2k/(3F)
//   multiphoton: K = ceil(Ip / w0) photons, w_MPI ~ F^{2K}, normalised to
//     equal ADK at the blend centre F* where the Keldysh parameter
//     gamma = w0 sqrt(2 Ip) / F equals 1.5:
//     ln w_MPI = ln w_ADK(F*) + 2K ln(F / F*)
//   blend (sigmoid in gamma, width 0.1, on the logarithm of the rates so that
//   neither power law leaks into the other regime):
//     S = 1 / (1 + exp(-(gamma - 1.5) / 0.1)),
//     ln w = S ln w_MPI + (1 - S) ln w_ADK.
#include <cmath>
#include <vector>

#include "ionize.cuh"

namespace hyb {

__device__ double adk_ln_rate(double F, double Ip, double Zc, int l) {
    const double ns = Zc / sqrt(2.0 * Ip), ls = ns - 1.0;
    const double lnC2 = 2.0 * ns * 0.69314718055994530942 - log(ns) - lgamma(ns + ls + 1.0) - lgamma(ns - ls);
    const double k = 2.0 * Ip * sqrt(2.0 * Ip);
    return lnC2 + log((2.0 * l + 1.0) * Ip) + (2.0 * ns - 1.0) * log(2.0 * k / F) - 2.0 * k / (3.0 * F);
}

__global__ void k_build_ion_lut(float *__restrict__ lnw, int zmax, const double *__restrict__ ip_au,
                                const int *__restrict__ lq, double w0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= zmax * ION_NL) return;
    const int Z = t / ION_NL, i = t % ION_NL;
    const double F = exp2((double)ION_E0 + (double)i / ION_NPO);
    const double Ip = ip_au[Z], Zc = Z + 1.0;
    const int l = lq[Z];
    const double lnadk = adk_ln_rate(F, Ip, Zc, l);
    const double K = ceil(Ip / w0);
    const double Fs = w0 * sqrt(2.0 * Ip) / 1.5;
    const double lnmpi = adk_ln_rate(Fs, Ip, Zc, l) + 2.0 * K * log(F / Fs);
    const double gam = w0 * sqrt(2.0 * Ip) / F;
    const double S = 1.0 / (1.0 + exp(-(gam - 1.5) / 0.1));
    lnw[t] = (float)(S * lnmpi + (1.0 - S) * lnadk);
}

__global__ void k_eval_ion(SpDev sp, int Z, const float *__restrict__ F, int n, float *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = ion_rate_lookup(sp, Z, F[t]);
}

// physical constants (CODATA 2018) for the unit conversions
static constexpr double C_LIGHT = 299792458.0, Q_E = 1.602176634e-19, ME_KG = 9.1093837015e-31;
static constexpr double T_AU = 2.4188843265857e-17, E_AU = 5.14220674763e11, HARTREE_EV = 27.211386245988;
static constexpr double MC2_EV = 510998.95;

hyb_status setup_ionization(hyb_ctx *c, SpDev &s, const hyb_species_desc *d) {
    if (d->zmax <= 0) return HYB_OK;
    if (d->zmax > 8) return set_error(HYB_EINVAL, "zmax must be <= 8");
    if (!d->zq) return set_error(HYB_EINVAL, "an ionizable species needs per-particle charge states (zq)");
    if (d->ionize_into < 0 || d->ionize_into >= (int)c->sp.size())
        return set_error(HYB_EINVAL, "ionize_into must name an already loaded species");
    for (int z = 0; z < d->zmax; ++z)
        if (!(d->ip_eV[z] > 0.0) || d->l_qn[z] < 0 || d->l_qn[z] > 3)
            return set_error(HYB_EINVAL, "bad ionization potential or quantum number");
    const double lambda = c->desc.lambda_um * 1e-6;
    if (!(lambda > 0.0)) return set_error(HYB_EINVAL, "ionization needs lambda_um > 0");
    const double w0 = 2.0 * M_PI * C_LIGHT / lambda;
    const double Eref = ME_KG * C_LIGHT * w0 / Q_E;
    s.zmax = d->zmax;
    s.ion_into = d->ionize_into;
    s.sp_index = (uint32_t)c->sp.size();
    s.e_ratio = (float)(Eref / E_AU);
    s.dt_au = (float)(c->g.dt_d / w0 / T_AU);
    std::vector<double> ip(d->zmax);
    std::vector<int> lq(d->zmax);
    for (int z = 0; z < d->zmax; ++z) {
        ip[z] = d->ip_eV[z] / HARTREE_EV;
        lq[z] = d->l_qn[z];
        s.ip_mc2[z] = d->ip_eV[z] / MC2_EV;
    }
    float *lnw = nullptr;
    double *dip = nullptr;
    int *dlq = nullptr;
    if (ctx_alloc(c, (void **)&lnw, sizeof(float) * d->zmax * ION_NL))
        return set_error(HYB_ENOMEM, "ionization table allocation failed");
    // the small parameter arrays are staged in temporary device buffers
    if (cudaMalloc(&dip, sizeof(double) * 8) != cudaSuccess || cudaMalloc(&dlq, sizeof(int) * 8) != cudaSuccess) {
        cudaFree(dip);
        return set_error(HYB_ENOMEM, "ionization parameter staging failed");
    }
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(dip, ip.data(), sizeof(double) * d->zmax, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dlq, lq.data(), sizeof(int) * d->zmax, cudaMemcpyHostToDevice, st);
    const int tot = d->zmax * ION_NL;
    k_build_ion_lut<<<(tot + 255) / 256, 256, 0, st>>>(lnw, d->zmax, dip, dlq, w0 * T_AU);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(dip);
    cudaFree(dlq);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("ionization table: ") + cudaGetErrorString(e));
    s.lnw = lnw;
    return HYB_OK;
}

hyb_status eval_ion_table(hyb_ctx *c, const SpDev &s, int Z, const float *x_host, int n, float *out_host) {
    if (s.zmax <= 0 || Z < 0 || Z >= s.zmax) return set_error(HYB_EINVAL, "species/level has no ionization table");
    float *dx = nullptr, *dy = nullptr;
    if (cudaMalloc(&dx, sizeof(float) * n) != cudaSuccess || cudaMalloc(&dy, sizeof(float) * n) != cudaSuccess) {
        cudaFree(dx);
        return set_error(HYB_ENOMEM, "eval staging failed");
    }
    cudaStream_t st = c->stream;
    cudaMemcpyAsync(dx, x_host, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    k_eval_ion<<<(n + 255) / 256, 256, 0, st>>>(s, Z, dx, n, dy);
    cudaMemcpyAsync(out_host, dy, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(dx);
    cudaFree(dy);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("eval: ") + cudaGetErrorString(e));
    return HYB_OK;
}

}  // namespace hyb
