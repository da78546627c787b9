// SwitchNet, the paper's per-cell regime classifier (Table 1 and Results: an
// MLP on ten features of a cell, 10 -> 128 -> 256 with ReLU, residual
// connections and dropout 0.2, a 4-head attention layer 256 -> 256, and a
// sigmoid output; trained with BCE and a physics term, scored by AUC).
//
// A cell's input is one feature vector, a sequence of one token, so the
// attention layer's softmax over its single key is 1 and the layer reduces to
// its value and output projections, out = W_o (W_v h + b_v) + b_o.  The four
// dense layers run on k_gemm_tc (tcgen05, FP32 out) in 128-column slices;
// k_act_finish adds bias, ReLU, dropout and the identity shortcut; the last
// layer (256 -> 1) is a dot product per cell.  Training: the classifier's
// energy-weighted BCE, data gradients through the same GEMM kernel with the
// transposed weights, weight gradients of the four dense layers as
// tensor-core contractions over the cells (wgrad_tc; the output layer's 256
// weights as a fixed-order FP32 reduction), Adam on FP32 masters.  See hyb_switchnet_* in include/hyb.h.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"
#include "philox.cuh"

namespace hyb {
namespace {

constexpr int SN_L = 4;                                      // dense layers on the tensor cores
constexpr int SN_CI[SN_L] = {10, 128, 256, 256}, SN_CO[SN_L] = {128, 256, 256, 256};
constexpr int SN_KP[SN_L] = {16, 128, 256, 256};             // K padded to 16
constexpr int SN_RELU[SN_L] = {1, 1, 0, 0};
constexpr int SN_RES[SN_L] = {1, 1, 0, 0};
constexpr int SN_DROP = 1;                                   // dropout after layer 1's ReLU
constexpr int NF = 10;                                       // features: E, B, J, rho
constexpr int RBS = 256;
constexpr int WCH = 4096;                                    // cells per weight-gradient partial

inline unsigned nbs(long long n, int b = RBS) { return (unsigned)((n + b - 1) / b); }

// features [10][n] -> normalised BF16 [n][16]
__global__ void k_sn_prep(const float *__restrict__ x, long long n, const float *__restrict__ mean,
                          const float *__restrict__ sd, __nv_bfloat16 *__restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(c < NF ? (x[c * n + t] - mean[c]) / sd[c] : 0.0f);
    uint4 *dst = reinterpret_cast<uint4 *>(out + t * 16);
    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// weights W [co][ci] -> 128-column slice `slice` of the K-major core layout
// [K/8][128][8] (K = kp); transposed: the slice of W^T (inputs co, outputs ci)
__global__ void k_sn_pack(const float *__restrict__ W, int ci_n, int co_n, int kp, int slice, int transpose,
                          __nv_bfloat16 *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kp * 128) return;
    const int j = t % 8, n = (t / 8) % 128, kc = t / (8 * 128);
    const int k = kc * 8 + j, row = slice * 128 + n;
    float v = 0.0f;
    if (!transpose) {
        if (row < co_n && k < ci_n) v = W[(long long)row * ci_n + k];
    } else {
        if (k < co_n && row < ci_n) v = W[(long long)k * ci_n + row];
    }
    out[t] = __float2bfloat16_rn(v);
}

// logit = sum_k bf16(w[k]) a[k] + b (the 256 -> 1 output layer)
__global__ void k_sn_last(const __nv_bfloat16 *__restrict__ a, const float *__restrict__ w, const float *__restrict__ b,
                          long long n, float *__restrict__ logit) {
    __shared__ float ws[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) ws[i] = __bfloat162float(__float2bfloat16_rn(w[i]));
    __syncthreads();
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint4 *src = reinterpret_cast<const uint4 *>(a + t * 256);
    float acc = 0.0f;
    for (int g = 0; g < 32; ++g) {
        uint4 u = src[g];
        const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc += ws[g * 8 + j] * __bfloat162float(h[j]);
    }
    logit[t] = acc + b[0];
}

// MC statistics of sigmoid(logit): pass k (1-based) into the running mean and M2
__global__ void k_sn_mc(const float *__restrict__ logit, long long n, int k, float *__restrict__ pm,
                        float *__restrict__ m2) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float p = 1.0f / (1.0f + expf(-logit[t]));
    if (k == 1) {
        pm[t] = p;
        m2[t] = 0.0f;
    } else {
        const float d = p - pm[t];
        const float mu = pm[t] + d / (float)k;
        pm[t] = mu;
        m2[t] += d * (p - mu);
    }
}

__global__ void k_sn_mc_final(long long n, int k, float *__restrict__ m2) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) m2[t] = sqrtf(fmaxf(m2[t], 0.0f) / (float)k);
}

// data gradient of the output layer: dz[c][k] = bf16(dlogit[c] bf16(w[k])), and
// the BF16 copy of dlogit (the operand of its weight gradient)
__global__ void k_sn_dlast(const float *__restrict__ dlogit, const float *__restrict__ w, long long n,
                           __nv_bfloat16 *__restrict__ dz, __nv_bfloat16 *__restrict__ dl16) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n * 32) return;
    const long long c = t / 32;
    const int g = (int)(t % 32);
    const float d = dlogit[c];
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(d * __bfloat162float(__float2bfloat16_rn(w[g * 8 + j])));
    *reinterpret_cast<uint4 *>(dz + c * 256 + g * 8) = *reinterpret_cast<const uint4 *>(o);
    if (g == 0) {
        __align__(16) __nv_bfloat16 z[8];
        z[0] = __float2bfloat16_rn(d);
        for (int j = 1; j < 8; ++j) z[j] = __float2bfloat16_rn(0.0f);
        *reinterpret_cast<uint4 *>(dl16 + c * 8) = *reinterpret_cast<const uint4 *>(z);
    }
}

// G[c][i] += R[c][i] for i < ci (the shortcut's share of a data gradient; R has cr columns)
__global__ void k_sn_addres(float *__restrict__ G, int cg, const float *__restrict__ R, int cr, int ci, long long n) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n * ci) return;
    const long long c = t / ci;
    const int i = (int)(t % ci);
    G[c * cg + i] += R[c * cr + i];
}

// weight-gradient partials of a dense layer: part[chunk][ci][co] = sum over
// the chunk's cells of A[c][ci0 + ci] dZ[c][co0 + co] (32 x 32 block), and the
// bias partials bpart[chunk][co] (ci0 = 0 blocks)
__global__ void __launch_bounds__(256) k_sn_wgrad(const __nv_bfloat16 *__restrict__ A, int ca, int ci0, int ci_n,
                                                  const __nv_bfloat16 *__restrict__ dZ, int cz, int co0, int co_n,
                                                  long long n, float *__restrict__ part, float *__restrict__ bpart) {
    __shared__ float sa[64][33], sz[64][33];
    const long long c0 = (long long)blockIdx.x * WCH, c1 = min(c0 + WCH, n);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f}, bacc = 0.0f;
    for (long long s0 = c0; s0 < c1; s0 += 64) {
        for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
            const int r = i / 32, ch = i % 32;
            const long long c = s0 + r;
            sa[r][ch] = (c < c1 && ch < ci_n) ? __bfloat162float(A[c * ca + ci0 + ch]) : 0.0f;
            sz[r][ch] = (c < c1 && ch < co_n) ? __bfloat162float(dZ[c * cz + co0 + ch]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int o = threadIdx.x + k * 256, ci = o / 32, co = o % 32;
            float s = 0.0f;
            for (int r = 0; r < 64; ++r) s += sa[r][ci] * sz[r][co];
            acc[k] += s;
        }
        if (threadIdx.x < 32)
            for (int r = 0; r < 64; ++r) bacc += sz[r][threadIdx.x];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) part[(long long)blockIdx.x * 1024 + threadIdx.x + k * 256] = acc[k];
    if (threadIdx.x < 32) bpart[(long long)blockIdx.x * 32 + threadIdx.x] = bacc;
}

// summed block [ci][co] (32 x 32) -> gw[co0 + co][ci0 + ci] (within ci_n x co_n)
__global__ void k_sn_scatter(const float *__restrict__ in, int ci_n, int co_n, int ci0, int co0, int CItot,
                             float *__restrict__ gw) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= 1024) return;
    const int ci = o / 32, co = o % 32;
    if (ci < ci_n && co < co_n) gw[(long long)(co0 + co) * CItot + ci0 + ci] = in[o];
}

}  // namespace
}  // namespace hyb

using namespace hyb;

struct hyb_switchnet {
    hyb_switchnet_desc d;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *w[SN_L + 1] = {}, *b[SN_L + 1] = {};              // masters [co][ci]; layer 4 = the 256 -> 1 output
    float *mw[SN_L + 1] = {}, *vw[SN_L + 1] = {}, *mb[SN_L + 1] = {}, *vb[SN_L + 1] = {};
    float *gw[SN_L + 1] = {}, *gb[SN_L + 1] = {};
    __nv_bfloat16 *pk[SN_L][2] = {}, *pkT[SN_L][2] = {};     // 128-column slices
    float *mean = nullptr, *std_ = nullptr;
    int *status = nullptr;
    long long cap = 0;
    __nv_bfloat16 *a[SN_L + 1] = {};                         // a[0] = x_hat [n][16], a[l + 1] = output of layer l
    float *z[SN_L] = {};                                      // pre-activations (no bias) [n][co]
    float *logit = nullptr, *dlogit = nullptr, *edens = nullptr;
    float *G1 = nullptr, *G2 = nullptr;                       // data gradients [n][256]
    __nv_bfloat16 *dz = nullptr, *dl16 = nullptr;
    float *wpart = nullptr, *wsum = nullptr;
    double *lpart = nullptr;
    int lblocks = 2 * 152;
    long long adam_t = 0;
    WgradScratch *wg = nullptr;                               // operands of the tensor-core weight gradients
    std::vector<void *> owned;
};

namespace {

cudaError_t sn_alloc(hyb_switchnet *m, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) m->owned.push_back(*p);
    return e;
}

void sn_free(hyb_switchnet *m, void *&p) {
    if (!p) return;
    for (auto it = m->owned.begin(); it != m->owned.end(); ++it)
        if (*it == p) {
            m->owned.erase(it);
            break;
        }
    cudaFree(p);
    p = nullptr;
}

inline int sn_ci(int l) { return l < SN_L ? SN_CI[l] : 256; }
inline int sn_co(int l) { return l < SN_L ? SN_CO[l] : 1; }

hyb_status sn_repack(hyb_switchnet *m) {
    for (int l = 0; l < SN_L; ++l) {
        for (int s = 0; s < SN_CO[l] / 128; ++s)
            k_sn_pack<<<nbs(SN_KP[l] * 128), RBS, 0, m->stream>>>(m->w[l], SN_CI[l], SN_CO[l], SN_KP[l], s, 0, m->pk[l][s]);
        if (l > 0)
            for (int s = 0; s < SN_CI[l] / 128; ++s)
                k_sn_pack<<<nbs(SN_CO[l] * 128), RBS, 0, m->stream>>>(m->w[l], SN_CI[l], SN_CO[l], SN_CO[l], s, 1,
                                                                      m->pkT[l][s]);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("switchnet packing: ") + cudaGetErrorString(e));
    return HYB_OK;
}

hyb_status sn_reserve(hyb_switchnet *m, long long n) {
    if (n <= m->cap) return HYB_OK;
    cudaStreamSynchronize(m->stream);
    for (int l = 0; l <= SN_L; ++l) {
        void *p = m->a[l];
        sn_free(m, p);
        m->a[l] = nullptr;
    }
    for (int l = 0; l < SN_L; ++l) {
        void *p = m->z[l];
        sn_free(m, p);
        m->z[l] = nullptr;
    }
    void *ps[8] = {m->logit, m->dlogit, m->edens, m->G1, m->G2, m->dz, m->dl16, m->wpart};
    for (void *&p : ps) sn_free(m, p);
    m->logit = m->dlogit = m->edens = m->G1 = m->G2 = m->wpart = nullptr;
    m->dz = m->dl16 = nullptr;
    m->cap = 0;
    const int aw[SN_L + 1] = {16, 128, 256, 256, 256};
    for (int l = 0; l <= SN_L; ++l)
        if (sn_alloc(m, (void **)&m->a[l], sizeof(__nv_bfloat16) * aw[l] * n))
            return set_error(HYB_ENOMEM, "switchnet activation buffers");
    for (int l = 0; l < SN_L; ++l)
        if (sn_alloc(m, (void **)&m->z[l], sizeof(float) * SN_CO[l] * n))
            return set_error(HYB_ENOMEM, "switchnet activation buffers");
    const long long nch = (n + WCH - 1) / WCH;
    if (sn_alloc(m, (void **)&m->logit, sizeof(float) * n) || sn_alloc(m, (void **)&m->dlogit, sizeof(float) * n) ||
        sn_alloc(m, (void **)&m->edens, sizeof(float) * n) || sn_alloc(m, (void **)&m->G1, sizeof(float) * 256 * n) ||
        sn_alloc(m, (void **)&m->G2, sizeof(float) * 256 * n) ||
        sn_alloc(m, (void **)&m->dz, sizeof(__nv_bfloat16) * 256 * n) ||
        sn_alloc(m, (void **)&m->dl16, sizeof(__nv_bfloat16) * 8 * n) ||
        sn_alloc(m, (void **)&m->wpart, sizeof(float) * nch * (1024 + 32)))
        return set_error(HYB_ENOMEM, "switchnet activation buffers");
    m->cap = n;
    return HYB_OK;
}

// out [n][pitch] FP32 = x [n][K] x packed slices (128 columns each)
hyb_status sn_gemm(hyb_switchnet *m, const __nv_bfloat16 *x, int K, __nv_bfloat16 *const *pks, int nslices, float *out,
                   int pitch, long long n) {
    for (int s = 0; s < nslices; ++s) {
        GemmArgs g;
        memset(&g, 0, sizeof(g));
        g.x = x;
        g.w = pks[s];
        g.y = out;
        g.rows = n;
        g.K = K;
        g.N = 128;
        g.pitch = pitch;
        g.off = s * 128;
        g.status = m->status;
        hyb_status st = launch_gemm_tc(g, m->stream);
        if (st != HYB_OK) return st;
    }
    return HYB_OK;
}

DropArgs sn_drop(const hyb_switchnet *m, int l, int pass) {
    DropArgs dr;
    memset(&dr, 0, sizeof(dr));
    if (l == SN_DROP && pass >= 0) {
        dr.thr = dropout_threshold(m->d.dropout);
        dr.scale = dropout_scale(dr.thr);
        dr.seed = m->d.seed;
        dr.pass = (uint32_t)pass;
        dr.layer = (uint32_t)l;
    }
    return dr;
}

// forward of the prepared features m->a[0] -> m->logit
hyb_status sn_forward(hyb_switchnet *m, long long n, int pass) {
    for (int l = 0; l < SN_L; ++l) {
        hyb_status s = sn_gemm(m, m->a[l], SN_KP[l], m->pk[l], SN_CO[l] / 128, m->z[l], SN_CO[l], n);
        if (s != HYB_OK) return s;
        k_act_finish<<<nbs(n * (SN_CO[l] / 8)), RBS, 0, m->stream>>>(
            m->z[l], m->b[l], SN_CO[l], SN_RELU[l], SN_RES[l] ? m->a[l] : nullptr, SN_KP[l], sn_drop(m, l, pass), 1, n,
            m->a[l + 1], nullptr);
    }
    k_sn_last<<<nbs(n), RBS, 0, m->stream>>>(m->a[SN_L], m->w[SN_L], m->b[SN_L], n, m->logit);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("switchnet forward: ") + cudaGetErrorString(e));
    return HYB_OK;
}

// weight and bias gradient of a dense layer (A [n][ca] with ci_n real columns, dZ [n][cz] with co_n)
void sn_wgrad(hyb_switchnet *m, const __nv_bfloat16 *A, int ca, int ci_n, const __nv_bfloat16 *dZ, int cz, int co_n,
              long long n, float *gw, float *gb) {
    const int nch = (int)((n + WCH - 1) / WCH);
    for (int ci0 = 0; ci0 < ci_n; ci0 += 32)
        for (int co0 = 0; co0 < co_n; co0 += 32) {
            const int cin = ci_n - ci0 < 32 ? ci_n - ci0 : 32, con = co_n - co0 < 32 ? co_n - co0 : 32;
            float *part = m->wpart, *bpart = m->wpart + (long long)nch * 1024;
            k_sn_wgrad<<<nch, 256, 0, m->stream>>>(A, ca, ci0, cin, dZ, cz, co0, con, n, part, bpart);
            k_sum_parts<<<4, 256, 0, m->stream>>>(part, nch, 1024, m->wsum);
            k_sn_scatter<<<4, 256, 0, m->stream>>>(m->wsum, cin, con, ci0, co0, ci_n, gw);
            if (ci0 == 0) {
                k_sum_parts<<<1, 32, 0, m->stream>>>(bpart, nch, 32, m->wsum + 1024);
                cudaMemcpyAsync(gb + co0, m->wsum + 1024, sizeof(float) * con, cudaMemcpyDeviceToDevice, m->stream);
            }
        }
}

hyb_status sn_check(hyb_switchnet *m, long long n) {
    if (n < 1) return set_error(HYB_EINVAL, "no cells");
    return sn_reserve(m, n);
}

}  // namespace

extern "C" {

void hyb_switchnet_destroy(hyb_switchnet *m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void *p : m->owned) cudaFree(p);
    delete m->wg;
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

hyb_status hyb_switchnet_create(const hyb_switchnet_desc *d, hyb_switchnet **out) {
    if (!d || !out) return set_error(HYB_EINVAL, "null argument");
    *out = nullptr;
    if (!(d->dropout >= 0.0 && d->dropout < 1.0)) return set_error(HYB_EINVAL, "dropout must be in [0, 1)");
    for (int c = 0; c < NF; ++c)
        if (!(d->std[c] > 0.0f)) return set_error(HYB_EINVAL, "normalisation std must be > 0");
    hyb_switchnet *m = new hyb_switchnet();
    m->wg = new WgradScratch();
    m->d = *d;
    m->d.dropout = dropout_threshold(d->dropout) / 65536.0;
    if (!(m->d.lr > 0)) m->d.lr = 1e-3;
    if (!(m->d.beta1 > 0)) m->d.beta1 = 0.9;
    if (!(m->d.beta2 > 0)) m->d.beta2 = 0.999;
    if (!(m->d.eps > 0)) m->d.eps = 1e-8;
    if (m->d.mc_passes <= 0) m->d.mc_passes = 1;
    if (d->stream) {
        m->stream = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete m;
            return set_error(HYB_ECUDA, "stream create");
        }
        m->own_stream = true;
    }
    auto fail = [&](const char *msg) {
        hyb_switchnet_destroy(m);
        return set_error(HYB_ENOMEM, msg);
    };
    for (int l = 0; l <= SN_L; ++l) {
        const size_t nw = (size_t)sn_co(l) * sn_ci(l), nb = (size_t)(l < SN_L ? SN_CO[l] : 1);
        if (sn_alloc(m, (void **)&m->w[l], sizeof(float) * nw) || sn_alloc(m, (void **)&m->b[l], sizeof(float) * nb) ||
            sn_alloc(m, (void **)&m->mw[l], sizeof(float) * nw) || sn_alloc(m, (void **)&m->vw[l], sizeof(float) * nw) ||
            sn_alloc(m, (void **)&m->mb[l], sizeof(float) * nb) || sn_alloc(m, (void **)&m->vb[l], sizeof(float) * nb) ||
            sn_alloc(m, (void **)&m->gw[l], sizeof(float) * nw) || sn_alloc(m, (void **)&m->gb[l], sizeof(float) * nb))
            return fail("switchnet allocation");
        cudaMemsetAsync(m->mw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->vw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->mb[l], 0, sizeof(float) * nb, m->stream);
        cudaMemsetAsync(m->vb[l], 0, sizeof(float) * nb, m->stream);
        cudaMemsetAsync(m->gw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->gb[l], 0, sizeof(float) * nb, m->stream);
    }
    for (int l = 0; l < SN_L; ++l) {
        for (int s = 0; s < SN_CO[l] / 128; ++s)
            if (sn_alloc(m, (void **)&m->pk[l][s], sizeof(__nv_bfloat16) * SN_KP[l] * 128)) return fail("switchnet allocation");
        if (l > 0)
            for (int s = 0; s < SN_CI[l] / 128; ++s)
                if (sn_alloc(m, (void **)&m->pkT[l][s], sizeof(__nv_bfloat16) * SN_CO[l] * 128))
                    return fail("switchnet allocation");
    }
    if (sn_alloc(m, (void **)&m->mean, sizeof(float) * NF) || sn_alloc(m, (void **)&m->std_, sizeof(float) * NF) ||
        sn_alloc(m, (void **)&m->status, sizeof(int)) || sn_alloc(m, (void **)&m->wsum, sizeof(float) * (1024 + 32)) ||
        sn_alloc(m, (void **)&m->lpart, sizeof(double) * 3 * m->lblocks))
        return fail("switchnet allocation");
    cudaMemcpyAsync(m->mean, d->mean, sizeof(float) * NF, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->std_, d->std, sizeof(float) * NF, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->status, 0, sizeof(int), m->stream);
    // He-uniform initialisation from the seed (Philox on the host), zero biases
    for (int l = 0; l <= SN_L; ++l) {
        const size_t nw = (size_t)sn_co(l) * sn_ci(l);
        std::vector<float> w(nw), b((size_t)sn_co(l), 0.0f);
        const float lim = std::sqrt(6.0f / (float)sn_ci(l));
        for (size_t i = 0; i < nw; ++i) {
            const u32x4 r = philox4x32_10((uint32_t)i, (uint32_t)l, 0x5317u, 0u, d->seed, 0xA3u);
            w[i] = (2.0f * u01f(r.v[0]) - 1.0f) * lim;
        }
        cudaMemcpy(m->w[l], w.data(), sizeof(float) * nw, cudaMemcpyHostToDevice);
        cudaMemcpy(m->b[l], b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice);
    }
    hyb_status s = sn_repack(m);
    if (s == HYB_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) s = set_error(HYB_ECUDA, "switchnet init");
    if (s != HYB_OK) {
        hyb_switchnet_destroy(m);
        return s;
    }
    *out = m;
    return HYB_OK;
}

hyb_status hyb_switchnet_set_layer(hyb_switchnet *m, int l, const float *w_host, const float *b_host) {
    if (!m || l < 0 || l > SN_L || !w_host || !b_host) return set_error(HYB_EINVAL, "bad argument");
    HYB_CUDA_TRY(cudaMemcpyAsync(m->w[l], w_host, sizeof(float) * sn_co(l) * sn_ci(l), cudaMemcpyHostToDevice, m->stream));
    HYB_CUDA_TRY(cudaMemcpyAsync(m->b[l], b_host, sizeof(float) * sn_co(l), cudaMemcpyHostToDevice, m->stream));
    hyb_status s = sn_repack(m);
    if (s != HYB_OK) return s;
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_switchnet_get_layer(hyb_switchnet *m, int l, float *w_host, float *b_host) {
    if (!m || l < 0 || l > SN_L) return set_error(HYB_EINVAL, "bad argument");
    if (w_host)
        HYB_CUDA_TRY(cudaMemcpyAsync(w_host, m->w[l], sizeof(float) * sn_co(l) * sn_ci(l), cudaMemcpyDeviceToHost, m->stream));
    if (b_host) HYB_CUDA_TRY(cudaMemcpyAsync(b_host, m->b[l], sizeof(float) * sn_co(l), cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_switchnet_get_grad(hyb_switchnet *m, int l, float *gw, float *gb) {
    if (!m || l < 0 || l > SN_L || m->adam_t == 0) return set_error(HYB_EINVAL, "no gradients (no training step yet)");
    if (gw) HYB_CUDA_TRY(cudaMemcpyAsync(gw, m->gw[l], sizeof(float) * sn_co(l) * sn_ci(l), cudaMemcpyDeviceToHost, m->stream));
    if (gb) HYB_CUDA_TRY(cudaMemcpyAsync(gb, m->gb[l], sizeof(float) * sn_co(l), cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_switchnet_forward(hyb_switchnet *m, const float *x, long long n, int pass, float *logit) {
    if (!m || !x || !logit) return set_error(HYB_EINVAL, "null argument");
    hyb_status s = sn_check(m, n);
    if (s != HYB_OK) return s;
    k_sn_prep<<<nbs(n), RBS, 0, m->stream>>>(x, n, m->mean, m->std_, m->a[0]);
    if ((s = sn_forward(m, n, pass)) != HYB_OK) return s;
    HYB_CUDA_TRY(cudaMemcpyAsync(logit, m->logit, sizeof(float) * n, cudaMemcpyDeviceToDevice, m->stream));
    return HYB_OK;
}

hyb_status hyb_switchnet_mc(hyb_switchnet *m, const float *x, long long n, float *pm, float *ps) {
    if (!m || !x || !pm || !ps) return set_error(HYB_EINVAL, "null argument");
    hyb_status s = sn_check(m, n);
    if (s != HYB_OK) return s;
    k_sn_prep<<<nbs(n), RBS, 0, m->stream>>>(x, n, m->mean, m->std_, m->a[0]);
    const int K = m->d.mc_passes;
    for (int k = 1; k <= K; ++k) {
        if ((s = sn_forward(m, n, k - 1)) != HYB_OK) return s;
        k_sn_mc<<<nbs(n), RBS, 0, m->stream>>>(m->logit, n, k, pm, ps);
    }
    k_sn_mc_final<<<nbs(n), RBS, 0, m->stream>>>(n, K, ps);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

hyb_status hyb_switchnet_train_step(hyb_switchnet *m, const float *x, const float *y, long long n,
                                    hyb_train_stats *out) {
    if (!m || !x || !y || !out) return set_error(HYB_EINVAL, "null argument");
    hyb_status s = sn_check(m, n);
    if (s != HYB_OK) return s;
    cudaStream_t st = m->stream;
    const int pass = (int)(m->adam_t & 0x7fffffff);
    k_sn_prep<<<nbs(n), RBS, 0, st>>>(x, n, m->mean, m->std_, m->a[0]);
    if ((s = sn_forward(m, n, pass)) != HYB_OK) return s;
    // energy-weighted BCE (the classifier's loss) with its gradient
    k_energy_density<<<m->lblocks, RBS, 0, st>>>(x, 1, n, m->edens, m->lpart);
    std::vector<double> hp((size_t)3 * m->lblocks);
    HYB_CUDA_TRY(cudaMemcpyAsync(hp.data(), m->lpart, sizeof(double) * m->lblocks, cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));
    double esum = 0.0;
    for (int k = 0; k < m->lblocks; ++k) esum += hp[k];
    const double emean = esum / (double)n;
    k_loss<<<m->lblocks, RBS, 0, st>>>(m->logit, y, m->edens, emean > 0.0 ? (float)(1.0 / emean) : 0.0f,
                                       (float)m->d.energy_weight, n, m->dlogit, m->lpart);
    // output layer: weight gradient from bf16(dlogit), data gradient dz3
    k_sn_dlast<<<nbs(n * 32), RBS, 0, st>>>(m->dlogit, m->w[SN_L], n, m->dz, m->dl16);
    sn_wgrad(m, m->a[SN_L], 256, 256, m->dl16, 8, 1, n, m->gw[SN_L], m->gb[SN_L]);
    // layers 3 .. 0; G holds dL/d a[l + 1] (FP32), dz the BF16 operand
    float *G = nullptr;
    for (int l = SN_L - 1; l >= 0; --l) {
        if (l < SN_L - 1)
            k_act_dz<<<nbs(n * (SN_CO[l] / 8)), RBS, 0, st>>>(G, m->z[l], m->b[l], SN_CO[l], SN_RELU[l],
                                                              sn_drop(m, l, pass), 1, n, m->dz);
        for (int co0 = 0; co0 < SN_CO[l]; co0 += 128) {
            WgradJob j;
            memset(&j, 0, sizeof(j));
            j.x = m->a[l];
            j.x_pitch = SN_KP[l];
            j.ci_n = SN_CI[l];
            j.ci_tot = SN_CI[l];
            j.dz = m->dz;
            j.dz_pitch = SN_CO[l];
            j.co0 = co0;
            j.co_n = 128;
            j.B = j.D = j.H = 1;
            j.W = (int)n;
            j.taps = 1;
            j.gw = m->gw[l];
            j.gb = m->gb[l];
            j.status = m->status;
            if ((s = wgrad_tc(j, *m->wg, st)) != HYB_OK) return s;
        }
        if (l > 0) {
            float *Gn = (G == m->G1) ? m->G2 : m->G1;
            if ((s = sn_gemm(m, m->dz, SN_CO[l], m->pkT[l], SN_CI[l] / 128, Gn, SN_CI[l], n)) != HYB_OK) return s;
            if (SN_RES[l]) k_sn_addres<<<nbs(n * SN_CI[l]), RBS, 0, st>>>(Gn, SN_CI[l], G, SN_CO[l], SN_CI[l], n);
            G = Gn;
        }
    }
    m->adam_t += 1;
    const float b1 = (float)m->d.beta1, b2 = (float)m->d.beta2;
    const float c1 = (float)(1.0 - std::pow(m->d.beta1, (double)m->adam_t));
    const float c2 = (float)(1.0 - std::pow(m->d.beta2, (double)m->adam_t));
    for (int l = 0; l <= SN_L; ++l) {
        const int nw = sn_co(l) * sn_ci(l);
        k_adam<<<nbs(nw), RBS, 0, st>>>(m->w[l], m->gw[l], m->mw[l], m->vw[l], nw, (float)m->d.lr, b1, b2,
                                        (float)m->d.eps, c1, c2);
        k_adam<<<nbs(sn_co(l)), RBS, 0, st>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], sn_co(l), (float)m->d.lr, b1, b2,
                                              (float)m->d.eps, c1, c2);
    }
    if ((s = sn_repack(m)) != HYB_OK) return s;
    HYB_CUDA_TRY(cudaMemcpyAsync(hp.data(), m->lpart, sizeof(double) * 3 * m->lblocks, cudaMemcpyDeviceToHost, st));
    int stw = 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(&stw, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));
    if (stw) return set_error(HYB_ETIMEOUT, "a tensor-core wait gave up");
    double L = 0, bce = 0, acc = 0;
    for (int k = 0; k < m->lblocks; ++k) {
        L += hp[3 * k];
        bce += hp[3 * k + 1];
        acc += hp[3 * k + 2];
    }
    out->loss = L / (double)n;
    out->bce = bce / (double)n;
    out->accuracy = acc / (double)n;
    out->step = m->adam_t;
    return HYB_OK;
}

}  // extern "C"
