// Field surrogate (arXiv 2510.11174, Results and Table 2: the StatePredictor,
// a 3D convolutional network with residual connections and dropout that
// predicts the plasma state from the per-channel normalised E, B, J and rho
// of a patch, trained with a Huber loss and a penalty on energy violation).
//
// The six 3x3x3 convolutions run on the classifier's tcgen05 kernel
// (k_conv3_tc) in channel chunks: one launch contracts 16 or 32 input
// channels into 16 or 32 output channels and adds its raw sums into the
// layer's FP32 pre-activation buffer (k_conv3_tc's accumulate mode); a
// finishing kernel adds the bias, applies ReLU, dropout and the identity
// shortcut, and stores the BF16 activation.  The data gradient is the same
// convolution with the transposed, flipped kernel; the weight gradient is the
// tensor-core contraction over the cells (wgrad_tc) in blocks of 32 x 32 channels;
// Adam updates FP32 masters.  See hyb_surrogate_* in include/hyb.h.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"
#include "philox.cuh"

namespace hyb {

// ---------------------------------------------------------------- activations shared by the per-layer networks
// keep bits (one per channel, bit j for channel 8 grp + j) of the dropout
// stream: Philox counter (cell, batch, layer << 16 | grp, pass), key (seed,
// 0xD0); channel j keeps when its 16-bit field is >= thr
__device__ __forceinline__ uint32_t keep_bits(uint32_t lin, uint32_t b, uint32_t layer, uint32_t grp, uint32_t pass,
                                              uint32_t seed, uint32_t thr) {
    const u32x4 r = philox4x32_10(lin, b, (layer << 16) | grp, pass, seed, 0xD0u);
    uint32_t k = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) k |= (((r.v[j >> 1] >> (16 * (j & 1))) & 0xFFFFu) >= thr ? 1u : 0u) << j;
    return k;
}

// a = relu(s + b) [dropout] [+ res]: one thread per cell and 8-channel group;
// BF16 out (hidden layers) or FP32 out (the last layer, no ReLU)
__global__ void k_act_finish(const float *__restrict__ s, const float *__restrict__ bias, int cop, int relu,
                             const __nv_bfloat16 *__restrict__ res, int cres, DropArgs dr, int B, long long V,
                             __nv_bfloat16 *__restrict__ out, float *__restrict__ outf) {
    const int ng = cop / 8;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V * ng) return;
    const long long cell = t / ng;
    const int grp = (int)(t % ng);
    const uint32_t keep = dr.thr ? keep_bits((uint32_t)(cell % V), (uint32_t)(cell / V), dr.layer, (uint32_t)grp,
                                             dr.pass, dr.seed, dr.thr)
                                 : 0xFFu;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int ch = grp * 8 + j;
        float a = s[cell * cop + ch] + bias[ch];
        if (relu) a = fmaxf(a, 0.0f);
        if (dr.thr) a = ((keep >> j) & 1u) ? a * dr.scale : 0.0f;
        if (res && ch < cres) a += __bfloat162float(res[cell * cres + ch]);
        v[j] = a;
    }
    if (outf) {
        float4 *o4 = reinterpret_cast<float4 *>(outf + cell * cop + grp * 8);
        o4[0] = make_float4(v[0], v[1], v[2], v[3]);
        o4[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(v[j]);
        *reinterpret_cast<uint4 *>(out + cell * cop + grp * 8) = *reinterpret_cast<const uint4 *>(o);
    }
}

// dz = bf16(G [s + b > 0] keep / (1 - p)): the data gradient at layer l's
// pre-activation from the gradient G of its output; one thread per cell and
// 8-channel group
__global__ void k_act_dz(const float *__restrict__ G, const float *__restrict__ s, const float *__restrict__ bias,
                         int cop, int relu, DropArgs dr, int B, long long V, __nv_bfloat16 *__restrict__ dz) {
    const int ng = cop / 8;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V * ng) return;
    const long long cell = t / ng;
    const int grp = (int)(t % ng);
    const uint32_t keep = dr.thr ? keep_bits((uint32_t)(cell % V), (uint32_t)(cell / V), dr.layer, (uint32_t)grp,
                                             dr.pass, dr.seed, dr.thr)
                                 : 0xFFu;
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long i = cell * cop + grp * 8 + j;
        float g = G[i];
        if (relu && !(s[i] + bias[grp * 8 + j] > 0.0f)) g = 0.0f;
        if (dr.thr) g = ((keep >> j) & 1u) ? g * dr.scale : 0.0f;
        o[j] = __float2bfloat16_rn(g);
    }
    *reinterpret_cast<uint4 *>(dz + cell * cop + grp * 8) = *reinterpret_cast<const uint4 *>(o);
}

namespace {

constexpr int SL = 6;                                            // convolutions
constexpr int CI[SL] = {10, 13, 32, 64, 128, 32}, CO[SL] = {13, 32, 64, 128, 32, 10};
constexpr int CIP[SL] = {16, 16, 32, 64, 128, 32}, COP[SL] = {16, 32, 64, 128, 32, 16};  // padded to 16
constexpr int RES[SL] = {1, 1, 1, 0, 0, 0};                      // identity shortcut (zero-padded channels)
constexpr int RELU[SL] = {1, 1, 1, 1, 1, 0};
constexpr int DROP_LAYER = 1;                                    // dropout after layer 1's ReLU
constexpr int NCH = 10;                                          // state channels: E, B, J, rho
constexpr int RB = 256;

inline int chunk_of(int c) { return c % 32 == 0 ? 32 : 16; }
inline unsigned nbk(long long n, int b = RB) { return (unsigned)((n + b - 1) / b); }

// states [B][10][V] FP32 -> normalised BF16 channels-last [B][V][16]
__global__ void k_sur_prep(const float *__restrict__ x, int B, long long V, const float *__restrict__ mean,
                           const float *__restrict__ sd, __nv_bfloat16 *__restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V) return;
    const long long b = t / V, v = t % V;
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(c < NCH ? (x[(b * NCH + c) * V + v] - mean[c]) / sd[c] : 0.0f);
    uint4 *dst = reinterpret_cast<uint4 *>(out + t * 16);
    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// prediction [B][10][V] = x + dstd_c y (y [B][V][16]: the change in units of its spread)
__global__ void k_sur_out(const float *__restrict__ y, const float *__restrict__ x, int B, long long V,
                          const float *__restrict__ sd, float *__restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V * NCH) return;
    const long long b = t / (V * NCH), c = (t / V) % NCH, v = t % V;
    out[t] = x[t] + y[(b * V + v) * 16 + c] * sd[c];
}

// MC statistics: pass k (1-based) folded into the running mean and M2 (Welford)
__global__ void k_sur_mc(const float *__restrict__ y, const float *__restrict__ x, int B, long long V,
                         const float *__restrict__ sd, int k, float *__restrict__ pm, float *__restrict__ m2) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V * NCH) return;
    const long long b = t / (V * NCH), c = (t / V) % NCH, v = t % V;
    const float val = x[t] + y[(b * V + v) * 16 + c] * sd[c];
    if (k == 1) {
        pm[t] = val;
        m2[t] = 0.0f;
    } else {
        const float d = val - pm[t];
        const float mu = pm[t] + d / (float)k;
        pm[t] = mu;
        m2[t] += d * (val - mu);
    }
}

__global__ void k_sur_mc_final(long long n, int k, float *__restrict__ m2) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) m2[t] = sqrtf(fmaxf(m2[t], 0.0f) / (float)k);
}

__device__ __forceinline__ double blk_sum(double v, double *sh) {
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

// per-sample field energies of prediction and target (de-normalised channels
// 0..5): grid (blocks, B), part[b][blk][2]
__global__ void __launch_bounds__(RB) k_sur_energy(const float *__restrict__ y, const float *__restrict__ tg,
                                                   const float *__restrict__ x, long long V,
                                                   const float *__restrict__ sd, double *__restrict__ part) {
    __shared__ double sh[RB];
    const int b = blockIdx.y;
    double wp = 0.0, wt = 0.0;
    for (long long v = blockIdx.x * (long long)RB + threadIdx.x; v < V; v += (long long)gridDim.x * RB) {
        float sp = 0.0f, st = 0.0f;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float p = x[((long long)b * NCH + c) * V + v] + y[((long long)b * V + v) * 16 + c] * sd[c];
            const float q = tg[((long long)b * NCH + c) * V + v];
            sp += p * p;
            st += q * q;
        }
        wp += 0.5 * (double)sp;
        wt += 0.5 * (double)st;
    }
    wp = blk_sum(wp, sh);
    wt = blk_sum(wt, sh);
    if (threadIdx.x == 0) {
        part[((long long)b * gridDim.x + blockIdx.x) * 2 + 0] = wp;
        part[((long long)b * gridDim.x + blockIdx.x) * 2 + 1] = wt;
    }
}

// esum[b][2] = the partials of sample b summed in block order
__global__ void k_sur_esum(const double *__restrict__ part, int B, int nblk, double *__restrict__ esum) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double wp = 0.0, wt = 0.0;
    for (int k = 0; k < nblk; ++k) {
        wp += part[((long long)b * nblk + k) * 2 + 0];
        wt += part[((long long)b * nblk + k) * 2 + 1];
    }
    esum[2 * b] = wp;
    esum[2 * b + 1] = wt;
}

// loss gradient dL/dy (FP32 G and its BF16 copy dz, [cells][16]) and the
// Huber partial sums
__global__ void __launch_bounds__(RB) k_sur_loss(const float *__restrict__ y, const float *__restrict__ tg,
                                                 const float *__restrict__ x, int B, long long V,
                                                 const float *__restrict__ sd, float delta, float lam,
                                                 const double *__restrict__ esum, float *__restrict__ G,
                                                 __nv_bfloat16 *__restrict__ dz, double *__restrict__ part) {
    __shared__ double sh[RB];
    const double inv_n = 1.0 / ((double)B * (double)V * NCH);
    // the batch's total energies; d(v^2)/dW_pred,b = 2 v / W_true,tot with
    // v = (W_pred,tot - W_true,tot) / W_true,tot (no energy term for W_true,tot = 0)
    double wp = 0.0, wt = 0.0;
    for (int b = 0; b < B; ++b) {
        wp += esum[2 * b];
        wt += esum[2 * b + 1];
    }
    const float ecoef = wt > 0.0 ? (float)(2.0 * (wp - wt) / (wt * wt)) : 0.0f;
    double hs = 0.0;
    for (long long t = blockIdx.x * (long long)RB + threadIdx.x; t < (long long)B * V;
         t += (long long)gridDim.x * RB) {
        const long long b = t / V, v = t % V;
        __align__(16) float g[16];
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float gc = 0.0f;
            if (c < NCH) {
                const float yc = y[t * 16 + c];
                const float xc = x[(b * NCH + c) * V + v];
                const float tn = (tg[(b * NCH + c) * V + v] - xc) / sd[c];
                const float r = yc - tn, ar = fabsf(r);
                hs += ar <= delta ? 0.5 * (double)r * r : (double)delta * ((double)ar - 0.5 * delta);
                gc = (ar <= delta ? r : copysignf(delta, r)) * (float)inv_n;
                if (c < 6) gc += lam * ecoef * sd[c] * (xc + yc * sd[c]);
            }
            g[c] = gc;
            o[c] = __float2bfloat16_rn(gc);
        }
        float4 *g4 = reinterpret_cast<float4 *>(G + t * 16);
#pragma unroll
        for (int q = 0; q < 4; ++q) g4[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
        uint4 *d4 = reinterpret_cast<uint4 *>(dz + t * 16);
        d4[0] = reinterpret_cast<const uint4 *>(o)[0];
        d4[1] = reinterpret_cast<const uint4 *>(o)[1];
    }
    hs = blk_sum(hs, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = hs;
}

// the shortcut's share of the data gradient: G_in[c][ch] += G_out[c][ch] for ch < cin
__global__ void k_sur_addres(float *__restrict__ Gin, const float *__restrict__ Gout, int cin, int cout,
                             long long cells) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cells * cin) return;
    const long long cell = t / cin;
    const int ch = (int)(t % cin);
    Gin[t] += Gout[cell * cout + ch];
}

// channel-chunk packs of a layer's weights W [co][ci][27] for k_conv3_tc:
// block (ic, os) holds input channels ic*cic .. and outputs os*nsl .. in the
// core layout [9 (dz, dy)][cic/8][3 (dx) nsl][8]; transposed packs (the data
// gradient) take the output channels as inputs and the taps flipped
__global__ void k_sur_pack(const float *__restrict__ W, int ci_n, int co_n, int nin, int nout, int cic, int nsl,
                           int transpose, __nv_bfloat16 *__restrict__ out) {
    const long long blk = 27LL * cic * nsl;
    const long long total = (long long)(nin / cic) * (nout / nsl) * blk;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int nos = nout / nsl;
    const long long bi = t / blk, e = t % blk;
    const int ic = (int)(bi / nos), os = (int)(bi % nos);
    const int j = (int)(e % 8), nn = (int)((e / 8) % (3 * nsl)), kc = (int)((e / (8 * 3 * nsl)) % (cic / 8));
    const int tap9 = (int)(e / (8LL * 3 * nsl * (cic / 8)));
    const int dx = nn / nsl, n = nn % nsl, tap = tap9 * 3 + dx;
    const int cin_ch = ic * cic + kc * 8 + j, cout_ch = os * nsl + n;
    float v = 0.0f;
    if (!transpose) {
        if (cin_ch < ci_n && cout_ch < co_n) v = W[((long long)cout_ch * ci_n + cin_ch) * 27 + tap];
    } else {
        // input channel = the layer's output co, output channel = its input ci
        if (cin_ch < co_n && cout_ch < ci_n) v = W[((long long)cin_ch * ci_n + cout_ch) * 27 + (26 - tap)];
    }
    out[t] = __float2bfloat16_rn(v);
}

// summed weight-gradient block [tap][ci][co] (ci_n x co_n) -> gw[co0 + co][ci0 + ci][tap]
__global__ void k_sur_scatter_wg(const float *__restrict__ in, int ci_n, int co_n, int ci0, int co0, int CItot,
                                 float *__restrict__ gw) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= 27 * ci_n * co_n) return;
    const int co = o % co_n, ci = (o / co_n) % ci_n, tap = o / (co_n * ci_n);
    gw[((long long)(co0 + co) * CItot + ci0 + ci) * 27 + tap] = in[o];
}

}  // namespace
}  // namespace hyb

using namespace hyb;

struct hyb_surrogate {
    hyb_surrogate_desc d;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *w[SL] = {}, *b[SL] = {};                   // FP32 masters: [co][ci][27], [COP] (zero-padded)
    float *mw[SL] = {}, *vw[SL] = {}, *mb[SL] = {}, *vb[SL] = {};
    float *gw[SL] = {}, *gb[SL] = {};                 // gradients of the last step
    __nv_bfloat16 *pk[SL] = {}, *pkT[SL] = {};        // channel-chunk packs (forward, data gradient)
    float *mean = nullptr, *std_ = nullptr, *dstd = nullptr;  // dstd: unit of the predicted change
    int *status = nullptr;
    long long cap = 0;                                // cells the activation buffers hold
    __nv_bfloat16 *a[SL] = {};                        // a[l]: input of layer l, [cells][CIP[l]]
    float *s[SL] = {};                                // pre-activation sums of layer l (no bias), [cells][COP[l]]
    float *G[SL + 1] = {};                            // G[l]: dL/d a[l] ([cells][CIP[l]]), G[SL] = dL/dy
    float *y = nullptr;                               // prediction [cells][16] (normalised)
    __nv_bfloat16 *dz = nullptr;                      // data gradient of the current layer, [cells][<= 128]
    WgradScratch *wg = nullptr;                       // operands of the tensor-core weight gradients
    double *lpart = nullptr, *epart = nullptr, *esum = nullptr;
    int lblocks = 2 * 152, eblocks = 64, ecap = 0;
    long long adam_t = 0;
    std::vector<void *> owned;
};

namespace {

cudaError_t s_alloc(hyb_surrogate *m, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) m->owned.push_back(*p);
    return e;
}

void s_free(hyb_surrogate *m, void *p) {
    if (!p) return;
    for (auto it = m->owned.begin(); it != m->owned.end(); ++it)
        if (*it == p) {
            m->owned.erase(it);
            break;
        }
    cudaFree(p);
}

hyb_status repack(hyb_surrogate *m) {
    for (int l = 0; l < SL; ++l) {
        const long long tot = 27LL * CIP[l] * COP[l];
        k_sur_pack<<<nbk(tot), RB, 0, m->stream>>>(m->w[l], CI[l], CO[l], CIP[l], COP[l], chunk_of(CIP[l]),
                                                   chunk_of(COP[l]), 0, m->pk[l]);
        k_sur_pack<<<nbk(tot), RB, 0, m->stream>>>(m->w[l], CI[l], CO[l], COP[l], CIP[l], chunk_of(COP[l]),
                                                   chunk_of(CIP[l]), 1, m->pkT[l]);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("surrogate packing: ") + cudaGetErrorString(e));
    return HYB_OK;
}

hyb_status reserve(hyb_surrogate *m, long long cells) {
    if (cells <= m->cap) return HYB_OK;
    cudaStreamSynchronize(m->stream);  // buffers are replaced only between stream-ordered uses
    for (int l = 0; l < SL; ++l) {
        s_free(m, m->a[l]);
        s_free(m, m->s[l]);
        m->a[l] = nullptr;
        m->s[l] = nullptr;
    }
    for (int l = 0; l <= SL; ++l) {
        s_free(m, m->G[l]);
        m->G[l] = nullptr;
    }
    s_free(m, m->y);
    s_free(m, m->dz);
    m->cap = 0;
    for (int l = 0; l < SL; ++l)
        if (s_alloc(m, (void **)&m->a[l], sizeof(__nv_bfloat16) * CIP[l] * cells) ||
            s_alloc(m, (void **)&m->s[l], sizeof(float) * COP[l] * cells) ||
            (l > 0 && s_alloc(m, (void **)&m->G[l], sizeof(float) * CIP[l] * cells)))
            return set_error(HYB_ENOMEM, "surrogate activation buffers");
    if (s_alloc(m, (void **)&m->G[SL], sizeof(float) * 16 * cells) || s_alloc(m, (void **)&m->y, sizeof(float) * 16 * cells) ||
        s_alloc(m, (void **)&m->dz, sizeof(__nv_bfloat16) * 128 * cells))
        return set_error(HYB_ENOMEM, "surrogate activation buffers");
    m->cap = cells;
    return HYB_OK;
}

// acc [cells][nout] (zeroed) += conv(x [cells][nin]; the packs pk) in channel chunks
hyb_status conv_chunks(hyb_surrogate *m, const __nv_bfloat16 *x, int nin, const __nv_bfloat16 *pk, int nout,
                       float *acc, int B, int D, int H, int W) {
    const int cic = chunk_of(nin), nsl = chunk_of(nout), nos = nout / nsl;
    const long long blk = 27LL * cic * nsl;
    for (int ic = 0; ic < nin / cic; ++ic)
        for (int os = 0; os < nos; ++os) {
            ConvArgs a;
            memset(&a, 0, sizeof(a));
            a.x = x;
            a.wt = pk + (ic * nos + os) * blk;
            a.B = B;
            a.D = D;
            a.H = H;
            a.W = W;
            a.cin = cic;
            a.cin_total = nin;
            a.cin_off = ic * cic;
            a.N = nsl;
            a.y_f32 = acc;
            a.out_pitch = nout;
            a.out_off = os * nsl;
            a.accum = 1;
            a.status = m->status;
            hyb_status st = launch_conv3_tc(a, m->stream);
            if (st != HYB_OK) return st;
        }
    return HYB_OK;
}

DropArgs drop_of(const hyb_surrogate *m, int l, int pass) {
    DropArgs dr;
    memset(&dr, 0, sizeof(dr));
    if (l == DROP_LAYER && pass >= 0) {
        dr.thr = dropout_threshold(m->d.dropout);
        dr.scale = dropout_scale(dr.thr);
        dr.seed = m->d.seed;
        dr.pass = (uint32_t)pass;
        dr.layer = (uint32_t)l;
    }
    return dr;
}

// forward pass of prepared inputs m->a[0] -> m->y
hyb_status forward(hyb_surrogate *m, int B, int D, int H, int W, int pass) {
    const long long V = (long long)D * H * W, cells = (long long)B * V;
    for (int l = 0; l < SL; ++l) {
        cudaMemsetAsync(m->s[l], 0, sizeof(float) * COP[l] * cells, m->stream);
        hyb_status st = conv_chunks(m, m->a[l], CIP[l], m->pk[l], COP[l], m->s[l], B, D, H, W);
        if (st != HYB_OK) return st;
        const bool last = l == SL - 1;
        k_act_finish<<<nbk(cells * (COP[l] / 8)), RB, 0, m->stream>>>(
            m->s[l], m->b[l], COP[l], RELU[l], RES[l] ? m->a[l] : nullptr, CIP[l], drop_of(m, l, pass), B, V,
            last ? nullptr : m->a[l + 1], last ? m->y : nullptr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("surrogate forward: ") + cudaGetErrorString(e));
    return HYB_OK;
}

hyb_status check_shape(int B, int D, int H, int W) {
    if (B <= 0 || D <= 0 || H <= 0 || W <= 0) return set_error(HYB_EINVAL, "bad patch shape");
    if (W % 8 != 0 || H % 16 != 0) return set_error(HYB_EINVAL, "the surrogate needs W % 8 == 0 and H % 16 == 0");
    return HYB_OK;
}

hyb_status read_status(hyb_surrogate *m) {
    int stw = 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(&stw, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (stw) return set_error(HYB_ETIMEOUT, "a tensor-core wait gave up");
    return HYB_OK;
}

// weight and bias gradient of layer l on the tensor cores, from its input
// a[l] and the BF16 data gradient dz, in blocks of 32 x 32 channels
hyb_status layer_wgrad(hyb_surrogate *m, int l, int B, int D, int H, int W) {
    for (int ci0 = 0; ci0 < CI[l]; ci0 += 32)
        for (int co0 = 0; co0 < CO[l]; co0 += 32) {
            WgradJob j;
            memset(&j, 0, sizeof(j));
            j.x = m->a[l];
            j.x_pitch = CIP[l];
            j.ci0 = ci0;
            j.ci_n = CI[l] - ci0 < 32 ? CI[l] - ci0 : 32;
            j.ci_tot = CI[l];
            j.dz = m->dz;
            j.dz_pitch = COP[l];
            j.co0 = co0;
            j.co_n = CO[l] - co0 < 32 ? CO[l] - co0 : 32;
            j.B = B;
            j.D = D;
            j.H = H;
            j.W = W;
            j.taps = 27;
            j.gw = m->gw[l];
            j.gb = ci0 == 0 ? m->gb[l] : nullptr;
            j.status = m->status;
            hyb_status s = wgrad_tc(j, *m->wg, m->stream);
            if (s != HYB_OK) return s;
        }
    return HYB_OK;
}

}  // namespace

extern "C" {

void hyb_surrogate_destroy(hyb_surrogate *m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void *p : m->owned) cudaFree(p);
    delete m->wg;
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

hyb_status hyb_surrogate_create(const hyb_surrogate_desc *d, hyb_surrogate **out) {
    if (!d || !out) return set_error(HYB_EINVAL, "null argument");
    *out = nullptr;
    if (!(d->dropout >= 0.0 && d->dropout < 1.0)) return set_error(HYB_EINVAL, "dropout must be in [0, 1)");
    for (int c = 0; c < NCH; ++c)
        if (!(d->std[c] > 0.0f)) return set_error(HYB_EINVAL, "normalisation std must be > 0");
    hyb_surrogate *m = new hyb_surrogate();
    m->wg = new WgradScratch();
    m->d = *d;
    m->d.dropout = dropout_threshold(d->dropout) / 65536.0;
    if (!(m->d.lr > 0)) m->d.lr = 1e-3;
    if (!(m->d.beta1 > 0)) m->d.beta1 = 0.9;
    if (!(m->d.beta2 > 0)) m->d.beta2 = 0.999;
    if (!(m->d.eps > 0)) m->d.eps = 1e-8;
    if (!(m->d.huber_delta > 0)) m->d.huber_delta = 0.01;
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
        hyb_surrogate_destroy(m);
        return set_error(HYB_ENOMEM, msg);
    };
    for (int l = 0; l < SL; ++l) {
        const size_t nw = (size_t)CO[l] * CI[l] * 27;
        if (s_alloc(m, (void **)&m->w[l], sizeof(float) * nw) || s_alloc(m, (void **)&m->b[l], sizeof(float) * COP[l]) ||
            s_alloc(m, (void **)&m->mw[l], sizeof(float) * nw) || s_alloc(m, (void **)&m->vw[l], sizeof(float) * nw) ||
            s_alloc(m, (void **)&m->mb[l], sizeof(float) * COP[l]) || s_alloc(m, (void **)&m->vb[l], sizeof(float) * COP[l]) ||
            s_alloc(m, (void **)&m->gw[l], sizeof(float) * nw) || s_alloc(m, (void **)&m->gb[l], sizeof(float) * COP[l]) ||
            s_alloc(m, (void **)&m->pk[l], sizeof(__nv_bfloat16) * 27 * CIP[l] * COP[l]) ||
            s_alloc(m, (void **)&m->pkT[l], sizeof(__nv_bfloat16) * 27 * CIP[l] * COP[l]))
            return fail("surrogate allocation");
        cudaMemsetAsync(m->mw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->vw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->mb[l], 0, sizeof(float) * COP[l], m->stream);
        cudaMemsetAsync(m->vb[l], 0, sizeof(float) * COP[l], m->stream);
        cudaMemsetAsync(m->gw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->gb[l], 0, sizeof(float) * COP[l], m->stream);
    }
    if (s_alloc(m, (void **)&m->mean, sizeof(float) * NCH) || s_alloc(m, (void **)&m->std_, sizeof(float) * NCH) ||
        s_alloc(m, (void **)&m->dstd, sizeof(float) * NCH) ||
        s_alloc(m, (void **)&m->status, sizeof(int)) || s_alloc(m, (void **)&m->lpart, sizeof(double) * m->lblocks))
        return fail("surrogate allocation");
    cudaMemcpyAsync(m->mean, d->mean, sizeof(float) * NCH, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->std_, d->std, sizeof(float) * NCH, cudaMemcpyHostToDevice, m->stream);
    for (int c = 0; c < NCH; ++c) m->d.dstd[c] = d->dstd[c] > 0.0f ? d->dstd[c] : d->std[c];
    cudaMemcpyAsync(m->dstd, m->d.dstd, sizeof(float) * NCH, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->status, 0, sizeof(int), m->stream);
    // He-uniform initialisation from the seed (Philox on the host):
    // w ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)), b = 0
    for (int l = 0; l < SL; ++l) {
        const size_t nw = (size_t)CO[l] * CI[l] * 27;
        std::vector<float> w(nw), b(COP[l], 0.0f);
        const float lim = std::sqrt(6.0f / (float)(CI[l] * 27));
        for (size_t i = 0; i < nw; ++i) {
            const u32x4 r = philox4x32_10((uint32_t)i, (uint32_t)l, 0x5122u, 0u, d->seed, 0xA2u);
            w[i] = (2.0f * u01f(r.v[0]) - 1.0f) * lim;
        }
        cudaMemcpy(m->w[l], w.data(), sizeof(float) * nw, cudaMemcpyHostToDevice);
        cudaMemcpy(m->b[l], b.data(), sizeof(float) * COP[l], cudaMemcpyHostToDevice);
    }
    hyb_status s = repack(m);
    if (s == HYB_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) s = set_error(HYB_ECUDA, "surrogate init");
    if (s != HYB_OK) {
        hyb_surrogate_destroy(m);
        return s;
    }
    *out = m;
    return HYB_OK;
}

hyb_status hyb_surrogate_set_layer(hyb_surrogate *m, int l, const float *w_host, const float *b_host) {
    if (!m || l < 0 || l >= SL || !w_host || !b_host) return set_error(HYB_EINVAL, "bad argument");
    const size_t nw = (size_t)CO[l] * CI[l] * 27;
    std::vector<float> b(COP[l], 0.0f);
    for (int c = 0; c < CO[l]; ++c) b[c] = b_host[c];
    HYB_CUDA_TRY(cudaMemcpyAsync(m->w[l], w_host, sizeof(float) * nw, cudaMemcpyHostToDevice, m->stream));
    HYB_CUDA_TRY(cudaMemcpyAsync(m->b[l], b.data(), sizeof(float) * COP[l], cudaMemcpyHostToDevice, m->stream));
    hyb_status s = repack(m);
    if (s != HYB_OK) return s;
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_surrogate_get_layer(hyb_surrogate *m, int l, float *w_host, float *b_host) {
    if (!m || l < 0 || l >= SL) return set_error(HYB_EINVAL, "bad argument");
    if (w_host)
        HYB_CUDA_TRY(cudaMemcpyAsync(w_host, m->w[l], sizeof(float) * CO[l] * CI[l] * 27, cudaMemcpyDeviceToHost,
                                     m->stream));
    if (b_host) HYB_CUDA_TRY(cudaMemcpyAsync(b_host, m->b[l], sizeof(float) * CO[l], cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_surrogate_forward(hyb_surrogate *m, const float *x, int B, int D, int H, int W, int pass, float *y) {
    if (!m || !x || !y) return set_error(HYB_EINVAL, "null argument");
    hyb_status s = check_shape(B, D, H, W);
    const long long V = (long long)D * H * W, cells = (long long)B * V;
    if (s == HYB_OK) s = reserve(m, cells);
    if (s != HYB_OK) return s;
    k_sur_prep<<<nbk(cells), RB, 0, m->stream>>>(x, B, V, m->mean, m->std_, m->a[0]);
    if ((s = forward(m, B, D, H, W, pass)) != HYB_OK) return s;
    k_sur_out<<<nbk(cells * NCH), RB, 0, m->stream>>>(m->y, x, B, V, m->dstd, y);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

hyb_status hyb_surrogate_mc(hyb_surrogate *m, const float *x, int B, int D, int H, int W, float *pm, float *ps) {
    if (!m || !x || !pm || !ps) return set_error(HYB_EINVAL, "null argument");
    hyb_status s = check_shape(B, D, H, W);
    const long long V = (long long)D * H * W, cells = (long long)B * V;
    if (s == HYB_OK) s = reserve(m, cells);
    if (s != HYB_OK) return s;
    k_sur_prep<<<nbk(cells), RB, 0, m->stream>>>(x, B, V, m->mean, m->std_, m->a[0]);
    const int K = m->d.mc_passes;
    for (int k = 1; k <= K; ++k) {
        if ((s = forward(m, B, D, H, W, k - 1)) != HYB_OK) return s;
        k_sur_mc<<<nbk(cells * NCH), RB, 0, m->stream>>>(m->y, x, B, V, m->dstd, k, pm, ps);
    }
    k_sur_mc_final<<<nbk(cells * NCH), RB, 0, m->stream>>>(cells * NCH, K, ps);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

hyb_status hyb_surrogate_train_step(hyb_surrogate *m, const float *x, const float *tg, int B, int D, int H, int W,
                                    hyb_surrogate_stats *out) {
    if (!m || !x || !tg || !out) return set_error(HYB_EINVAL, "null argument");
    hyb_status s = check_shape(B, D, H, W);
    const long long V = (long long)D * H * W, cells = (long long)B * V;
    if (s == HYB_OK) s = reserve(m, cells);
    if (s != HYB_OK) return s;
    if (B > m->ecap) {
        s_free(m, m->epart);
        s_free(m, m->esum);
        m->epart = m->esum = nullptr;
        m->ecap = 0;
        if (s_alloc(m, (void **)&m->epart, sizeof(double) * 2 * m->eblocks * B) ||
            s_alloc(m, (void **)&m->esum, sizeof(double) * 2 * B))
            return set_error(HYB_ENOMEM, "surrogate loss buffers");
        m->ecap = B;
    }
    cudaStream_t st = m->stream;
    const int pass = (int)(m->adam_t & 0x7fffffff);
    k_sur_prep<<<nbk(cells), RB, 0, st>>>(x, B, V, m->mean, m->std_, m->a[0]);
    if ((s = forward(m, B, D, H, W, pass)) != HYB_OK) return s;
    // loss: per-sample energies, then the gradient dL/dy (G[SL] and dz)
    k_sur_energy<<<dim3(m->eblocks, B), RB, 0, st>>>(m->y, tg, x, V, m->dstd, m->epart);
    k_sur_esum<<<nbk(B), RB, 0, st>>>(m->epart, B, m->eblocks, m->esum);
    k_sur_loss<<<m->lblocks, RB, 0, st>>>(m->y, tg, x, B, V, m->dstd, (float)m->d.huber_delta,
                                          (float)m->d.energy_weight, m->esum, m->G[SL], m->dz, m->lpart);
    // backward, last layer first
    for (int l = SL - 1; l >= 0; --l) {
        if (l < SL - 1)
            k_act_dz<<<nbk(cells * (COP[l] / 8)), RB, 0, st>>>(m->G[l + 1], m->s[l], m->b[l], COP[l], RELU[l],
                                                              drop_of(m, l, pass), B, V, m->dz);
        if ((s = layer_wgrad(m, l, B, D, H, W)) != HYB_OK) return s;
        if (l > 0) {
            cudaMemsetAsync(m->G[l], 0, sizeof(float) * CIP[l] * cells, st);
            if ((s = conv_chunks(m, m->dz, COP[l], m->pkT[l], CIP[l], m->G[l], B, D, H, W)) != HYB_OK) return s;
            if (RES[l]) k_sur_addres<<<nbk(cells * CIP[l]), RB, 0, st>>>(m->G[l], m->G[l + 1], CIP[l], COP[l], cells);
        }
    }
    // Adam on the FP32 masters, then the BF16 packs
    m->adam_t += 1;
    const float b1 = (float)m->d.beta1, b2 = (float)m->d.beta2;
    const float c1 = (float)(1.0 - std::pow(m->d.beta1, (double)m->adam_t));
    const float c2 = (float)(1.0 - std::pow(m->d.beta2, (double)m->adam_t));
    for (int l = 0; l < SL; ++l) {
        const int nw = CO[l] * CI[l] * 27;
        k_adam<<<nbk(nw), RB, 0, st>>>(m->w[l], m->gw[l], m->mw[l], m->vw[l], nw, (float)m->d.lr, b1, b2,
                                       (float)m->d.eps, c1, c2);
        k_adam<<<nbk(CO[l]), RB, 0, st>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], CO[l], (float)m->d.lr, b1, b2,
                                          (float)m->d.eps, c1, c2);
    }
    if ((s = repack(m)) != HYB_OK) return s;
    std::vector<double> hp((size_t)m->lblocks), es((size_t)2 * B);
    HYB_CUDA_TRY(cudaMemcpyAsync(hp.data(), m->lpart, sizeof(double) * m->lblocks, cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaMemcpyAsync(es.data(), m->esum, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, st));
    if ((s = read_status(m)) != HYB_OK) return s;
    double hub = 0.0, ev = 0.0, wp = 0.0, wt = 0.0;
    for (int k = 0; k < m->lblocks; ++k) hub += hp[k];
    hub /= (double)cells * NCH;
    for (int b = 0; b < B; ++b) {
        wp += es[2 * b];
        wt += es[2 * b + 1];
    }
    if (wt > 0.0) ev = ((wp - wt) / wt) * ((wp - wt) / wt);
    out->huber = hub;
    out->energy = ev;
    out->loss = hub + m->d.energy_weight * ev;
    out->step = m->adam_t;
    return HYB_OK;
}

hyb_status hyb_surrogate_get_grad(hyb_surrogate *m, int l, float *gw, float *gb) {
    if (!m || l < 0 || l >= SL || m->adam_t == 0) return set_error(HYB_EINVAL, "no gradients (no training step yet)");
    if (gw) HYB_CUDA_TRY(cudaMemcpyAsync(gw, m->gw[l], sizeof(float) * CO[l] * CI[l] * 27, cudaMemcpyDeviceToHost, m->stream));
    if (gb) HYB_CUDA_TRY(cudaMemcpyAsync(gb, m->gb[l], sizeof(float) * CO[l], cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

}  // extern "C"
