// The regime classifier around the tensor-core convolution (arXiv 2510.11174,
// Methodology and Results: convolutional network on per-channel normalised
// fields; Monte Carlo dropout for the uncertainty of the switch).
//
// Network: conv3(6->32) ReLU drop, conv3(32->32) ReLU drop, conv3(32->16) ReLU
// drop, conv3(16->1), sigmoid.  Layers 0-2 run on the tensor cores
// (k_conv3_tc, BF16 operands, FP32 accumulation, BF16 channels-last
// activations); the 16->1 layer is a 432-MAC dot product per cell on the CUDA
// cores with BF16-rounded weights.  Classification runs mc_passes passes with
// independent dropout masks and keeps the running mean and variance of the
// sigmoid per node (Welford).
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"
#include "philox.cuh"


static constexpr int NL = 4;
static constexpr int CIN[NL] = {6, 32, 32, 16}, COUT[NL] = {32, 32, 16, 1};
static constexpr int CINP[NL] = {16, 32, 32, 16};  // input channels padded for the tensor-core layout
static constexpr int MC_GROUP = 4;                  // MC passes whose layer-1 inputs one dropout launch writes

struct hyb_model {
    hyb_model_desc d;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *w[NL] = {}, *b[NL] = {};      // FP32 master weights [co][ci][27], biases
    float *mw[NL] = {}, *vw[NL] = {}, *mb[NL] = {}, *vb[NL] = {};  // Adam moments
    __nv_bfloat16 *wt[3] = {};           // packed forward weights, layers 0..2
    __nv_bfloat16 *wtT[3] = {};          // packed transposed + flipped (data gradient)
    float *w4r = nullptr;                // layer 3 weights rounded to BF16 (as FP32), [16][27]
    uint32_t w4pk[256] = {};             // w4r as BF16 B operand [ci / 8][tap (32)][ci % 8] (kernel parameter)
    float b4h = 0.0f;
    float *mean = nullptr, *std_ = nullptr;
    int xr_lo = 0, xr_hi = 0;            // a classification's x-range of final outputs (xr_hi <= xr_lo: all)
    // activation buffers (capacity in cells)
    long long cap = 0;
    __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;
    __nv_bfloat16 *h0s = nullptr;        // layer-0 output scaled by 1 / (1 - p), shared by the MC passes
    float *logit = nullptr, *pm = nullptr, *ps = nullptr;
    int *status = nullptr;
    long long adam_t = 0;
    void *train = nullptr;  // training buffers (allocated by the first training step)
    std::vector<void *> owned;
};

namespace hyb {

static cudaError_t m_alloc(hyb_model *m, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 256);
    if (e == cudaSuccess) m->owned.push_back(*p);
    return e;
}

// forward pack: wt[(dz, dy)][kc][dx n + o][8] = W[o][kc*8+j][tap (dz, dy, dx)]
// (zero for padded channels); transposed: the data gradient is the
// convolution of dY with W^T flipped, wtT[...][dx ci + i][8] = W[kc*8+j][i][26 - tap]
__global__ void k_pack(const float *__restrict__ W, int cin, int cinp, int cout, int transpose,
                       __nv_bfloat16 *__restrict__ out) {
    const int ci_n = transpose ? cout : cinp;  // input channels of the packed conv
    const int n_n = transpose ? cin : cout;    // output channels of the packed conv
    const int KC = ci_n / 8;
    const int total = 27 * KC * n_n * 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    // layout [9 (dz, dy)][KC][3 (dx) x n_n][8]: the three x-taps side by side in N
    const int j = t % 8, nn = (t / 8) % (3 * n_n), kc = (t / (8 * 3 * n_n)) % KC, tap9 = t / (8 * 3 * n_n * KC);
    const int dx = nn / n_n, n = nn % n_n, tap = tap9 * 3 + dx;
    const int c = kc * 8 + j;
    float v = 0.0f;
    if (!transpose) {
        if (c < cin) v = W[((long long)n * cin + c) * 27 + tap];
    } else {
        if (c < cout && n < cin) v = W[((long long)c * cin + n) * 27 + (26 - tap)];
    }
    out[t] = __float2bfloat16_rn(v);
}

__global__ void k_round_bf16(const float *__restrict__ in, float *__restrict__ out, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = __bfloat162float(__float2bfloat16_rn(in[t]));
}

// patches [B][6][D][H][W] FP32 -> normalised BF16 channels-last [B][D][H][W][16]
__global__ void k_prep_patches_cl(const float *__restrict__ x, int B, long long V, const float *__restrict__ mean,
                                  const float *__restrict__ sd, __nv_bfloat16 *__restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V) return;
    const long long b = t / V, v = t % V;
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        float s = 0.0f;
        if (c < 6) s = (x[(b * 6 + c) * V + v] - mean[c]) / sd[c];
        o[c] = __float2bfloat16_rn(s);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(out + t * 16);
    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// context fields at the nodes (E averaged from the Yee edges, B from the four
// faces around the node) -> normalised BF16 channels-last [D=nz][H=ny][W=nx][16]
__global__ void k_prep_fields(GridDev g, const float *__restrict__ E, const float *__restrict__ Bf,
                              const float *__restrict__ mean, const float *__restrict__ sd,
                              __nv_bfloat16 *__restrict__ out) {
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long c = ((long long)k * ny + j) * nx + i;
    auto fv = [&](const float *F, int a, int bb, int cc) -> float {
        int idx[3] = {a, bb, cc};
        for (int ax = 0; ax < 3; ++ax) {
            if (g.bc[ax] == 0) idx[ax] = idx[ax] < 0 ? idx[ax] + g.n[ax] : (idx[ax] >= g.n[ax] ? idx[ax] - g.n[ax] : idx[ax]);
            else if (idx[ax] < 0 || idx[ax] > g.n[ax] - 1) return 0.0f;
        }
        return F[cidx(g, idx[0], idx[1], idx[2])];
    };
    const long long N = g.N;
    float f[6];
    f[0] = 0.5f * (fv(E, i - 1, j, k) + fv(E, i, j, k));
    f[1] = 0.5f * (fv(E + N, i, j - 1, k) + fv(E + N, i, j, k));
    f[2] = 0.5f * (fv(E + 2 * N, i, j, k - 1) + fv(E + 2 * N, i, j, k));
    f[3] = 0.25f * (fv(Bf, i, j - 1, k - 1) + fv(Bf, i, j, k - 1) + fv(Bf, i, j - 1, k) + fv(Bf, i, j, k));
    f[4] = 0.25f * (fv(Bf + N, i - 1, j, k - 1) + fv(Bf + N, i, j, k - 1) + fv(Bf + N, i - 1, j, k) +
                    fv(Bf + N, i, j, k));
    f[5] = 0.25f * (fv(Bf + 2 * N, i - 1, j - 1, k) + fv(Bf + 2 * N, i, j - 1, k) + fv(Bf + 2 * N, i - 1, j, k) +
                    fv(Bf + 2 * N, i, j, k));
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q] = __float2bfloat16_rn(q < 6 ? (f[q] - mean[q]) / sd[q] : 0.0f);
    uint4 *dst = reinterpret_cast<uint4 *>(out + c * 16);
    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// the same node fields in FP32, not normalised, channel-first [6][nz][ny][nx]
// (training patches cut from a run)
// (with J: channels 6..8 hold J averaged over the two Yee edges at the node)
__global__ void k_node_fields_f32(GridDev g, const float *__restrict__ E, const float *__restrict__ Bf,
                                  const float *__restrict__ J, float *__restrict__ out) {
    const int nx = g.n[0], ny = g.n[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long c = ((long long)k * ny + j) * nx + i;
    auto fv = [&](const float *F, int a, int bb, int cc) -> float {
        int idx[3] = {a, bb, cc};
        for (int ax = 0; ax < 3; ++ax) {
            if (g.bc[ax] == 0) idx[ax] = idx[ax] < 0 ? idx[ax] + g.n[ax] : (idx[ax] >= g.n[ax] ? idx[ax] - g.n[ax] : idx[ax]);
            else if (idx[ax] < 0 || idx[ax] > g.n[ax] - 1) return 0.0f;
        }
        return F[cidx(g, idx[0], idx[1], idx[2])];
    };
    const long long N = g.N;
    out[c] = 0.5f * (fv(E, i - 1, j, k) + fv(E, i, j, k));
    out[N + c] = 0.5f * (fv(E + N, i, j - 1, k) + fv(E + N, i, j, k));
    out[2 * N + c] = 0.5f * (fv(E + 2 * N, i, j, k - 1) + fv(E + 2 * N, i, j, k));
    out[3 * N + c] = 0.25f * (fv(Bf, i, j - 1, k - 1) + fv(Bf, i, j, k - 1) + fv(Bf, i, j - 1, k) + fv(Bf, i, j, k));
    out[4 * N + c] = 0.25f * (fv(Bf + N, i - 1, j, k - 1) + fv(Bf + N, i, j, k - 1) + fv(Bf + N, i - 1, j, k) +
                              fv(Bf + N, i, j, k));
    out[5 * N + c] = 0.25f * (fv(Bf + 2 * N, i - 1, j - 1, k) + fv(Bf + 2 * N, i, j - 1, k) +
                              fv(Bf + 2 * N, i - 1, j, k) + fv(Bf + 2 * N, i, j, k));
    if (J) {
        out[6 * N + c] = 0.5f * (fv(J, i - 1, j, k) + fv(J, i, j, k));
        out[7 * N + c] = 0.5f * (fv(J + N, i, j - 1, k) + fv(J + N, i, j, k));
        out[8 * N + c] = 0.5f * (fv(J + 2 * N, i, j, k - 1) + fv(J + 2 * N, i, j, k));
    }
}

// layer-1 inputs of the passes pass0 .. pass0 + G - 1: a1[g] = h0s where the
// layer-0 dropout mask of pass pass0 + g keeps the channel, else 0 (h0s holds
// bf16(relu(layer 0) / (1 - p)), the kept value of every pass).  The 16-bit
// Philox field of channel j is the low (even j) or high (odd j) half of word
// j / 2, the same half that holds channel j in a word of two BF16 values, so
// one SIMD compare per word gives the mask.
__global__ void k_dropout_select(const __nv_bfloat16 *__restrict__ h0s, long long cells, long long V, uint32_t seed,
                                 uint32_t pass0, int G, uint32_t thr, __nv_bfloat16 *__restrict__ a1,
                                 long long pitch, int W, int x_lo, int x_hi) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cells) return;
    const uint32_t b = (uint32_t)(t / V), lin = (uint32_t)(t % V);
    if (x_hi > x_lo) {
        const int x = (int)(lin % (uint32_t)W);
        if (x < x_lo || x >= x_hi) return;  // outside the classified x-range
    }
    const uint4 *src = reinterpret_cast<const uint4 *>(h0s + t * 32);
    uint4 h[4];
#pragma unroll
    for (int g8 = 0; g8 < 4; ++g8) h[g8] = src[g8];
    const uint32_t thr2 = thr | (thr << 16);
    for (int g = 0; g < G; ++g) {
        uint4 *dst = reinterpret_cast<uint4 *>(a1 + g * pitch + t * 32);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
            const u32x4 r = philox4x32_10(lin, b, (0u << 16) | (uint32_t)g8, pass0 + (uint32_t)g, seed, 0xD0u);
            uint4 o;
            o.x = h[g8].x & __vcmpgeu2(r.v[0], thr2);
            o.y = h[g8].y & __vcmpgeu2(r.v[1], thr2);
            o.z = h[g8].z & __vcmpgeu2(r.v[2], thr2);
            o.w = h[g8].w & __vcmpgeu2(r.v[3], thr2);
            dst[g8] = o;
        }
    }
}
__global__ void k_mc_final(long long n, int k, const float *m2, float *ps) {  // may run in place
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) ps[t] = sqrtf(fmaxf(m2[t], 0.0f) / (float)k);  // population standard deviation over the passes
}

static inline unsigned nb(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

hyb_status model_repack(hyb_model *m) {
    for (int l = 0; l < 3; ++l) {
        const int tot = 27 * (CINP[l] / 8) * COUT[l] * 8;
        k_pack<<<nb(tot), 256, 0, m->stream>>>(m->w[l], CIN[l], CINP[l], COUT[l], 0, m->wt[l]);
        const int totT = 27 * (COUT[l] / 8) * CIN[l] * 8;
        if (l > 0) k_pack<<<nb(totT), 256, 0, m->stream>>>(m->w[l], CIN[l], CINP[l], COUT[l], 1, m->wtT[l]);
    }
    k_round_bf16<<<nb(16 * 27), 256, 0, m->stream>>>(m->w[3], m->w4r, 16 * 27);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("weight packing: ") + cudaGetErrorString(e));
    // the last layer takes its weights as a kernel parameter: keep a host copy
    float w4[16 * 27];
    e = cudaMemcpyAsync(w4, m->w4r, sizeof(w4), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m->b4h, m->b[3], sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("weight copy: ") + cudaGetErrorString(e));
    // the values are BF16-rounded already: their BF16 code is the upper half
    uint16_t pk[512];
    for (int e = 0; e < 512; ++e) {
        const int j = e % 8, tap = (e / 8) % 32, kc = e / 256, ci = kc * 8 + j;
        uint32_t bits = 0;
        if (tap < 27) memcpy(&bits, &w4[ci * 27 + tap], 4);
        pk[e] = (uint16_t)(bits >> 16);
    }
    for (int i = 0; i < 256; ++i) m->w4pk[i] = (uint32_t)pk[2 * i] | ((uint32_t)pk[2 * i + 1] << 16);
    return HYB_OK;
}

static hyb_status model_reserve(hyb_model *m, long long cells) {
    if (cells <= m->cap) return HYB_OK;
    // buffers are replaced only between stream-ordered uses
    cudaStreamSynchronize(m->stream);
    void *bufs[8] = {m->x0, m->a1, m->a2, m->a3, m->logit, m->pm, m->ps, m->h0s};
    for (void *p : bufs) {
        if (!p) continue;
        for (auto it = m->owned.begin(); it != m->owned.end(); ++it)
            if (*it == p) {
                m->owned.erase(it);
                break;
            }
        cudaFree(p);
    }
    if (m_alloc(m, (void **)&m->x0, sizeof(__nv_bfloat16) * 16 * cells) ||
        m_alloc(m, (void **)&m->a1, sizeof(__nv_bfloat16) * 32 * cells * MC_GROUP) ||
        m_alloc(m, (void **)&m->a2, sizeof(__nv_bfloat16) * 32 * cells) ||
        m_alloc(m, (void **)&m->a3, sizeof(__nv_bfloat16) * 16 * cells) ||
        m_alloc(m, (void **)&m->h0s, sizeof(__nv_bfloat16) * 32 * cells) ||
        m_alloc(m, (void **)&m->logit, sizeof(float) * cells) || m_alloc(m, (void **)&m->pm, sizeof(float) * cells) ||
        m_alloc(m, (void **)&m->ps, sizeof(float) * cells))
        return set_error(HYB_ENOMEM, "classifier activation buffers");
    // defined contents: a classification restricted to an x-range reads, but does
    // not use, activations just outside it
    cudaMemsetAsync(m->x0, 0, sizeof(__nv_bfloat16) * 16 * cells, m->stream);
    cudaMemsetAsync(m->a1, 0, sizeof(__nv_bfloat16) * 32 * cells * MC_GROUP, m->stream);
    cudaMemsetAsync(m->a2, 0, sizeof(__nv_bfloat16) * 32 * cells, m->stream);
    cudaMemsetAsync(m->a3, 0, sizeof(__nv_bfloat16) * 16 * cells, m->stream);
    cudaMemsetAsync(m->h0s, 0, sizeof(__nv_bfloat16) * 32 * cells, m->stream);
    const cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("activation buffers: ") + cudaGetErrorString(e));
    m->cap = cells;
    return HYB_OK;
}


// layers 0..3 on the prepared input m->x0 (B x D x H x W cells) -> m->logit
static ConvArgs conv_args(hyb_model *m, int l, int B, int D, int H, int W, int pass) {
    const uint32_t thr = pass >= 0 ? dropout_threshold(m->d.dropout) : 0u;
    __nv_bfloat16 *ins[3] = {m->x0, m->a1, m->a2}, *outs[3] = {m->a1, m->a2, m->a3};
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.x = ins[l];
    a.wt = m->wt[l];
    a.bias = m->b[l];
    a.y = outs[l];
    a.B = B;
    a.D = D;
    a.H = H;
    a.W = W;
    a.cin = CINP[l];
    a.N = COUT[l];
    a.relu = 1;
    a.drop_thr = thr;
    a.drop_scale = dropout_scale(thr);
    a.scale_out = thr != 0;
    a.seed = m->d.seed;
    a.pass = (uint32_t)(pass >= 0 ? pass : 0);
    a.layer = (uint32_t)l;
    a.status = m->status;
    if (m->xr_hi > m->xr_lo) {
        // layer l feeds 3 - l more 3x3x3 layers: its outputs are needed that far beyond the range
        a.x_lo = std::max(0, m->xr_lo - (3 - l));
        a.x_hi = std::min(W, m->xr_hi + (3 - l));
    }
    return a;
}

static hyb_status launch_last(hyb_model *m, int B, int D, int H, int W, int mc_k, cudaStream_t st) {
    LastArgs a;
    memset(&a, 0, sizeof(a));
    a.x = m->a3;
    memcpy(a.w, m->w4pk, sizeof(a.w));
    a.bias = m->b4h;
    a.B = B;
    a.D = D;
    a.H = H;
    a.W = W;
    a.logit = m->logit;
    a.mc_k = mc_k;
    a.pm = m->pm;
    a.m2 = m->ps;
    a.status = m->status;
    a.x_lo = m->xr_lo;
    a.x_hi = m->xr_hi;
    return launch_conv_last_tc(a, st);
}

// layers first_layer..3 on m->x0 (or on m->a1 when first_layer = 1) for
// B x D x H x W cells; mc_k = 0 writes m->logit, mc_k >= 1 folds the pass
// into the MC statistics (see k_conv_last_tc)
static hyb_status model_run(hyb_model *m, int B, int D, int H, int W, int pass, int mc_k = 0, int first_layer = 0) {
    for (int l = first_layer; l < 3; ++l) {
        hyb_status s = launch_conv3_tc(conv_args(m, l, B, D, H, W, pass), m->stream);
        if (s != HYB_OK) return s;
    }
    hyb_status s = launch_last(m, B, D, H, W, mc_k, m->stream);
    if (s != HYB_OK) return s;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("classifier: ") + cudaGetErrorString(e));
    return HYB_OK;
}

// Classification of the context's fields: K = mc_passes MC-dropout passes.
// Layer 0 is the same in every pass up to its dropout, so it runs once (FP32
// output before dropout) and each pass applies its own layer-0 mask before
// layers 1..3; the last layer folds each pass into the running mean and M2.
hyb_status classifier_forward(hyb_ctx *c, const hyb_model *mc, float *p_mean_dev, float *p_std_dev) {
    hyb_model *m = const_cast<hyb_model *>(mc);
    const GridDev &g = c->g;
    const int D = g.n[2], H = g.n[1], W = g.n[0];
    if (W % 8 != 0 || H % 16 != 0) return set_error(HYB_EINVAL, "classifier needs nx % 8 == 0 and ny % 16 == 0");
    hyb_status s = model_reserve(m, g.N);
    if (s != HYB_OK) return s;
    // the model runs on the context's stream for the classification
    // with a reach, only the x-range within reach + dilate nodes of matter is
    // classified; p_mean = p_std = 0 elsewhere (see hyb_regime_desc.reach)
    m->xr_lo = m->xr_hi = 0;
    if (c->regime.reach > 0) {
        int xa = 0, xb = 0;
        s = matter_x_range(c, c->regime.reach + c->regime.dilate, &xa, &xb);
        if (s != HYB_OK) return s;
        HYB_CUDA_TRY(cudaMemsetAsync(m->pm, 0, sizeof(float) * g.N, c->stream));
        HYB_CUDA_TRY(cudaMemsetAsync(m->ps, 0, sizeof(float) * g.N, c->stream));
        if (xb <= xa) {
            // no matter anywhere: nothing to classify
            c->classified_cells = 0;
            if (p_mean_dev) HYB_CUDA_TRY(cudaMemcpyAsync(p_mean_dev, m->pm, sizeof(float) * g.N, cudaMemcpyDeviceToDevice, c->stream));
            if (p_std_dev) HYB_CUDA_TRY(cudaMemcpyAsync(p_std_dev, m->ps, sizeof(float) * g.N, cudaMemcpyDeviceToDevice, c->stream));
            return HYB_OK;
        }
        if (xa > 0 || xb < W) {
            m->xr_lo = xa;
            m->xr_hi = xb;
        }
    }
    c->classified_cells = m->xr_hi > m->xr_lo ? (long long)(m->xr_hi - m->xr_lo) * H * D : g.N;
    cudaStream_t saved = m->stream;
    m->stream = c->stream;
    k_prep_fields<<<node_grid(g), node_block(g), 0, c->stream>>>(g, c->E, c->B, m->mean, m->std_, m->x0);
    const int K = m->d.mc_passes > 0 ? m->d.mc_passes : 1;
    const uint32_t thr = dropout_threshold(m->d.dropout);
    long long launches = 1;
    if (K > 1 && thr > 0) {
        // layer 0 once, its outputs scaled as kept values: bf16(relu(.) / (1 - p))
        ConvArgs a0 = conv_args(m, 0, 1, D, H, W, -1);
        a0.y = m->h0s;
        a0.drop_scale = dropout_scale(thr);
        a0.scale_out = 1;
        s = launch_conv3_tc(a0, c->stream);
        ++launches;
        // profiling: events around the layer-1 and layer-2 convolutions of every pass
        const bool prof = c->profiling;
        if (prof) {
            const size_t need = (size_t)2 * K * 2;
            while (c->conv_ev.size() < need) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) {
                    m->stream = saved;
                    m->xr_lo = m->xr_hi = 0;
                    return set_error(HYB_ECUDA, "profiling event creation");
                }
                c->conv_ev.push_back(e);
            }
            c->conv_ev_passes = K;
            c->phase_ran[HYB_PH_CONV1] = c->phase_ran[HYB_PH_CONV2] = true;
        }
        for (int k = 1; k <= K && s == HYB_OK; ++k) {
            const int slot = (k - 1) % MC_GROUP;
            if (slot == 0) {
                // the layer-0 dropout of the next MC_GROUP passes, one read of h0s
                const int G = std::min(MC_GROUP, K - (k - 1));
                const int dlo = m->xr_hi > m->xr_lo ? std::max(0, m->xr_lo - 3) : 0;
                const int dhi = m->xr_hi > m->xr_lo ? std::min(W, m->xr_hi + 3) : 0;
                k_dropout_select<<<nb(g.N), 256, 0, c->stream>>>(m->h0s, g.N, g.N, m->d.seed, (uint32_t)(k - 1), G,
                                                                 thr, m->a1, g.N * 32, W, dlo, dhi);
                ++launches;
            }
            for (int l = 1; l < 3 && s == HYB_OK; ++l) {
                ConvArgs a = conv_args(m, l, 1, D, H, W, k - 1);
                if (l == 1) a.x = m->a1 + (size_t)slot * g.N * 32;
                if (prof) cudaEventRecord(c->conv_ev[((l - 1) * K + (k - 1)) * 2], c->stream);
                s = launch_conv3_tc(a, c->stream);
                if (prof) cudaEventRecord(c->conv_ev[((l - 1) * K + (k - 1)) * 2 + 1], c->stream);
            }
            if (s == HYB_OK) s = launch_last(m, 1, D, H, W, k, c->stream);
            launches += 3;
        }
    } else {
        for (int k = 1; k <= K && s == HYB_OK; ++k) {
            s = model_run(m, 1, D, H, W, K > 1 ? k - 1 : -1, k, 0);
            launches += 4;
        }
    }
    if (s == HYB_OK) {
        // ps held M2; turn it into the standard deviation in place
        k_mc_final<<<nb(g.N), 256, 0, c->stream>>>(g.N, K, m->ps, m->ps);
        c->launches_classify += launches + 1;
        if (p_mean_dev) cudaMemcpyAsync(p_mean_dev, m->pm, sizeof(float) * g.N, cudaMemcpyDeviceToDevice, c->stream);
        if (p_std_dev) cudaMemcpyAsync(p_std_dev, m->ps, sizeof(float) * g.N, cudaMemcpyDeviceToDevice, c->stream);
    }
    m->stream = saved;
    m->xr_lo = m->xr_hi = 0;
    return s;
}

const float *model_p_mean(const hyb_model *m) { return m->pm; }
const float *model_p_std(const hyb_model *m) { return m->ps; }

}  // namespace hyb

namespace hyb {
void train_free(hyb_model *m);
}

using namespace hyb;

extern "C" {

hyb_status hyb_model_create(const hyb_model_desc *d, hyb_model **out) {
    if (!d || !out) return set_error(HYB_EINVAL, "null argument");
    *out = nullptr;
    if (!(d->dropout >= 0.0 && d->dropout < 1.0)) return set_error(HYB_EINVAL, "dropout must be in [0, 1)");
    for (int c = 0; c < 6; ++c)
        if (!(d->std[c] > 0.0f)) return set_error(HYB_EINVAL, "normalisation std must be > 0");
    hyb_model *m = new hyb_model();
    m->d = *d;
    m->d.dropout = dropout_threshold(d->dropout) / 65536.0;
    if (!(m->d.lr > 0)) m->d.lr = 1e-3;
    if (!(m->d.beta1 > 0)) m->d.beta1 = 0.9;
    if (!(m->d.beta2 > 0)) m->d.beta2 = 0.999;
    if (!(m->d.eps > 0)) m->d.eps = 1e-8;
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
        hyb_model_destroy(m);
        return set_error(HYB_ENOMEM, msg);
    };
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)COUT[l] * CIN[l] * 27;
        if (m_alloc(m, (void **)&m->w[l], sizeof(float) * nw) || m_alloc(m, (void **)&m->b[l], sizeof(float) * COUT[l]) ||
            m_alloc(m, (void **)&m->mw[l], sizeof(float) * nw) || m_alloc(m, (void **)&m->vw[l], sizeof(float) * nw) ||
            m_alloc(m, (void **)&m->mb[l], sizeof(float) * COUT[l]) ||
            m_alloc(m, (void **)&m->vb[l], sizeof(float) * COUT[l]))
            return fail("model allocation");
        cudaMemsetAsync(m->mw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->vw[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->mb[l], 0, sizeof(float) * COUT[l], m->stream);
        cudaMemsetAsync(m->vb[l], 0, sizeof(float) * COUT[l], m->stream);
    }
    for (int l = 0; l < 3; ++l) {
        if (m_alloc(m, (void **)&m->wt[l], sizeof(__nv_bfloat16) * 27 * CINP[l] * COUT[l]) ||
            m_alloc(m, (void **)&m->wtT[l], sizeof(__nv_bfloat16) * 27 * COUT[l] * CIN[l] + 256))
            return fail("model allocation");
    }
    if (m_alloc(m, (void **)&m->w4r, sizeof(float) * 16 * 27) || m_alloc(m, (void **)&m->mean, sizeof(float) * 6) ||
        m_alloc(m, (void **)&m->std_, sizeof(float) * 6) || m_alloc(m, (void **)&m->status, sizeof(int)))
        return fail("model allocation");
    cudaMemcpyAsync(m->mean, d->mean, sizeof(float) * 6, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->std_, d->std, sizeof(float) * 6, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->status, 0, sizeof(int), m->stream);
    // He-uniform initialisation from the seed (Philox on the host):
    // w ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)), b = 0
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)COUT[l] * CIN[l] * 27;
        std::vector<float> w(nw), b(COUT[l], 0.0f);
        const float lim = std::sqrt(6.0f / (float)(CIN[l] * 27));
        for (size_t i = 0; i < nw; ++i) {
            const u32x4 r = philox4x32_10((uint32_t)i, (uint32_t)l, 0x1417u, 0u, d->seed, 0xA1u);
            w[i] = (2.0f * u01f(r.v[0]) - 1.0f) * lim;
        }
        cudaMemcpy(m->w[l], w.data(), sizeof(float) * nw, cudaMemcpyHostToDevice);
        cudaMemcpy(m->b[l], b.data(), sizeof(float) * COUT[l], cudaMemcpyHostToDevice);
    }
    hyb_status s = model_repack(m);
    if (s == HYB_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) s = set_error(HYB_ECUDA, "model init");
    if (s != HYB_OK) {
        hyb_model_destroy(m);
        return s;
    }
    *out = m;
    return HYB_OK;
}

void hyb_model_destroy(hyb_model *m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void *p : m->owned) cudaFree(p);
    train_free(m);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

hyb_status hyb_model_set_layer(hyb_model *m, int l, const float *w, const float *b) {
    if (!m || l < 0 || l >= NL || !w || !b) return set_error(HYB_EINVAL, "bad argument");
    HYB_CUDA_TRY(cudaMemcpyAsync(m->w[l], w, sizeof(float) * COUT[l] * CIN[l] * 27, cudaMemcpyHostToDevice, m->stream));
    HYB_CUDA_TRY(cudaMemcpyAsync(m->b[l], b, sizeof(float) * COUT[l], cudaMemcpyHostToDevice, m->stream));
    hyb_status s = model_repack(m);
    if (s != HYB_OK) return s;
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_model_get_layer(hyb_model *m, int l, float *w, float *b) {
    if (!m || l < 0 || l >= NL) return set_error(HYB_EINVAL, "bad argument");
    if (w) HYB_CUDA_TRY(cudaMemcpyAsync(w, m->w[l], sizeof(float) * COUT[l] * CIN[l] * 27, cudaMemcpyDeviceToHost, m->stream));
    if (b) HYB_CUDA_TRY(cudaMemcpyAsync(b, m->b[l], sizeof(float) * COUT[l], cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

hyb_status hyb_model_forward(hyb_model *m, const float *x, int B, int D, int H, int W, int pass, float *logits) {
    if (!m || !x || !logits || B <= 0 || D <= 0 || H <= 0 || W <= 0) return set_error(HYB_EINVAL, "bad argument");
    if (W % 8 != 0 || H % 16 != 0) return set_error(HYB_EINVAL, "forward needs W % 8 == 0 and H % 16 == 0");
    const long long V = (long long)D * H * W, cells = (long long)B * V;
    hyb_status s = model_reserve(m, cells);
    if (s != HYB_OK) return s;
    k_prep_patches_cl<<<nb(cells), 256, 0, m->stream>>>(x, B, V, m->mean, m->std_, m->x0);
    s = model_run(m, B, D, H, W, pass);
    if (s != HYB_OK) return s;
    HYB_CUDA_TRY(cudaMemcpyAsync(logits, m->logit, sizeof(float) * cells, cudaMemcpyDeviceToDevice, m->stream));
    int st = 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (st) return set_error(HYB_ETIMEOUT, "a tensor-core wait gave up");
    return HYB_OK;
}

hyb_status hyb_node_fields(hyb_ctx *c, float *out_dev) {
    if (!c || !out_dev) return set_error(HYB_EINVAL, "null argument");
    k_node_fields_f32<<<node_grid(c->g), node_block(c->g), 0, c->stream>>>(c->g, c->E, c->B, nullptr, out_dev);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

hyb_status hyb_node_state(hyb_ctx *c, float *out_dev) {
    if (!c || !out_dev) return set_error(HYB_EINVAL, "null argument");
    k_node_fields_f32<<<node_grid(c->g), node_block(c->g), 0, c->stream>>>(c->g, c->E, c->B, c->J, out_dev);
    HYB_CUDA_TRY(cudaGetLastError());
    return charge_density(c, out_dev + 9 * c->g.N);
}

}  // extern "C"

// ============================================================================ training
// Loss, backward and Adam (see hyb_train_step in include/hyb.h).
namespace hyb {

static constexpr int RBT = 256;

struct TrainBufs {
    float *gw[NL] = {}, *gb[NL] = {};
    float *dlogit = nullptr, *edens = nullptr;
    __nv_bfloat16 *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;  // data gradients (BF16, channels-last)
    double *lpart = nullptr;  // loss partials
    long long cap = 0, wcap = 0;
    int lblocks = 0;
    WgradScratch wg;          // operands of the tensor-core weight gradients
};

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RBT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// field energy density per cell (|E|^2 + |B|^2)/2 of the raw patches; FP64 partial sums
__global__ void __launch_bounds__(RBT) k_energy_density(const float *__restrict__ x, int B, long long V,
                                                        float *__restrict__ e, double *__restrict__ part) {
    __shared__ double sh[RBT];
    double acc = 0.0;
    for (long long t = blockIdx.x * (long long)RBT + threadIdx.x; t < (long long)B * V; t += (long long)gridDim.x * RBT) {
        const long long b = t / V, v = t % V;
        float s = 0.0f;
        for (int c = 0; c < 6; ++c) {
            const float q = x[(b * 6 + c) * V + v];
            s += q * q;
        }
        e[t] = 0.5f * s;
        acc += 0.5 * (double)s;
    }
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// weighted BCE with logits, its gradient, and FP64 partial sums (loss, bce, correct)
__global__ void __launch_bounds__(RBT) k_loss(const float *__restrict__ logit, const float *__restrict__ y,
                                              const float *__restrict__ e, float inv_emean, float lam, long long n,
                                              float *__restrict__ dlogit, double *__restrict__ part) {
    __shared__ double sh[RBT];
    double al = 0.0, ab = 0.0, ac = 0.0;
    const float invn = 1.0f / (float)n;
    for (long long t = blockIdx.x * (long long)RBT + threadIdx.x; t < n; t += (long long)gridDim.x * RBT) {
        const float l = logit[t], yy = y[t];
        const float w = 1.0f + lam * e[t] * inv_emean;
        // BCE(sigmoid(l), y) = max(l, 0) - l y + log(1 + exp(-|l|))
        const float bce = fmaxf(l, 0.0f) - l * yy + log1pf(expf(-fabsf(l)));
        const float p = 1.0f / (1.0f + expf(-l));
        dlogit[t] = w * (p - yy) * invn;
        al += (double)w * bce;
        ab += bce;
        ac += ((p >= 0.5f) == (yy >= 0.5f)) ? 1.0 : 0.0;
    }
    al = block_sum_d(al, sh);
    ab = block_sum_d(ab, sh);
    ac = block_sum_d(ac, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = al;
        part[blockIdx.x * 3 + 1] = ab;
        part[blockIdx.x * 3 + 2] = ac;
    }
}

// layer 3 data gradient: dA3[c][ci] = sum_tap W[ci][tap] dlogit[c - s(tap)], then
// dz3 = bf16(dA3 [a3 > 0] / (1 - p)) (ReLU and dropout of layer 2's output)
__global__ void k_dgrad_last(const float *__restrict__ dlogit, const float *__restrict__ w4r,
                             const __nv_bfloat16 *__restrict__ a3, int B, int D, int H, int W, float inv_keep,
                             __nv_bfloat16 *__restrict__ dz3) {
    __shared__ float ws[16 * 27];
    for (int i = threadIdx.x; i < 16 * 27; i += blockDim.x) ws[i] = w4r[i];
    __syncthreads();
    const long long V = (long long)D * H * W;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)B * V) return;
    const long long b = t / V, v = t % V;
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((long long)W * H));
    float acc[16];
#pragma unroll
    for (int ci = 0; ci < 16; ++ci) acc[ci] = 0.0f;
    for (int tap = 0; tap < 27; ++tap) {
        const int zz = z - (tap / 9 - 1), yy = y - ((tap / 3) % 3 - 1), xx = x - (tap % 3 - 1);
        if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
        const float g = dlogit[b * V + ((long long)zz * H + yy) * W + xx];
#pragma unroll
        for (int ci = 0; ci < 16; ++ci) acc[ci] += ws[ci * 27 + tap] * g;
    }
    __align__(16) __nv_bfloat16 h[16], o[16];
    reinterpret_cast<uint4 *>(h)[0] = reinterpret_cast<const uint4 *>(a3 + t * 16)[0];
    reinterpret_cast<uint4 *>(h)[1] = reinterpret_cast<const uint4 *>(a3 + t * 16)[1];
#pragma unroll
    for (int ci = 0; ci < 16; ++ci)
        o[ci] = __float2bfloat16_rn(__bfloat162float(h[ci]) > 0.0f ? acc[ci] * inv_keep : 0.0f);
    reinterpret_cast<uint4 *>(dz3 + t * 16)[0] = reinterpret_cast<const uint4 *>(o)[0];
    reinterpret_cast<uint4 *>(dz3 + t * 16)[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// dz = bf16(dA [a > 0] / (1 - p)) in place (dA from the tensor-core data gradient)
// (n a multiple of 8: eight values per thread, 16-byte loads and stores)
__global__ void k_mask_grad(__nv_bfloat16 *__restrict__ d, const __nv_bfloat16 *__restrict__ a, long long n,
                            float inv_keep) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t * 8 >= n) return;
    uint4 dv = reinterpret_cast<const uint4 *>(d)[t], av = reinterpret_cast<const uint4 *>(a)[t];
    __nv_bfloat16 *dh = reinterpret_cast<__nv_bfloat16 *>(&dv);
    const __nv_bfloat16 *ah = reinterpret_cast<const __nv_bfloat16 *>(&av);
#pragma unroll
    for (int j = 0; j < 8; ++j)
        dh[j] = __float2bfloat16_rn(__bfloat162float(ah[j]) > 0.0f ? __bfloat162float(dh[j]) * inv_keep : 0.0f);
    reinterpret_cast<uint4 *>(d)[t] = dv;
}

// sum the chunk partials in chunk order: out[o] = sum_k part[k][o]
__global__ void k_sum_parts(const float *__restrict__ part, int nchunks, int nout, float *__restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    float s = 0.0f;
    for (int k = 0; k < nchunks; ++k) s += part[(long long)k * nout + o];
    out[o] = s;
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static inline unsigned nbl(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

// training buffers, allocated on the first step and grown with the batch
static hyb_status train_reserve(hyb_model *m, long long cells) {
    if (!m->train) m->train = new TrainBufs();
    TrainBufs &t = *static_cast<TrainBufs *>(m->train);
    if (!t.gw[0]) {
        for (int l = 0; l < NL; ++l)
            if (m_alloc(m, (void **)&t.gw[l], sizeof(float) * COUT[l] * CIN[l] * 27) ||
                m_alloc(m, (void **)&t.gb[l], sizeof(float) * COUT[l]))
                return set_error(HYB_ENOMEM, "gradient buffers");
        t.lblocks = 152 * 2;
        if (m_alloc(m, (void **)&t.lpart, sizeof(double) * 3 * t.lblocks))
            return set_error(HYB_ENOMEM, "loss partials");
    }
    if (cells > t.cap) {
        cudaStreamSynchronize(m->stream);
        // old buffers stay owned by the model until it is destroyed
        if (m_alloc(m, (void **)&t.dlogit, sizeof(float) * cells) || m_alloc(m, (void **)&t.edens, sizeof(float) * cells) ||
            m_alloc(m, (void **)&t.dz3, sizeof(__nv_bfloat16) * 16 * cells) ||
            m_alloc(m, (void **)&t.dz2, sizeof(__nv_bfloat16) * 32 * cells) ||
            m_alloc(m, (void **)&t.dz1, sizeof(__nv_bfloat16) * 32 * cells))
            return set_error(HYB_ENOMEM, "training buffers");
        t.cap = cells;
    }
    return HYB_OK;
}

// weight and bias gradient of layer l on the tensor cores from its input A
// (ca channels per cell, CIN[l] real) and dZ (COUT[l] channels), or, for the
// last layer, from the FP32 dlogit
static hyb_status layer_wgrad(hyb_model *m, TrainBufs &t, int l, const __nv_bfloat16 *A, int ca,
                              const __nv_bfloat16 *dZ, const float *dZf, int B, int D, int H, int W) {
    WgradJob j;
    memset(&j, 0, sizeof(j));
    j.x = A;
    j.x_pitch = ca;
    j.ci_n = CIN[l];
    j.ci_tot = CIN[l];
    j.dz = dZ;
    j.dz_f32 = dZf;
    j.dz_pitch = COUT[l];
    j.co_n = COUT[l];
    j.B = B;
    j.D = D;
    j.H = H;
    j.W = W;
    j.taps = 27;
    j.gw = t.gw[l];
    j.gb = t.gb[l];
    j.status = m->status;
    return wgrad_tc(j, t.wg, m->stream);
}

}  // namespace hyb

namespace hyb {
void train_free(hyb_model *m) {
    delete static_cast<TrainBufs *>(m->train);
    m->train = nullptr;
}
}  // namespace hyb

extern "C" {

hyb_status hyb_train_step(hyb_model *m, const float *x, const float *y, int B, int D, int H, int W,
                          hyb_train_stats *out) {
    if (!m || !x || !y || !out || B <= 0 || D <= 0 || H <= 0 || W <= 0) return set_error(HYB_EINVAL, "bad argument");
    if (W % 8 != 0 || H % 16 != 0) return set_error(HYB_EINVAL, "training needs W % 8 == 0 and H % 16 == 0");
    const long long V = (long long)D * H * W, cells = (long long)B * V;
    hyb_status s = model_reserve(m, cells);
    if (s == HYB_OK) s = train_reserve(m, cells);
    if (s != HYB_OK) return s;
    TrainBufs &t = *static_cast<TrainBufs *>(m->train);
    cudaStream_t st = m->stream;
    const float inv_keep = dropout_scale(dropout_threshold(m->d.dropout));
    // forward, dropout masks of pass = the step index
    k_prep_patches_cl<<<nbl(cells), 256, 0, st>>>(x, B, V, m->mean, m->std_, m->x0);
    s = model_run(m, B, D, H, W, (int)(m->adam_t & 0x7fffffff));
    if (s != HYB_OK) return s;
    // energy weights: mean field energy density of the batch
    k_energy_density<<<t.lblocks, RBT, 0, st>>>(x, B, V, t.edens, t.lpart);
    std::vector<double> hp((size_t)3 * t.lblocks);
    HYB_CUDA_TRY(cudaMemcpyAsync(hp.data(), t.lpart, sizeof(double) * t.lblocks, cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));
    double esum = 0.0;
    for (int k = 0; k < t.lblocks; ++k) esum += hp[k];
    const double emean = esum / (double)cells;
    const float inv_emean = emean > 0.0 ? (float)(1.0 / emean) : 0.0f;
    k_loss<<<t.lblocks, RBT, 0, st>>>(m->logit, y, t.edens, inv_emean, (float)m->d.energy_weight, cells, t.dlogit,
                                      t.lpart);
    // layer 3 (16 -> 1): weight gradient from bf16(dlogit), data gradient on the CUDA cores
    if ((s = layer_wgrad(m, t, 3, m->a3, 16, nullptr, t.dlogit, B, D, H, W)) != HYB_OK) return s;
    k_dgrad_last<<<nbl(cells), 256, 0, st>>>(t.dlogit, m->w4r, m->a3, B, D, H, W, inv_keep, t.dz3);
    // layer 2 (32 -> 16): weight gradient, then the data gradient on the tensor cores
    if ((s = layer_wgrad(m, t, 2, m->a2, 32, t.dz3, nullptr, B, D, H, W)) != HYB_OK) return s;
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.B = B; a.D = D; a.H = H; a.W = W;
    a.status = m->status;
    a.x = t.dz3; a.wt = m->wtT[2]; a.cin = 16; a.N = 32; a.y = t.dz2;
    if ((s = launch_conv3_tc(a, st)) != HYB_OK) return s;
    k_mask_grad<<<nbl(cells * 4), 256, 0, st>>>(t.dz2, m->a2, cells * 32, inv_keep);
    // layer 1 (32 -> 32)
    if ((s = layer_wgrad(m, t, 1, m->a1, 32, t.dz2, nullptr, B, D, H, W)) != HYB_OK) return s;
    a.x = t.dz2; a.wt = m->wtT[1]; a.cin = 32; a.N = 32; a.y = t.dz1;
    if ((s = launch_conv3_tc(a, st)) != HYB_OK) return s;
    k_mask_grad<<<nbl(cells * 4), 256, 0, st>>>(t.dz1, m->a1, cells * 32, inv_keep);
    // layer 0 (6 -> 32): weight gradient only
    if ((s = layer_wgrad(m, t, 0, m->x0, 16, t.dz1, nullptr, B, D, H, W)) != HYB_OK) return s;
    // Adam on the FP32 master weights, then the BF16 copies
    m->adam_t += 1;
    const float b1 = (float)m->d.beta1, b2 = (float)m->d.beta2;
    const float c1 = (float)(1.0 - std::pow(m->d.beta1, (double)m->adam_t));
    const float c2 = (float)(1.0 - std::pow(m->d.beta2, (double)m->adam_t));
    for (int l = 0; l < NL; ++l) {
        const int nw = COUT[l] * CIN[l] * 27;
        k_adam<<<nbl(nw), 256, 0, st>>>(m->w[l], t.gw[l], m->mw[l], m->vw[l], nw, (float)m->d.lr, b1, b2,
                                        (float)m->d.eps, c1, c2);
        k_adam<<<nbl(COUT[l]), 256, 0, st>>>(m->b[l], t.gb[l], m->mb[l], m->vb[l], COUT[l], (float)m->d.lr, b1, b2,
                                             (float)m->d.eps, c1, c2);
    }
    if ((s = model_repack(m)) != HYB_OK) return s;
    HYB_CUDA_TRY(cudaMemcpyAsync(hp.data(), t.lpart, sizeof(double) * 3 * t.lblocks, cudaMemcpyDeviceToHost, st));
    int stw = 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(&stw, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HYB_CUDA_TRY(cudaStreamSynchronize(st));
    if (stw) return set_error(HYB_ETIMEOUT, "a tensor-core wait gave up");
    double L = 0, bce = 0, acc = 0;
    for (int k = 0; k < t.lblocks; ++k) {
        L += hp[3 * k];
        bce += hp[3 * k + 1];
        acc += hp[3 * k + 2];
    }
    out->loss = L / (double)cells;
    out->bce = bce / (double)cells;
    out->accuracy = acc / (double)cells;
    out->step = m->adam_t;
    return HYB_OK;
}

hyb_status hyb_model_get_grad(hyb_model *m, int l, float *gw, float *gb) {
    if (!m || l < 0 || l >= NL || !m->train) return set_error(HYB_EINVAL, "no gradients (no training step yet)");
    TrainBufs &t = *static_cast<TrainBufs *>(m->train);
    if (gw) HYB_CUDA_TRY(cudaMemcpyAsync(gw, t.gw[l], sizeof(float) * COUT[l] * CIN[l] * 27, cudaMemcpyDeviceToHost, m->stream));
    if (gb) HYB_CUDA_TRY(cudaMemcpyAsync(gb, t.gb[l], sizeof(float) * COUT[l], cudaMemcpyDeviceToHost, m->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return HYB_OK;
}

}  // extern "C"
