// Weight gradients on the 5th-generation tensor cores, for the 3x3x3
// convolutions of the regime classifier and the field surrogate and for the
// dense layers of SwitchNet (paper, Methodology and Results: the networks are
// trained on data the simulation generates).
//
//   dW[co][ci][t] = sum over cells of dZ[cell][co] X[cell + s(t)][ci]
//
// is a contraction over the cells.  Both operands are first laid out over
// the zero-padded volume (positions p of B x (D+2) x (H+2) x Wp, Wp = W + 2
// rounded up to 16) in chunks of 16 positions, [p / 16][channel][p % 16], so
// that a cell's neighbour along z or y is a shift by whole chunks and the 16
// positions of every channel of one chunk are one contiguous block (one TMA
// box, one stretch of memory); the x-shift comes from three copies of dZ
// shifted by -1, 0, +1 in x.  With p' = p - s(t):
//   dW[co][ci][t] = sum_p ZT_dx[co][p - s_zy(t)] XT[ci][p],
// so the MMA's M rows are (tap, co) pairs of several taps -- each a TMA box
// of ZT at its own shifted coordinate -- and its N columns are ci; K runs
// over the positions.  Taps are grouped 128 / COP per MMA; every group has
// its own TMEM accumulator.  The positions are split across the CTAs
// (split-K); each CTA writes its FP32 partial sums, and a reduction adds the
// partials in CTA order (deterministic) into the [co][ci][t] gradient.
// A dense layer is the same with one tap and no padding.
//   warp 0      TMA producer: per K-step of 16 positions one box of XT and
//               one box of ZT per tap slot, into a ring of stages;
//   warp 1      MMA issuer: one tcgen05.mma (128 x N x 16) per tap group;
//   warps 2..5  epilogue at the end of the CTA's range: tcgen05.ld of every
//               accumulator, FP32 partials to global memory.
// Waits are bounded (ST_TIMEOUT on giving up, as in the convolutions).
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"

namespace hyb {

static constexpr long long WG_MBAR_LIMIT = 1LL << 26;
static constexpr int WG_MAX_SLOTS = 32;

struct WgradTcArgs {
    float *part;             // [grid][G][128][N] FP32 partials
    long long ksteps;        // K-steps of 16 positions
    int nslots;              // tap slots used (<= G * TG)
    int nboxes;              // ZT boxes per K-step
    int box_rows;            // rows of one ZT box (the slots of its taps times COP)
    int koff[WG_MAX_SLOTS];  // per box: shift of the box in chunks of 16 positions
    int xrow;                // first XT row of the N columns
    int *status;
};

// box of (16 positions, rows) of the chunked layout at (row r0, chunk k)
__device__ __forceinline__ void tma_load_chunk(uint32_t dst, const void *tmap, int r0, int k, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"(tmap), "r"(0), "r"(r0), "r"(k), "r"(mbar)
        : "memory");
}

template <int COP, int N>
struct WgCfg {
    static constexpr int TG = 128 / COP;                             // tap slots per MMA
    static constexpr int BBYTES = N * 32;                            // XT box: N rows x 16 positions
    static constexpr int ABYTES = COP * 32;                          // one ZT box
    static constexpr int GMAX = N <= 32 ? 7 : 1;                     // tap groups (27 taps: 7 of 4 or 4 of 8)
    static constexpr int STAGE = ((BBYTES + GMAX * 4096) + 1023) / 1024 * 1024;
    static constexpr int SMEM_MAX = 227 * 1024 - 1024;
    static constexpr int STAGES = (SMEM_MAX - 1024) / STAGE > 6 ? 6 : (SMEM_MAX - 1024) / STAGE;
    static constexpr int SMEM = STAGES * STAGE + 1024;
    static constexpr int TCOLS = GMAX * N <= 32 ? 32 : (GMAX * N <= 64 ? 64 : (GMAX * N <= 128 ? 128 :
                                 (GMAX * N <= 256 ? 256 : 512)));
    static constexpr int NTHREADS = 192;
};

template <int COP, int N>
__global__ void __launch_bounds__(192, 1) k_wgrad_tc(const __grid_constant__ CUtensorMap tz,
                                                     const __grid_constant__ CUtensorMap tx,
                                                     const __grid_constant__ WgradTcArgs a) {
    using Cfg = WgCfg<COP, N>;
    constexpr int STAGES = Cfg::STAGES, TG = Cfg::TG;
    static_assert(STAGES >= 2, "shared memory holds fewer than two stages");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_b[STAGES], empty_b[STAGES], done_b;
    __shared__ uint32_t taddr_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = (a.nslots + TG - 1) / TG;
    if (warp == 1) {
        tmem_alloc(smem_u32(&taddr_s), Cfg::TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full_b[s]), 1);
            mbar_init(smem_u32(&empty_b[s]), 1);
        }
        mbar_init(smem_u32(&done_b), 1);
        abort_s = 0;
        fence_mbar_init();
        prefetch_tmap(&tz);
        prefetch_tmap(&tx);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = taddr_s;
    // this CTA's K-steps
    const long long per = (a.ksteps + gridDim.x - 1) / gridDim.x;
    const long long k0 = (long long)blockIdx.x * per, k1 = min(k0 + per, a.ksteps);
    const uint32_t ring_s = smem_u32(ring);
    const uint32_t box_bytes = (uint32_t)(a.box_rows * 32);
    const uint32_t stage_bytes = (uint32_t)Cfg::BBYTES + (uint32_t)a.nboxes * box_bytes;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            long long issued = 0;
            for (long long k = k0; k < k1; ++k) {
                if (!mbar_wait(smem_u32(&empty_b[s]), ph ^ 1, WG_MBAR_LIMIT) || *(volatile int *)&abort_s) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                    break;
                }
                const uint32_t fb = smem_u32(&full_b[s]);
                mbar_arrive_expect_tx(fb, stage_bytes);
                const uint32_t st = ring_s + (uint32_t)(s * Cfg::STAGE);
                tma_load_chunk(st, &tx, a.xrow, (int)k, fb);
                // the boxes land back to back: row (tap, co) of the A tiles is tap * COP + co
                for (int bx = 0; bx < a.nboxes; ++bx)
                    tma_load_chunk(st + (uint32_t)Cfg::BBYTES + (uint32_t)bx * box_bytes, &tz, 0, (int)k - a.koff[bx], fb);
                ++issued;
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1;
                }
            }
            if (*(volatile int *)&abort_s) {
                for (int k = 0; k < STAGES && issued > 0; ++k, --issued) {
                    if (--s < 0) {
                        s = STAGES - 1;
                        ph ^= 1;
                    }
                    mbar_wait(smem_u32(&full_b[s]), ph, WG_MBAR_LIMIT);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, N);
            int s = 0;
            uint32_t ph = 0;
            for (long long k = k0; k < k1; ++k) {
                if (!mbar_wait(smem_u32(&full_b[s]), ph, WG_MBAR_LIMIT) || *(volatile int *)&abort_s) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                    break;
                }
                fence_after_sync();
                const uint32_t st = ring_s + (uint32_t)(s * Cfg::STAGE);
                const uint64_t bd = smem_desc_sw32(st, 8 * 32);
                for (int g = 0; g < G; ++g) {
                    const uint64_t ad = smem_desc_sw32(st + (uint32_t)(Cfg::BBYTES + g * 4096), 8 * 32);
                    umma_bf16(taddr + (uint32_t)(g * N), ad, bd, idesc, k != k0);
                }
                umma_commit(smem_u32(&empty_b[s]));
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1;
                }
            }
            umma_commit(smem_u32(&done_b));
        }
    } else {
        // epilogue: the accumulators once every MMA of the range has completed
        const int q = warp & 3;
        const bool ok = k1 > k0 ? mbar_wait(smem_u32(&done_b), 0, WG_MBAR_LIMIT) : true;
        if (!__all_sync(0xffffffffu, ok) || *(volatile int *)&abort_s) {
            if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
        } else {
            fence_after_sync();
            const int row = q * 32 + lane;
            for (int g = 0; g < G; ++g) {
                float *dst = a.part + (((long long)blockIdx.x * G + g) * 128 + row) * N;
                if (k1 <= k0) {
                    for (int c = 0; c < N; ++c) dst[c] = 0.0f;
                    continue;
                }
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float v[16];
                    tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * N + c0), v);
                    float4 *d4 = reinterpret_cast<float4 *>(dst + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(taddr, Cfg::TCOLS);
}

// element (row r, position p) of the chunked layout with R rows
__device__ __forceinline__ long long chunk_idx(long long p, int r, int R) { return ((p >> 4) * R + r) * 16 + (p & 15); }

// channels-last BF16 src [cells][pitch] (channels c0 .. c0 + nc - 1, c0 a
// multiple of 16, c0 + nc rounded up to 16 within the pitch) -> rows r0 ..
// r0 + nc - 1 of the chunked layout (R rows) over the padded volume, at the
// position of the cell shifted by dx along x (dst zeroed before); one thread
// per cell (16-byte loads)
__global__ void k_to_padded(const __nv_bfloat16 *__restrict__ src, int pitch, int c0, int nc, int B, int D, int H,
                            int W, int Wp, int dx, int r0, int R, __nv_bfloat16 *__restrict__ dst) {
    const long long cells = (long long)B * D * H * W;
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    const int x = (int)(cell % W), y = (int)((cell / W) % H), z = (int)((cell / ((long long)W * H)) % D);
    const long long b = cell / ((long long)W * H * D);
    const long long p = ((b * (D + 2) + z + 1) * (H + 2) + y + 1) * Wp + x + 1 + dx;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + cell * pitch + c0);
    for (int g = 0; g * 8 < nc; ++g) {
        uint4 u = s4[g];
        const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (g * 8 + j < nc) dst[chunk_idx(p, r0 + g * 8 + j, R)] = h[j];
    }
}

// FP32 [cells] -> BF16 row r0 of the chunked layout (the last layer's dlogit)
__global__ void k_f32_to_padded(const float *__restrict__ src, int B, int D, int H, int W, int Wp, int dx, int r0,
                                int R, __nv_bfloat16 *__restrict__ dst) {
    const long long cells = (long long)B * D * H * W;
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    const int x = (int)(cell % W), y = (int)((cell / W) % H), z = (int)((cell / ((long long)W * H)) % D);
    const long long b = cell / ((long long)W * H * D);
    dst[chunk_idx(((b * (D + 2) + z + 1) * (H + 2) + y + 1) * Wp + x + 1 + dx, r0, R)] = __float2bfloat16_rn(src[cell]);
}

// channels-last BF16 src [cells][pitch] (as k_to_padded) -> rows 0 .. nc - 1 of
// the chunked layout (R rows) over the cells (dense layers)
__global__ void k_to_cm(const __nv_bfloat16 *__restrict__ src, int pitch, int c0, int nc, long long cells, int R,
                        __nv_bfloat16 *__restrict__ dst) {
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + cell * pitch + c0);
    for (int g = 0; g * 8 < nc; ++g) {
        uint4 u = s4[g];
        const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (g * 8 + j < nc) dst[chunk_idx(cell, g * 8 + j, R)] = h[j];
    }
}

// out[c] = sum over k of part[k][c] (nk rows of nc columns): one block per
// column, thread i adds rows i, i + 256, ... in order, then a fixed-shape tree
// (the same sum in every run)
__global__ void __launch_bounds__(256) k_sum_cols(const float *__restrict__ part, int nk, int nc,
                                                  float *__restrict__ out) {
    __shared__ float sh[256];
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int k = threadIdx.x; k < nk; k += 256) s += part[(long long)k * nc + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// bias partials of an FP32 gradient of one channel: bpart[blk] = sum over the block's cells
__global__ void k_bias_part_f32(const float *__restrict__ dz, long long cells, long long per, float *__restrict__ bpart) {
    if (threadIdx.x != 0) return;
    const long long a0 = blockIdx.x * per, a1 = min(a0 + per, cells);
    float s = 0.0f;
    for (long long i = a0; i < a1; ++i) s += dz[i];
    bpart[blockIdx.x] = s;
}

// gw[co][ci][t] (ci_tot inputs, nt taps; rows co0.., columns ci0..) = sum over
// CTAs in order of part[cta][slot / TG][(slot % TG) * COP + co][ci]
__global__ void k_wgrad_tc_reduce(const float *__restrict__ part, int ncta, int G, int N, int COP, int TG, int nt,
                                  int co_n, int ci_n, int co0, int ci0, int ci_tot, float *__restrict__ gw) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nt * co_n * ci_n) return;
    const int ci = o % ci_n, co = (o / ci_n) % co_n, t = o / (ci_n * co_n);
    const int g = t / TG, j = t % TG, row = j * COP + co;
    float s = 0.0f;
    for (int k = 0; k < ncta; ++k) s += part[(((long long)k * G + g) * 128 + row) * N + ci];
    gw[((long long)(co0 + co) * ci_tot + ci0 + ci) * nt + t] = s;
}

// bias gradient partials: bpart[blk][c] = sum over the block's cells of dZ[cell][c0 + c] (c < nc)
__global__ void __launch_bounds__(256) k_bias_part(const __nv_bfloat16 *__restrict__ dz, int pitch, int c0, int nc,
                                                   long long cells, long long per, float *__restrict__ bpart) {
    // thread t: channel t % nc over the cells t / nc, t / nc + R, ... of the block's range (R = 256 / nc),
    // then the R row sums of each channel in order
    __shared__ float sh[256];
    const int R = 256 / nc, t = threadIdx.x, c = t % nc, r = t / nc;
    const long long a0 = blockIdx.x * per, a1 = min(a0 + per, cells);
    float s = 0.0f;
    if (r < R)
        for (long long i = a0 + r; i < a1; i += R) s += __bfloat162float(dz[i * pitch + c0 + c]);
    sh[t] = s;
    __syncthreads();
    if (t < nc) {
        float b = 0.0f;
        for (int k = 0; k < R; ++k) b += sh[k * nc + t];
        bpart[(long long)blockIdx.x * nc + t] = b;
    }
}

typedef CUresult (*EncodeTiledFn3)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn3 encode_fn3() {
    static EncodeTiledFn3 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn3)p;
    });
    return fn;
}

// 3D map over the chunked layout [P / 16][rows][16] (BF16), box (16 positions, box_rows, 1 chunk)
static hyb_status cm_map(CUtensorMap *tm, const __nv_bfloat16 *base, long long P, int rows, int box_rows) {
    EncodeTiledFn3 enc = encode_fn3();
    if (!enc) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[3] = {16, (cuuint64_t)rows, (cuuint64_t)(P / 16)};
    const cuuint64_t strides[2] = {32, (cuuint64_t)rows * 32};
    const cuuint32_t box[3] = {16, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return HYB_OK;
}

template <int COP, int N>
static hyb_status wg_launch(const CUtensorMap &tz, const CUtensorMap &tx, const WgradTcArgs &a, int grid,
                            cudaStream_t st) {
    using Cfg = WgCfg<COP, N>;
    static std::mutex mu;
    static int ready_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return set_error(HYB_EINVAL, "device index out of range");
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready_dev[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<COP, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM);
            if (e != cudaSuccess)
                return set_error(HYB_ECUDA, std::string("wgrad smem attribute: ") + cudaGetErrorString(e));
            ready_dev[dev] = 1;
        }
    }
    k_wgrad_tc<COP, N><<<grid, Cfg::NTHREADS, Cfg::SMEM, st>>>(tz, tx, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("wgrad launch: ") + cudaGetErrorString(e));
    return HYB_OK;
}

static int n_sms() {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    return nsm;
}

hyb_status wgrad_tc(const WgradJob &j, WgradScratch &ws, cudaStream_t st) {
    const bool conv = j.taps == 27;
    if (!(j.taps == 27 || j.taps == 1)) return set_error(HYB_EINVAL, "wgrad: 27 or 1 taps");
    const long long cells = (long long)j.B * j.D * j.H * j.W;
    if (cells < 1 || j.co_n < 1 || j.ci_n < 1) return set_error(HYB_EINVAL, "wgrad: empty operand");
    if (cells >= (1LL << 30)) return set_error(HYB_EINVAL, "wgrad: more than 2^30 cells");
    // positions: the padded volume (conv) or the cells (dense)
    const int Wp = conv ? (j.W + 2 + 15) / 16 * 16 : 1;
    const long long P = conv ? (long long)j.B * (j.D + 2) * (j.H + 2) * Wp : cells;
    const long long Pr = (P + 15) / 16 * 16;
    const int cop = j.co_n <= 16 ? 16 : (j.co_n <= 32 ? 32 : 128);
    if (j.co_n > 128 || (!conv && cop != 128) || (conv && cop == 128))
        return set_error(HYB_EINVAL, "wgrad: output block of 1..32 channels (conv) or 1..128 (dense)");
    const int nch_x = (j.ci_n + 15) / 16 * 16;
    const int N = nch_x <= 16 ? 16 : (nch_x <= 32 ? 32 : (nch_x <= 128 ? 128 : 256));
    if (nch_x > 256 || (conv && N > 32)) return set_error(HYB_EINVAL, "wgrad: input block too wide");
    const int ncp = conv ? 3 : 1;
    const long long zbytes = (long long)ncp * cop * Pr * 2, xbytes = (long long)N * Pr * 2;
    if (ws.bytes < zbytes + xbytes) {
        if (ws.buf) cudaFree(ws.buf);
        ws.buf = nullptr;
        ws.bytes = 0;
        if (cudaMalloc(&ws.buf, (size_t)(zbytes + xbytes)) != cudaSuccess)
            return set_error(HYB_ENOMEM, "wgrad operand buffers");
        ws.bytes = zbytes + xbytes;
    }
    __nv_bfloat16 *ZT = (__nv_bfloat16 *)ws.buf, *XT = (__nv_bfloat16 *)((char *)ws.buf + zbytes);
    cudaMemsetAsync(ws.buf, 0, (size_t)(zbytes + xbytes), st);
    if (j.ci0 % 16 || j.co0 % 16) return set_error(HYB_EINVAL, "wgrad: channel blocks start at multiples of 16");
    const unsigned nbz = (unsigned)((cells + 255) / 256), nbx = nbz;
    if (conv) {
        // copy dx + 1 holds dZ at the position of the cell shifted by dx along x
        for (int c = 0; c < 3; ++c) {
            if (j.dz_f32)
                k_f32_to_padded<<<nbz, 256, 0, st>>>(j.dz_f32, j.B, j.D, j.H, j.W, Wp, c - 1, c * cop, 3 * cop, ZT);
            else
                k_to_padded<<<nbz, 256, 0, st>>>(j.dz, j.dz_pitch, j.co0, j.co_n, j.B, j.D, j.H, j.W, Wp, c - 1,
                                                 c * cop, 3 * cop, ZT);
        }
        k_to_padded<<<nbx, 256, 0, st>>>(j.x, j.x_pitch, j.ci0, j.ci_n, j.B, j.D, j.H, j.W, Wp, 0, 0, N, XT);
    } else {
        k_to_cm<<<nbz, 256, 0, st>>>(j.dz, j.dz_pitch, j.co0, j.co_n, cells, cop, ZT);
        k_to_cm<<<nbx, 256, 0, st>>>(j.x, j.x_pitch, j.ci0, j.ci_n, cells, N, XT);
    }
    WgradTcArgs a;
    memset(&a, 0, sizeof(a));
    a.ksteps = Pr / 16;
    a.status = j.status;
    a.xrow = 0;
    const int TG = 128 / cop;
    if (conv) {
        // tap t = (dz, dy, dx) = 3 (3 (dz + 1) + dy + 1) + dx + 1: ZT copy dx + 1 at
        // the position shifted back by dz (H + 2) Wp + dy Wp (a multiple of 8
        // positions); the three copies of one (dz, dy) are one box of 3 COP rows
        a.nslots = 27;
        a.nboxes = 9;
        a.box_rows = 3 * cop;
        for (int bx = 0; bx < 9; ++bx) {
            const int dz = bx / 3 - 1, dy = bx % 3 - 1;
            a.koff[bx] = (dz * (j.H + 2) * Wp + dy * Wp) / 16;
        }
    } else {
        a.nslots = 1;
        a.nboxes = 1;
        a.box_rows = cop;
    }
    const int G = (a.nslots + TG - 1) / TG;
    const int grid = (int)std::min<long long>(a.ksteps, (long long)n_sms());
    const long long pneed = (long long)grid * G * 128 * N;
    const long long bneed = 2048LL * 128;
    if (ws.pbytes < (pneed > bneed ? pneed : bneed) * 4) {
        if (ws.part) cudaFree(ws.part);
        ws.part = nullptr;
        ws.pbytes = 0;
        const long long nb = pneed > bneed ? pneed : bneed;
        if (cudaMalloc((void **)&ws.part, (size_t)nb * 4) != cudaSuccess)
            return set_error(HYB_ENOMEM, "wgrad partial buffers");
        ws.pbytes = nb * 4;
    }
    a.part = ws.part;
    CUtensorMap tz, tx;
    hyb_status s = cm_map(&tz, ZT, Pr, ncp * cop, a.box_rows);
    if (s == HYB_OK) s = cm_map(&tx, XT, Pr, N, N);
    if (s != HYB_OK) return s;
    if (cop == 16 && N == 16) s = wg_launch<16, 16>(tz, tx, a, grid, st);
    else if (cop == 16 && N == 32) s = wg_launch<16, 32>(tz, tx, a, grid, st);
    else if (cop == 32 && N == 16) s = wg_launch<32, 16>(tz, tx, a, grid, st);
    else if (cop == 32 && N == 32) s = wg_launch<32, 32>(tz, tx, a, grid, st);
    else if (cop == 128 && N == 16) s = wg_launch<128, 16>(tz, tx, a, grid, st);
    else if (cop == 128 && N == 128) s = wg_launch<128, 128>(tz, tx, a, grid, st);
    else if (cop == 128 && N == 256) s = wg_launch<128, 256>(tz, tx, a, grid, st);
    else return set_error(HYB_EINVAL, "wgrad: unsupported channel block");
    if (s != HYB_OK) return s;
    const int nt = conv ? 27 : 1;
    k_wgrad_tc_reduce<<<(unsigned)((nt * j.co_n * j.ci_n + 255) / 256), 256, 0, st>>>(
        ws.part, grid, G, N, cop, TG, nt, j.co_n, j.ci_n, j.co0, j.ci0, j.ci_tot, j.gw);
    if (j.gb) {
        // bias: per-block sums over the cells, then the blocks in order
        const int nblk = 2048;
        const long long per = (cells + nblk - 1) / nblk;
        float *bpart = ws.part;  // the partials above are consumed by the reduction first (stream order)
        if (j.dz_f32)
            k_bias_part_f32<<<nblk, 32, 0, st>>>(j.dz_f32, cells, per, bpart);
        else
            k_bias_part<<<nblk, 256, 0, st>>>(j.dz, j.dz_pitch, j.co0, j.co_n, cells, per, bpart);
        const int nc = j.dz_f32 ? 1 : j.co_n;
        k_sum_cols<<<nc, 256, 0, st>>>(bpart, nblk, nc, j.gb + j.co0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("wgrad: ") + cudaGetErrorString(e));
    return HYB_OK;
}

}  // namespace hyb
