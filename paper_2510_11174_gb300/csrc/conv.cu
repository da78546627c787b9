// 3x3x3 convolutions of the regime classifier (arXiv 2510.11174, Methodology
// and Results: a convolutional network on per-channel normalised fields, with
// Monte Carlo dropout for uncertainty; here the 3D CNN 6->32->32->16->1 with
// BF16 weights and FP32 accumulation).
//
// k_conv3_tc: implicit GEMM on the 5th-generation tensor cores, persistent
// and warp-specialised.  The three x-taps of the stencil go into the N
// dimension: for each of the 9 (dz, dy) taps one tcgen05.mma multiplies the
// 128 input cells of a 16 (x) x 8 (y) x 1 (z) block, shifted by (dz, dy), by
// the weights of all three x-taps side by side (N = 3 C_out), so every A tile
// read from shared memory feeds three times the math (the A-operand fetch,
// not the math, limits narrow layers).  The epilogue adds the three partial
// sums of neighbouring x cells (lanes m - 1, m, m + 1, one warp shuffle each
// way), so a tile yields the 14 (x) x 8 (y) interior outputs of its block;
// tiles step by 14 cells in x.  The block halo (16 x 10 x 3 cells) is
// fetched by TMA, one 16-channel block per copy, into a ring of 5 to 8
// shared-memory buffers laid out [block][z][y][x][16 channels] with the
// 32-byte swizzle (the TMA and the tensor core both apply it to the absolute
// shared address, so an operand may start at any cell of the halo); all
// 27 x C_in x C_out weights stay resident in shared memory.
//   warp 0      TMA producer: waits for a free stage, posts the expected bytes
//               on the stage's "full" barrier and issues the chunk copies
//               (zero fill outside the volume comes from the tensor map);
//   warp 1      MMA issuer: per tile 9 taps x C_in/16 tcgen05.mma of shape
//               M = 128 cells x N = 3 C_out x K = 16 into one of 2 or 4 TMEM
//               accumulators; commits free the stage and hand the
//               accumulator to the epilogue;
//   warps 2..   epilogue, one warp per TMEM lane quarter and 8-channel
//               output group (4 C_out / 8 warps; warp w reads TMEM lanes
//               32 (w % 4) .. and channels 8 ((w - 2) / 4) ..): tcgen05.ld of
//               the accumulator rows, the x-tap sum across lanes, bias, ReLU,
//               Philox dropout with inverted scaling, channels-last stores.
//               What does not depend on the accumulator (the tile position,
//               stepped with carries; the cell's validity; the dropout bits;
//               the bias) is computed before waiting for it, so it overlaps
//               the MMAs instead of lengthening the epilogue's chain.
// The operand of tap (dz, dy) is the halo shifted by that tap: its 128 cells
// are 128 consecutive 32-byte rows (one swizzle atom wide in K, 8-row groups
// 256 bytes apart), so every tap and 16-channel block is a plain K-major SW32
// matrix descriptor -- no im2col.
// Every wait is bounded: a wait that gives up sets ST_TIMEOUT, the roles stop
// issuing work, copies and MMAs in flight are waited for (bounded) and TMEM
// is released.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"
#include "philox.cuh"

namespace hyb {

static constexpr int TX = 16, TY = 8;                 // A block (cells): M = 128 rows
static constexpr int TXO = TX - 2;                     // output cells per block row (the interior)
static constexpr int HY = TY + 2, HZ = 3;              // halo (x needs none: the x-taps live in N)
static constexpr int HCELLS = TX * HY * HZ;            // 480
static constexpr int CHB = HCELLS * 32;                // bytes one 16-channel copy writes (15360)
static constexpr int CHBP = (CHB + 1023) / 1024 * 1024; // block pitch in shared memory (15360)
static constexpr long long MBAR_LIMIT = 1LL << 26;     // polls before a wait gives up

// dropout keep decision of channel ch at cell (b, lin): Philox counter
// (lin, b, (layer << 16) | (ch >> 3), pass), key (seed, 0xD0); 16-bit field
// ch & 7 of the output (word (ch & 7) >> 1, low half for even ch); kept when
// the field is >= thr = round(p 2^16)
__host__ __device__ inline bool dropout_keep(uint32_t seed, uint32_t pass, uint32_t layer, uint32_t b, uint32_t lin,
                                             int ch, uint32_t thr) {
    const u32x4 r = philox4x32_10(lin, b, (layer << 16) | ((uint32_t)ch >> 3), pass, seed, 0xD0u);
    const uint32_t f = (r.v[(ch & 7) >> 1] >> (16 * (ch & 1))) & 0xFFFFu;
    return f >= thr;
}

// the tile columns (x) a launch covers: all, or those whose 14 outputs per
// row meet the requested x-range
__host__ __device__ inline void conv_tiles_x(int W, int x_lo, int x_hi, int &tx0, int &ntx) {
    const int all = (W + TXO - 1) / TXO;
    if (x_hi > x_lo) {
        tx0 = x_lo / TXO;
        const int tx1 = (x_hi + TXO - 1) / TXO;
        ntx = (tx1 < all ? tx1 : all) - tx0;
        if (ntx < 0) ntx = 0;
    } else {
        tx0 = 0;
        ntx = all;
    }
}

// position of a persistent CTA's tile in (x tile, y tile, z, batch) digits,
// stepped by the grid size with carries instead of divisions
struct TileCursor {
    int tx, ty, z, b;        // the current tile
    int sx, sy, sz, sb;      // the step (grid size) in the same digits
    int nx, ny, nz;
    __device__ void init(uint32_t t, uint32_t step, int nx_, int ny_, int nz_) {
        nx = nx_;
        ny = ny_;
        nz = nz_;
        tx = (int)(t % (uint32_t)nx);
        t /= (uint32_t)nx;
        ty = (int)(t % (uint32_t)ny);
        t /= (uint32_t)ny;
        z = (int)(t % (uint32_t)nz);
        b = (int)(t / (uint32_t)nz);
        sx = (int)(step % (uint32_t)nx);
        step /= (uint32_t)nx;
        sy = (int)(step % (uint32_t)ny);
        step /= (uint32_t)ny;
        sz = (int)(step % (uint32_t)nz);
        sb = (int)(step / (uint32_t)nz);
    }
    __device__ void next() {
        tx += sx;
        int c = tx >= nx;
        tx -= c ? nx : 0;
        ty += sy + c;
        c = ty >= ny;
        ty -= c ? ny : 0;
        z += sz + c;
        c = z >= nz;
        z -= c ? nz : 0;
        b += sb + c;
    }
};

template <int KC, int N>
struct ConvCfg {
    static constexpr int NP = 3 * N;                   // MMA N: the three x-taps side by side
    static constexpr int WBYTES = 27 * KC * N * 16;    // weights, core layout [9][KC][3 N][8]
    static constexpr int RING = (WBYTES + 1023) / 1024 * 1024;  // halo ring offset (swizzle-aligned)
    static constexpr int STAGE = (KC / 2) * CHBP;      // one halo buffer (16-channel blocks)
    // as many halo buffers as shared memory holds (up to 8): the copies in
    // flight must cover the L2 latency of a stage
    static constexpr int SMEM_MAX = 227 * 1024 - 512;  // dynamic share (static barriers take the rest)
    static constexpr int STAGES = (SMEM_MAX - 1024 - RING) / STAGE > 8 ? 8 : (SMEM_MAX - 1024 - RING) / STAGE;
    static constexpr int SMEM = RING + STAGES * STAGE + 1024;  // + alignment slack
    // TMEM accumulators: four when they fit the 512 columns (the MMAs may run
    // three tiles ahead of the slowest epilogue warp), else two
    static constexpr int NACC = 4 * NP <= 512 ? 4 : 2;
    static constexpr int TCOLS = NACC * NP <= 32 ? 32 : (NACC * NP <= 64 ? 64 : (NACC * NP <= 128 ? 128 :
                                 (NACC * NP <= 256 ? 256 : 512)));
    static constexpr int NG = N / 8;                   // 8-channel output groups
    static constexpr int NEPI = 4 * NG;                // epilogue warps: one per lane quarter and group
    static constexpr int NTHREADS = 64 + 32 * NEPI;    // + producer and MMA issuer
};

template <int KC, int N>
__global__ void __launch_bounds__(ConvCfg<KC, N>::NTHREADS, 1)
    k_conv3_tc(const __grid_constant__ CUtensorMap tmap, ConvArgs a) {
    using Cfg = ConvCfg<KC, N>;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned base: weights first, then the halo ring
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *wsm = smem;
    uint8_t *ring = smem + Cfg::RING;
    constexpr int STAGES = Cfg::STAGES;
    static_assert(STAGES >= 2, "shared memory holds fewer than two halo buffers");
    __shared__ __align__(8) uint64_t full_b[STAGES], empty_b[STAGES], tfull_b[Cfg::NACC], tempty_b[Cfg::NACC], done_b;
    __shared__ uint32_t taddr_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 1) {
        tmem_alloc(smem_u32(&taddr_s), Cfg::TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full_b[s]), 1);
            mbar_init(smem_u32(&empty_b[s]), 1);
        }
        for (int k = 0; k < Cfg::NACC; ++k) {
            mbar_init(smem_u32(&tfull_b[k]), 1);
            mbar_init(smem_u32(&tempty_b[k]), Cfg::NEPI);
        }
        mbar_init(smem_u32(&done_b), 1);
        abort_s = 0;
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    // weights: straight 16-byte copies (already in core layout)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.wt);
        uint4 *dst = reinterpret_cast<uint4 *>(wsm);
        for (int i = tid; i < Cfg::WBYTES / 16; i += Cfg::NTHREADS) dst[i] = src[i];
    }
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = taddr_s;
    int tx0, tiles_x;
    conv_tiles_x(a.W, a.x_lo, a.x_hi, tx0, tiles_x);
    const int tiles_y = a.H / TY;
    const long long ntiles = (long long)a.B * a.D * tiles_y * tiles_x;
    const uint32_t ring_s = smem_u32(ring), w_s = smem_u32(wsm);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            long long issued = 0;
            TileCursor cur;
            cur.init(blockIdx.x, gridDim.x, tiles_x, tiles_y, a.D);
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, cur.next()) {
                if (!mbar_wait(smem_u32(&empty_b[s]), ph ^ 1, MBAR_LIMIT) || *(volatile int *)&abort_s) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                    break;
                }
                const int tx = cur.tx + tx0, ty = cur.ty, z0 = cur.z, b = cur.b;
                const uint32_t fb = smem_u32(&full_b[s]);
                mbar_arrive_expect_tx(fb, (KC / 2) * CHB);
                const uint32_t dst = ring_s + (uint32_t)(s * Cfg::STAGE);
#pragma unroll
                for (int c = 0; c < KC / 2; ++c)
                    tma_load_5d(dst + (uint32_t)(c * CHBP), &tmap, a.cin_off + 16 * c, tx * TXO - 1, ty * TY - 1, z0 - 1,
                                b, fb);
                ++issued;
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1;
                }
            }
            // copies still in flight when the loop stopped early complete before exit
            if (*(volatile int *)&abort_s) {
                for (int k = 0; k < STAGES && issued > 0; ++k, --issued) {
                    if (--s < 0) {
                        s = STAGES - 1;
                        ph ^= 1;
                    }
                    mbar_wait(smem_u32(&full_b[s]), ph, MBAR_LIMIT);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, Cfg::NP);
            const uint64_t a0 = smem_desc_sw32(ring_s, 8 * 32);
            const uint64_t b0 = smem_desc(w_s, Cfg::NP * 16, 128);
            int s = 0;
            uint32_t ph = 0;
            long long it = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const int acc = (int)(it % Cfg::NACC);
                const uint32_t aph = (uint32_t)((it / Cfg::NACC) & 1);
                if (!mbar_wait(smem_u32(&tempty_b[acc]), aph ^ 1, MBAR_LIMIT) ||
                    !mbar_wait(smem_u32(&full_b[s]), ph, MBAR_LIMIT) || *(volatile int *)&abort_s) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                    break;
                }
                fence_after_sync();
                const uint32_t d = taddr + (uint32_t)(acc * Cfg::NP);
                const uint64_t as = a0 + (uint64_t)((s * Cfg::STAGE) >> 4);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dz = tap / 3, dy = tap % 3;
                    const uint32_t toff = (uint32_t)((dz * HY + dy) * TX * 32);
#pragma unroll
                    for (int kk = 0; kk < KC / 2; ++kk) {
                        const uint64_t ad = as + (uint64_t)((toff + (uint32_t)(kk * CHBP)) >> 4);
                        const uint64_t bd = b0 + (uint64_t)(((tap * KC + 2 * kk) * Cfg::NP * 16) >> 4);
                        umma_bf16(d, ad, bd, idesc, (tap | kk) != 0);
                    }
                }
                umma_commit(smem_u32(&empty_b[s]));    // the stage may be refilled
                umma_commit(smem_u32(&tfull_b[acc]));  // the accumulator is ready
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1;
                }
            }
            // every MMA issued has finished reading shared memory before exit
            umma_commit(smem_u32(&done_b));
            mbar_wait(smem_u32(&done_b), 0, MBAR_LIMIT);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int grp = (warp - 2) >> 2;     // the 8 output channels 8 grp .. 8 grp + 7 of this warp
        const int m = q * 32 + lane;         // accumulator row = cell of the tile
        const float scale = a.drop_scale;
        const int bx = m & (TX - 1);         // cell of the block row (0 and TX - 1 are halo)
        const long long opitch = a.out_pitch ? a.out_pitch : N;
        float bias8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) bias8[j] = a.bias ? __ldg(a.bias + grp * 8 + j) : 0.0f;
        TileCursor cur;                      // tile counts fit in 32 bits (checked at launch)
        cur.init(blockIdx.x, gridDim.x, tiles_x, tiles_y, a.D);
        long long it = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it, cur.next()) {
            // first what does not need the accumulator (it overlaps the MMAs):
            // the cell, its validity and its dropout bits
            const int tx = cur.tx + tx0, ty = cur.ty, z0 = cur.z, b = cur.b;
            const int cx = tx * TXO + bx - 1, cy = ty * TY + (m >> 4);
            // the halo cells of the block row, and cells past the volume, write nothing
            const bool valid = bx != 0 && bx != TX - 1 && cx < a.W;
            const uint32_t lin = (uint32_t)(((long long)z0 * a.H + cy) * a.W + (valid ? cx : 0));
            const long long obase = ((((long long)b * a.D + z0) * a.H + cy) * a.W + (valid ? cx : 0)) * opitch +
                                    a.out_off + grp * 8;
            uint32_t keep16[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
            if (a.drop_thr) {
                const u32x4 r = philox4x32_10(lin, (uint32_t)b, (a.layer << 16) | (uint32_t)grp, a.pass, a.seed, 0xD0u);
#pragma unroll
                for (int w = 0; w < 4; ++w) keep16[w] = r.v[w];
            }

            const int acc = (int)(it % Cfg::NACC);
            const uint32_t aph = (uint32_t)((it / Cfg::NACC) & 1);
            const bool ok = mbar_wait(smem_u32(&tfull_b[acc]), aph, MBAR_LIMIT);
            if (!__all_sync(0xffffffffu, ok) || *(volatile int *)&abort_s) {
                if (lane == 0) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                }
                break;
            }
            fence_after_sync();
            // row m holds, per x-tap dx, the partial sum of the outputs at cell
            // x - dx + 1; the output at x is D_0[x - 1] + D_1[x] + D_2[x + 1]
            float v[8];
            {
                float p[24];
                const uint32_t rowa = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * Cfg::NP + grp * 8);
                tmem_ld8x3(rowa, rowa + (uint32_t)N, rowa + (uint32_t)(2 * N), p);
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty_b[acc]));
                // lanes m - 1 and m + 1 are the x-neighbours (same block row for
                // the interior cells that produce output)
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const float left = __shfl_up_sync(0xffffffffu, p[o], 1);
                    const float right = __shfl_down_sync(0xffffffffu, p[16 + o], 1);
                    v[o] = left + p[8 + o] + right;
                }
            }
            __nv_bfloat16 *out = a.y ? a.y + obase : nullptr;
            float *outf = a.y_f32 ? a.y_f32 + obase : nullptr;
            if (valid) {
                float r8[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float s = v[j] + bias8[j];
                    if (a.relu) s = fmaxf(s, 0.0f);
                    if (a.scale_out) {
                        const uint32_t f = (keep16[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                        s = f >= a.drop_thr ? s * scale : 0.0f;
                    }
                    r8[j] = s;
                }
                if (outf && a.accum) {
                    // partial sums of one input-channel chunk: add the raw accumulator
                    float4 *o4 = reinterpret_cast<float4 *>(outf);
                    const float4 p0 = o4[0], p1 = o4[1];
                    o4[0] = make_float4(p0.x + v[0], p0.y + v[1], p0.z + v[2], p0.w + v[3]);
                    o4[1] = make_float4(p1.x + v[4], p1.y + v[5], p1.z + v[6], p1.w + v[7]);
                } else if (outf) {
                    reinterpret_cast<float4 *>(outf)[0] = make_float4(r8[0], r8[1], r8[2], r8[3]);
                    reinterpret_cast<float4 *>(outf)[1] = make_float4(r8[4], r8[5], r8[6], r8[7]);
                } else {
                    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(r8[j]);
                    *reinterpret_cast<uint4 *>(out) = *reinterpret_cast<const uint4 *>(o);
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(taddr, Cfg::TCOLS);
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// tensor map of a channels-last BF16 activation [B][D][H][W][C]: dims
// (C, W, H, D, B), box (8 channels, halo x, halo y, halo z, 1)
static hyb_status make_tmap(CUtensorMap *tm, const ConvArgs &a) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t C = (cuuint64_t)(a.cin_total ? a.cin_total : a.cin);
    const cuuint64_t dims[5] = {C, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D, (cuuint64_t)a.B};
    const cuuint64_t es = 2;
    const cuuint64_t strides[4] = {es * C, es * C * a.W, es * C * a.W * a.H, es * C * a.W * a.H * a.D};
    const cuuint32_t box[5] = {16, (cuuint32_t)TX, (cuuint32_t)HY, (cuuint32_t)HZ, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void *)a.x, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return HYB_OK;
}

template <int KC, int N>
static hyb_status launch_cfg(const ConvArgs &a, cudaStream_t st) {
    using Cfg = ConvCfg<KC, N>;
    CUtensorMap tm;
    hyb_status s = make_tmap(&tm, a);
    if (s != HYB_OK) return s;
    // per-device launch set-up, done once (its host cost shows on small grids)
    static std::mutex mu;
    static int ready_dev[64] = {0}, nsm_dev[64] = {0}, per_sm_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return set_error(HYB_EINVAL, "device index out of range");
    int nsm, per_sm;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready_dev[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_conv3_tc<KC, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM);
            if (e != cudaSuccess)
                return set_error(HYB_ECUDA, std::string("conv smem attribute: ") + cudaGetErrorString(e));
            cudaDeviceGetAttribute(&nsm_dev[dev], cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_dev[dev], k_conv3_tc<KC, N>, Cfg::NTHREADS,
                                                          Cfg::SMEM);
            ready_dev[dev] = 1;
        }
        nsm = nsm_dev[dev];
        per_sm = per_sm_dev[dev];
    }
    cudaError_t e;
    int tx0, ntx;
    conv_tiles_x(a.W, a.x_lo, a.x_hi, tx0, ntx);
    const long long ntiles = (long long)a.B * a.D * (a.H / TY) * ntx;
    if (ntiles == 0) return HYB_OK;
    const long long grid = std::min<long long>(ntiles, (long long)nsm * std::max(per_sm, 1));
    k_conv3_tc<KC, N><<<(unsigned)grid, Cfg::NTHREADS, Cfg::SMEM, st>>>(tm, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("conv launch: ") + cudaGetErrorString(e));
    return HYB_OK;
}

hyb_status launch_conv3_tc(const ConvArgs &a, cudaStream_t st) {
    if (a.W < 1 || a.H % TY != 0 || a.B < 1 || a.D < 1)
        return set_error(HYB_EINVAL, "conv shape: H % 8 == 0 required");
    if ((long long)a.B * a.D * (a.H / TY) * ((a.W + TXO - 1) / TXO) >= (1LL << 31))
        return set_error(HYB_EINVAL, "conv shape: more than 2^31 tiles");
    if (((uintptr_t)a.x & 15) || ((uintptr_t)a.y & 15) || ((uintptr_t)a.y_f32 & 15) || ((uintptr_t)a.wt & 15) ||
        (!a.y && !a.y_f32))
        return set_error(HYB_EINVAL, "conv operands must be present and 16-byte aligned");
    {
        // channel chunks: 16-channel aligned input slices (TMA x coordinate in
        // 32-byte steps), 8-channel aligned output slices (16-byte stores)
        const int ct = a.cin_total ? a.cin_total : a.cin, op = a.out_pitch ? a.out_pitch : a.N;
        if (ct % 16 || a.cin_off < 0 || a.cin_off % 16 || a.cin_off + a.cin > ct || op % 8 || a.out_off < 0 ||
            a.out_off % 8 || a.out_off + a.N > op || (a.accum && !a.y_f32))
            return set_error(HYB_EINVAL, "conv channel slices out of range or misaligned");
    }
    if (a.cin == 16 && a.N == 32) return launch_cfg<2, 32>(a, st);
    if (a.cin == 32 && a.N == 32) return launch_cfg<4, 32>(a, st);
    if (a.cin == 32 && a.N == 16) return launch_cfg<4, 16>(a, st);
    if (a.cin == 16 && a.N == 16) return launch_cfg<2, 16>(a, st);
    return set_error(HYB_EINVAL, "conv channels: (C_in, C_out) in {16, 32} x {16, 32}");
}


// ---------------------------------------------------------------- last layer
// k_conv_last_tc: the 16 -> 1 channel layer with all 27 taps in the MMA N
// dimension.  A plane block of 16 (x) x 8 (y) cells (M = 128 rows, K = the 16
// channels) times the weights of the 27 taps (N = 32, padded) gives, per cell
// c and tap t, the partial product P[c][t] = sum_ci x[c][ci] w[t][ci] -- one
// MMA per plane.  The output at cell c is y[c] = b + sum_t P[c + offset(t)][t]:
// the z part of the sum runs in registers (a cell's own partials of three
// consecutive planes), the in-plane 3 x 3 part through shared memory; the
// 14 x 6 interior cells of the block have all their neighbours in it.  A CTA walks a column of such blocks through z
// (chunks of LZC output planes plus one plane of halo on either side), so
// every plane is multiplied once and used by three output planes.
//   warp 0      TMA producer: one 16 x 8 x 1 x 16-channel box per plane
//               (zero fill outside the volume) into a ring of LSTAGES;
//   warp 1      MMA issuer: one tcgen05.mma (128 x 32 x 16) per plane into
//               one of two TMEM accumulators;
//   warps 2..5  epilogue: tcgen05.ld of the 32 columns, the z sums in
//               registers, the 9 in-plane partials of the completed output
//               plane into shared memory, a named barrier of the four warps,
//               the 3 x 3 gather, bias, and the logit or the sigmoid folded
//               into the MC mean / M2 (Welford).
// Waits are bounded; a warp whose wait gives up records ST_TIMEOUT and stops
// waiting, but the epilogue warps keep meeting at their barrier until the
// end, so no warp is left behind at it.
static constexpr int LTX = 16, LTY = 8;            // block (cells) = 128 MMA rows
static constexpr int LOX = LTX - 2, LOY = LTY - 2; // interior outputs per block row / column
static constexpr int LZC = 32;                     // output planes per work unit
static constexpr int LSTAGES = 4;
static constexpr int LCTAS = 4;                    // CTAs per SM (64 TMEM columns each)
static constexpr int LPF = 3;                      // planes of MC statistics read ahead
static constexpr int LSTAGE = LTX * LTY * 32;      // bytes of one plane block (4096)
static constexpr int LSMEM = LSTAGES * LSTAGE + 2 * 9 * 128 * 4 + 1024 + 1024;  // ring, 2 x Q, weights, slack

struct LastTiles {
    int tx0, tx_n, ty_n, zc_n;
    long long units;
};

// work units of the last layer: all block columns, or those whose outputs
// meet x_lo <= x < x_hi when x_hi > x_lo
__host__ __device__ inline LastTiles last_tiles(int B, int D, int H, int W, int x_lo, int x_hi) {
    LastTiles t;
    const int all = (W + LOX - 1) / LOX;
    if (x_hi > x_lo) {
        t.tx0 = x_lo / LOX;
        const int tx1 = (x_hi + LOX - 1) / LOX;
        t.tx_n = (tx1 < all ? tx1 : all) - t.tx0;
        if (t.tx_n < 0) t.tx_n = 0;
    } else {
        t.tx0 = 0;
        t.tx_n = all;
    }
    t.ty_n = (H + LOY - 1) / LOY;
    t.zc_n = (D + LZC - 1) / LZC;
    t.units = (long long)B * t.zc_n * t.ty_n * t.tx_n;
    return t;
}

// unit u -> block position and z range; planes z = zlo - 1 .. zhi
__device__ inline void last_unit(long long u, const LastTiles &t, int D, int &tx, int &ty, int &zlo, int &zhi,
                                 int &b) {
    tx = (int)(u % t.tx_n) + t.tx0;
    u /= t.tx_n;
    ty = (int)(u % t.ty_n);
    u /= t.ty_n;
    const int zc = (int)(u % t.zc_n);
    b = (int)(u / t.zc_n);
    zlo = zc * LZC;
    zhi = min(zlo + LZC, D);
}

__global__ void __launch_bounds__(192, LCTAS) k_conv_last_tc(const __grid_constant__ CUtensorMap tmap,
                                                      const __grid_constant__ LastArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = smem;                                          // LSTAGES x 4 KB (1 KB aligned)
    uint8_t *wsm = smem + LSTAGES * LSTAGE;                        // 1 KB of weights
    float *qs = reinterpret_cast<float *>(wsm + 1024);             // [2][9][128] in-plane partials Q
    __shared__ __align__(8) uint64_t full_b[LSTAGES], empty_b[LSTAGES], tfull_b[2], tempty_b[2], done_b;
    __shared__ uint32_t taddr_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 1) {
        tmem_alloc(smem_u32(&taddr_s), 64);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < LSTAGES; ++s) {
            mbar_init(smem_u32(&full_b[s]), 1);
            mbar_init(smem_u32(&empty_b[s]), 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(smem_u32(&tfull_b[k]), 1);
            mbar_init(smem_u32(&tempty_b[k]), 4);
        }
        mbar_init(smem_u32(&done_b), 1);
        abort_s = 0;
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    for (int i = tid; i < 256; i += 192) reinterpret_cast<uint32_t *>(wsm)[i] = a.w[i];
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = taddr_s;
    const LastTiles lt = last_tiles(a.B, a.D, a.H, a.W, a.x_lo, a.x_hi);
    const uint32_t ring_s = smem_u32(ring), w_s = smem_u32(wsm);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            long long issued = 0;
            bool stop = false;
            for (long long u = blockIdx.x; u < lt.units && !stop; u += gridDim.x) {
                int tx, ty, zlo, zhi, b;
                last_unit(u, lt, a.D, tx, ty, zlo, zhi, b);
                for (int z = zlo - 1; z <= zhi; ++z) {
                    if (!mbar_wait(smem_u32(&empty_b[s]), ph ^ 1, MBAR_LIMIT) || *(volatile int *)&abort_s) {
                        atomicOr(a.status, ST_TIMEOUT);
                        *(volatile int *)&abort_s = 1;
                        stop = true;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_b[s]);
                    mbar_arrive_expect_tx(fb, LSTAGE);
                    tma_load_5d(ring_s + (uint32_t)(s * LSTAGE), &tmap, 0, tx * LOX - 1, ty * LOY - 1, z, b, fb);
                    ++issued;
                    if (++s == LSTAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (*(volatile int *)&abort_s) {
                for (int k = 0; k < LSTAGES && issued > 0; ++k, --issued) {
                    if (--s < 0) {
                        s = LSTAGES - 1;
                        ph ^= 1;
                    }
                    mbar_wait(smem_u32(&full_b[s]), ph, MBAR_LIMIT);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, 32);
            const uint64_t a0 = smem_desc_sw32(ring_s, 8 * 32);
            const uint64_t bd = smem_desc(w_s, 32 * 16, 128);
            int s = 0;
            uint32_t ph = 0;
            long long it = 0;
            bool stop = false;
            for (long long u = blockIdx.x; u < lt.units && !stop; u += gridDim.x) {
                int tx, ty, zlo, zhi, b;
                last_unit(u, lt, a.D, tx, ty, zlo, zhi, b);
                for (int z = zlo - 1; z <= zhi; ++z, ++it) {
                    const int acc = (int)(it & 1);
                    const uint32_t aph = (uint32_t)((it >> 1) & 1);
                    if (!mbar_wait(smem_u32(&tempty_b[acc]), aph ^ 1, MBAR_LIMIT) ||
                        !mbar_wait(smem_u32(&full_b[s]), ph, MBAR_LIMIT) || *(volatile int *)&abort_s) {
                        atomicOr(a.status, ST_TIMEOUT);
                        *(volatile int *)&abort_s = 1;
                        stop = true;
                        break;
                    }
                    fence_after_sync();
                    umma_bf16(taddr + (uint32_t)(acc * 32), a0 + (uint64_t)((s * LSTAGE) >> 4), bd, idesc, 0);
                    umma_commit(smem_u32(&empty_b[s]));
                    umma_commit(smem_u32(&tfull_b[acc]));
                    if (++s == LSTAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            umma_commit(smem_u32(&done_b));
            mbar_wait(smem_u32(&done_b), 0, MBAR_LIMIT);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // With P_z[c][t] the partials of plane z, the output of plane o at
        // cell c is b + sum over (dy, dx) of Q_o[c + (dy - 1, dx - 1)][dy, dx],
        // where Q_o[c][dy, dx] = sum over dz of P_{o + dz - 1}[c][(dz, dy, dx)]
        // needs only the cell's own rows: each thread accumulates it in
        // registers as the planes stream past (r1: plane o + 1's part so far,
        // r2: plane o's), and only the 9 values of Q cross threads, through a
        // double-buffered shared array and one barrier per plane.
        const int q = warp & 3;
        const int m = q * 32 + lane;                 // row = cell of the block
        const int lx = m & (LTX - 1), ly = m >> 4;
        const bool interior = lx >= 1 && lx <= LOX && ly >= 1 && ly <= LOY;
        const float inv_k = a.mc_k > 0 ? 1.0f / (float)a.mc_k : 0.0f;  // the Welford weight of this pass
        bool dead = false;
        const long long V = (long long)a.D * a.H * a.W;
        long long it = 0;
        for (long long u = blockIdx.x; u < lt.units; u += gridDim.x) {
            int tx, ty, zlo, zhi, b;
            last_unit(u, lt, a.D, tx, ty, zlo, zhi, b);
            const int cx = tx * LOX + lx - 1, cy = ty * LOY + ly - 1;
            // with an x-range, the block's cells outside it keep their statistics
            const bool valid = interior && cx < a.W && cy < a.H && (a.x_hi <= a.x_lo || (cx >= a.x_lo && cx < a.x_hi));
            float r1[9], r2[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) r1[k] = r2[k] = 0.0f;
            // MC statistics of output planes zo .. zo + LPF - 1, read LPF planes
            // ahead so that their latency spans several planes
            // (at the top of the iteration for output plane zo, entry k holds plane zo + k)
            const long long HW = (long long)a.H * a.W;
            const long long t0 = (long long)b * V + ((long long)(zlo - 2) * a.H + cy) * a.W + cx;
            float pmq[LPF], m2q[LPF];
#pragma unroll
            for (int k = 0; k < LPF; ++k) {
                pmq[k] = m2q[k] = 0.0f;
                const int zk = zlo - 2 + k;
                if (valid && a.mc_k >= 2 && zk >= zlo && zk < zhi) {
                    pmq[k] = a.pm[t0 + k * HW];
                    m2q[k] = a.m2[t0 + k * HW];
                }
            }
            for (int z = zlo - 1; z <= zhi; ++z, ++it) {
                const int acc = (int)(it & 1);
                const uint32_t aph = (uint32_t)((it >> 1) & 1);
                const int zo = z - 1;                // output plane completed by plane z
                const bool out = valid && zo >= zlo;
                const long long t = (long long)b * V + ((long long)zo * a.H + cy) * a.W + cx;
                const float mo = pmq[0], m2o = m2q[0];
#pragma unroll
                for (int k = 0; k + 1 < LPF; ++k) {
                    pmq[k] = pmq[k + 1];
                    m2q[k] = m2q[k + 1];
                }
                pmq[LPF - 1] = m2q[LPF - 1] = 0.0f;
                if (valid && a.mc_k >= 2 && zo + LPF >= zlo && zo + LPF < zhi) {
                    pmq[LPF - 1] = a.pm[t + LPF * HW];
                    m2q[LPF - 1] = a.m2[t + LPF * HW];
                }
                if (!dead) {
                    const bool ok = mbar_wait(smem_u32(&tfull_b[acc]), aph, MBAR_LIMIT) &&
                                    !*(volatile int *)&abort_s;
                    if (!__all_sync(0xffffffffu, ok)) {
                        if (lane == 0) {
                            atomicOr(a.status, ST_TIMEOUT);
                            *(volatile int *)&abort_s = 1;
                        }
                        dead = true;
                    }
                }
                float p[32];
                if (!dead) {
                    fence_after_sync();
                    tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 32), p);
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&tempty_b[acc]));
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) p[k] = 0.0f;
                }
                // plane z is tap dz = 2 of output zo, dz = 1 of zo + 1, dz = 0 of zo + 2
                float *qb = qs + (int)(it & 1) * (9 * 128);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    qb[k * 128 + m] = r2[k] + p[18 + k];
                    r2[k] = r1[k] + p[9 + k];
                    r1[k] = p[k];
                }
                // Q of plane zo is complete (and the buffer written two planes
                // ago is no longer read): the four epilogue warps meet
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (!dead && out) {
                    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        s0 += qb[(0 * 3 + dx) * 128 + m - LTX + dx - 1];
                        s1 += qb[(1 * 3 + dx) * 128 + m + dx - 1];
                        s2 += qb[(2 * 3 + dx) * 128 + m + LTX + dx - 1];
                    }
                    const float logit = a.bias + s0 + s1 + s2;
                    if (a.mc_k == 0) {
                        a.logit[t] = logit;
                    } else {
                        const float pv = __frcp_rn(1.0f + __expf(-logit));
                        if (a.mc_k == 1) {
                            a.pm[t] = pv;
                            a.m2[t] = 0.0f;
                        } else {
                            const float d = pv - mo;
                            const float mn = mo + d * inv_k;
                            a.pm[t] = mn;
                            a.m2[t] = m2o + d * (pv - mn);
                        }
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(taddr, 64);
}

hyb_status launch_conv_last_tc(const LastArgs &a, cudaStream_t st) {
    if (a.B < 1 || a.D < 1 || a.H < 1 || a.W < 1) return set_error(HYB_EINVAL, "last layer: empty volume");
    if (((uintptr_t)a.x & 15) || (a.mc_k == 0 && !a.logit) || (a.mc_k > 0 && (!a.pm || !a.m2)))
        return set_error(HYB_EINVAL, "last layer: operands missing or not 16-byte aligned");
    const LastTiles lt = last_tiles(a.B, a.D, a.H, a.W, a.x_lo, a.x_hi);
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled is not available");
    CUtensorMap tm;
    const cuuint64_t dims[5] = {16, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D, (cuuint64_t)a.B};
    const cuuint64_t strides[4] = {32ull, 32ull * a.W, 32ull * a.W * a.H, 32ull * a.W * a.H * a.D};
    const cuuint32_t box[5] = {16, (cuuint32_t)LTX, (cuuint32_t)LTY, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void *)a.x, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(HYB_ECUDA, "last layer: tensor map (" + std::to_string((int)r) + ")");
    static std::mutex mu;
    static int ready_dev[64] = {0}, nsm_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return set_error(HYB_EINVAL, "device index out of range");
    int nsm;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready_dev[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_conv_last_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, LSMEM);
            if (e != cudaSuccess)
                return set_error(HYB_ECUDA, std::string("last layer smem attribute: ") + cudaGetErrorString(e));
            cudaDeviceGetAttribute(&nsm_dev[dev], cudaDevAttrMultiProcessorCount, dev);
            ready_dev[dev] = 1;
        }
        nsm = nsm_dev[dev];
    }
    // LCTAS CTAs per SM by registers and shared memory (the occupancy query
    // answers 1 for kernels that allocate tensor memory); units are
    // independent, so any residency gives the same result
    if (lt.units == 0) return HYB_OK;
    const long long grid = std::min<long long>(lt.units, (long long)nsm * LCTAS);
    k_conv_last_tc<<<(unsigned)grid, 192, LSMEM, st>>>(tm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("last layer launch: ") + cudaGetErrorString(e));
    return HYB_OK;
}

// Self-test of the bounded barrier wait the convolutions use: one thread
// waits on an mbarrier that nothing arrives at, gives up after `polls` polls
// and latches ST_TIMEOUT -- the path a stalled tensor-core pipeline takes.
__global__ void k_wait_selftest(long long polls, int *__restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
        if (!mbar_wait(smem_u32(&bar), 0, polls)) atomicOr(status, ST_TIMEOUT);
    }
}

void launch_wait_selftest(long long polls, int *status, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(polls, status);
}

}  // namespace hyb
