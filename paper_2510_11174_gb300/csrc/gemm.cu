// Dense layer on the 5th-generation tensor cores: Y[r][off + n] = sum_k
// A[r][k] W[n][k] for the per-cell networks (the paper's SwitchNet, Table 1:
// linear layers on a per-cell feature vector), FP32 out.
//
// k_gemm_tc: persistent and warp-specialised like k_conv3_tc.  A tile is 128
// rows of A (M = 128) with all K columns: K / 16 TMA boxes of 128 rows x 16
// BF16 (32-byte rows, 32-byte swizzle) land in one stage of a ring; the
// weights W (N x K, packed in the K-major core layout [K/8][N][8]) stay in
// shared memory.  One thread issues K / 16 tcgen05.mma (128 x N x 16) into
// one of two TMEM accumulators; the epilogue warps (one per TMEM lane quarter
// and 32 output columns) load 32 columns with one tcgen05.ld and store them
// as FP32.  Bias, activation and dropout are applied by the caller's
// finishing kernels.  Every wait is bounded; a wait that gives up sets
// ST_TIMEOUT and the roles stop, wait (bounded) for work in flight and free
// TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"

namespace hyb {

static constexpr long long GEMM_MBAR_LIMIT = 1LL << 26;  // polls before a wait gives up

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int c0, int c1, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(mbar)
        : "memory");
}

template <int K, int N>
struct GemmCfg {
    static constexpr int WBYTES = K * N * 2;                        // packed weights
    static constexpr int RING = (WBYTES + 1023) / 1024 * 1024;
    static constexpr int BOX = 128 * 32;                            // one 128 x 16 BF16 box
    static constexpr int STAGE = (K / 16) * BOX;
    static constexpr int SMEM_MAX = 227 * 1024 - 512;
    static constexpr int STAGES = (SMEM_MAX - 1024 - RING) / STAGE > 4 ? 4 : (SMEM_MAX - 1024 - RING) / STAGE;
    static constexpr int SMEM = RING + STAGES * STAGE + 1024;
    static constexpr int TCOLS = 2 * N <= 32 ? 32 : (2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : 256));
    static constexpr int NEPI = 4 * (N / 32);                       // one warp per lane quarter and 32 columns
    static constexpr int NTHREADS = 64 + 32 * NEPI;
};

template <int K, int N>
__global__ void __launch_bounds__(GemmCfg<K, N>::NTHREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmap, GemmArgs a) {
    using Cfg = GemmCfg<K, N>;
    static_assert(Cfg::STAGES >= 2, "shared memory holds fewer than two stages");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *wsm = smem, *ring = smem + Cfg::RING;
    constexpr int STAGES = Cfg::STAGES;
    __shared__ __align__(8) uint64_t full_b[STAGES], empty_b[STAGES], tfull_b[2], tempty_b[2], done_b;
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
        for (int k = 0; k < 2; ++k) {
            mbar_init(smem_u32(&tfull_b[k]), 1);
            mbar_init(smem_u32(&tempty_b[k]), Cfg::NEPI);
        }
        mbar_init(smem_u32(&done_b), 1);
        abort_s = 0;
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.w);
        uint4 *dst = reinterpret_cast<uint4 *>(wsm);
        for (int i = tid; i < Cfg::WBYTES / 16; i += Cfg::NTHREADS) dst[i] = src[i];
    }
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = taddr_s;
    const long long ntiles = (a.rows + 127) / 128;
    const uint32_t ring_s = smem_u32(ring), w_s = smem_u32(wsm);

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            long long issued = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                if (!mbar_wait(smem_u32(&empty_b[s]), ph ^ 1, GEMM_MBAR_LIMIT) || *(volatile int *)&abort_s) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                    break;
                }
                const uint32_t fb = smem_u32(&full_b[s]);
                mbar_arrive_expect_tx(fb, (uint32_t)Cfg::STAGE);
                const uint32_t dst = ring_s + (uint32_t)(s * Cfg::STAGE);
#pragma unroll
                for (int c = 0; c < K / 16; ++c) tma_load_2d(dst + (uint32_t)(c * Cfg::BOX), &tmap, 16 * c, (int)(tile * 128), fb);
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
                    mbar_wait(smem_u32(&full_b[s]), ph, GEMM_MBAR_LIMIT);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, N);
            const uint64_t a0 = smem_desc_sw32(ring_s, 8 * 32);
            const uint64_t b0 = smem_desc(w_s, N * 16, 128);
            int s = 0;
            uint32_t ph = 0;
            long long it = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const int acc = (int)(it & 1);
                const uint32_t aph = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(smem_u32(&tempty_b[acc]), aph ^ 1, GEMM_MBAR_LIMIT) ||
                    !mbar_wait(smem_u32(&full_b[s]), ph, GEMM_MBAR_LIMIT) || *(volatile int *)&abort_s) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                    break;
                }
                fence_after_sync();
                const uint32_t d = taddr + (uint32_t)(acc * N);
                const uint64_t as = a0 + (uint64_t)((s * Cfg::STAGE) >> 4);
#pragma unroll
                for (int kk = 0; kk < K / 16; ++kk) {
                    const uint64_t ad = as + (uint64_t)((kk * Cfg::BOX) >> 4);
                    const uint64_t bd = b0 + (uint64_t)((2 * kk * N * 16) >> 4);
                    umma_bf16(d, ad, bd, idesc, kk != 0);
                }
                umma_commit(smem_u32(&empty_b[s]));
                umma_commit(smem_u32(&tfull_b[acc]));
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1;
                }
            }
            umma_commit(smem_u32(&done_b));
            mbar_wait(smem_u32(&done_b), 0, GEMM_MBAR_LIMIT);
        }
    } else {
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const int grp = (warp - 2) >> 2;      // columns 32 grp .. 32 grp + 31
        long long it = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int acc = (int)(it & 1);
            const uint32_t aph = (uint32_t)((it >> 1) & 1);
            const bool ok = mbar_wait(smem_u32(&tfull_b[acc]), aph, GEMM_MBAR_LIMIT);
            if (!__all_sync(0xffffffffu, ok) || *(volatile int *)&abort_s) {
                if (lane == 0) {
                    atomicOr(a.status, ST_TIMEOUT);
                    *(volatile int *)&abort_s = 1;
                }
                break;
            }
            fence_after_sync();
            float v[32];
            tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * N + grp * 32), v);
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty_b[acc]));
            const long long r = tile * 128 + q * 32 + lane;
            if (r < a.rows) {
                float4 *o4 = reinterpret_cast<float4 *>(a.y + r * a.pitch + a.off + grp * 32);
#pragma unroll
                for (int j = 0; j < 8; ++j) o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(taddr, Cfg::TCOLS);
}

typedef CUresult (*EncodeTiledFn2)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn2 encode_fn2() {
    static EncodeTiledFn2 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn2)p;
    });
    return fn;
}

template <int K, int N>
static hyb_status gemm_cfg(const GemmArgs &a, cudaStream_t st) {
    using Cfg = GemmCfg<K, N>;
    EncodeTiledFn2 enc = encode_fn2();
    if (!enc) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled is not available");
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)a.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {16, 128};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)a.x, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(HYB_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    static std::mutex mu;
    static int ready_dev[64] = {0}, nsm_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return set_error(HYB_EINVAL, "device index out of range");
    int nsm;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready_dev[dev]) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
            if (e != cudaSuccess)
                return set_error(HYB_ECUDA, std::string("gemm smem attribute: ") + cudaGetErrorString(e));
            cudaDeviceGetAttribute(&nsm_dev[dev], cudaDevAttrMultiProcessorCount, dev);
            ready_dev[dev] = 1;
        }
        nsm = nsm_dev[dev];
    }
    const long long ntiles = (a.rows + 127) / 128;
    const long long grid = std::min<long long>(ntiles, (long long)nsm);
    k_gemm_tc<K, N><<<(unsigned)grid, Cfg::NTHREADS, Cfg::SMEM, st>>>(tm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("gemm launch: ") + cudaGetErrorString(e));
    return HYB_OK;
}

hyb_status launch_gemm_tc(const GemmArgs &a, cudaStream_t st) {
    if (a.rows < 1 || !a.x || !a.w || !a.y) return set_error(HYB_EINVAL, "gemm: empty or null operand");
    if (a.rows >= (1LL << 31) - 128) return set_error(HYB_EINVAL, "gemm: more than 2^31 rows");
    if (((uintptr_t)a.x & 15) || ((uintptr_t)a.w & 15) || ((uintptr_t)a.y & 15) || a.pitch % 4 || a.off % 32 ||
        a.off + a.N > a.pitch)
        return set_error(HYB_EINVAL, "gemm operands misaligned or output slice out of range");
    if (a.K == 16 && a.N == 128) return gemm_cfg<16, 128>(a, st);
    if (a.K == 128 && a.N == 128) return gemm_cfg<128, 128>(a, st);
    if (a.K == 256 && a.N == 128) return gemm_cfg<256, 128>(a, st);
    return set_error(HYB_EINVAL, "gemm shape: (K, N) in {(16, 128), (128, 128), (256, 128)}");
}

}  // namespace hyb
