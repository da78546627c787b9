// 3x3x3 convolutions of the regime classifier (arXiv 2510.11174, Methodology
// and Results: a convolutional network on per-channel normalised fields, with
// Monte Carlo dropout for uncertainty; here the 3D CNN 6->32->32->16->1 with
// BF16 weights and FP32 accumulation).
//
// k_conv3_tc: implicit GEMM on the 5th-generation tensor cores.  A CTA owns
// an output tile of 128 cells = 8 (x) x 16 (y) x 1 (z).  It stages the input
// halo (10 x 18 x 3 cells, channels in 8-wide chunks) and all 27 x C_in x
// C_out weights in shared memory, and one thread issues, for each of the 27
// taps and each 16-channel slice of the input, one tcgen05.mma of shape
// M = 128 (cells) x N = C_out x K = 16 that accumulates into TMEM.  The
// operand of tap (dz, dy, dx) is the halo shifted by that tap: with the
// chunk-major halo layout [chunk][z][y][x][8 channels], the 8 cells of one
// output row are 8 consecutive 16-byte rows (one core matrix) and the 16
// rows of the tile are 160 bytes apart, so every tap is a plain matrix
// descriptor (start shifted by the tap; leading byte offset = one chunk block,
// stride byte offset = 160 B) -- no im2col copy.  The epilogue reads the
// accumulator from TMEM (tcgen05.ld), adds the bias, applies ReLU and the
// Philox dropout mask (inverted scaling 1/(1-p)), converts to BF16 and stores
// channels-last.  Each CTA loops over tiles (persistent grid).
#include <cuda_bf16.h>

#include "conv_tc.cuh"
#include "hyb_internal.cuh"
#include "philox.cuh"

namespace hyb {

static constexpr int TX = 8, TY = 16;                 // output tile (cells)
static constexpr int HX = TX + 2, HY = TY + 2, HZ = 3; // halo
static constexpr int HCELLS = HX * HY * HZ;            // 540
static constexpr int CHB = HCELLS * 16;                // bytes of one 8-channel chunk block
static constexpr long long MBAR_LIMIT = 1LL << 26;     // polls before a wait gives up

// dropout keep decision of channel ch at cell (b, lin): Philox counter
// (lin, b, (layer << 16) | (ch >> 2), pass), key (seed, 0xD0); word ch & 3
__host__ __device__ inline bool dropout_keep(uint32_t seed, uint32_t pass, uint32_t layer, uint32_t b, uint32_t lin,
                                             int ch, float p) {
    const u32x4 r = philox4x32_10(lin, b, (layer << 16) | ((uint32_t)ch >> 2), pass, seed, 0xD0u);
    return !(u01f(r.v[ch & 3]) < p);
}

size_t conv_smem_bytes(int cin, int N) {
    const size_t halo = (size_t)(cin / 8) * CHB;
    const size_t w = (size_t)27 * (cin / 8) * N * 16;
    // the operand descriptors of every tap stay inside this allocation for
    // either reading of the leading/stride offsets (halo first)
    const size_t need = halo + w;
    const size_t worst = (size_t)(cin / 8 - 2) * CHB + (2 * HY + 2) * HX * 16 + 32 + 15 * (size_t)CHB + 288;
    return need > worst ? need : worst;
}

__global__ void __launch_bounds__(128) k_conv3_tc(ConvArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t taddr_s;
    const int KC = a.cin / 8;
    uint8_t *halo = smem;
    uint8_t *wsm = smem + (size_t)KC * CHB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tmem_alloc(smem_u32(&taddr_s), 32);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar), 1);
        fence_proxy_async_smem();
    }
    // weights: straight 16-byte copies (already in core layout)
    {
        const int nv = 27 * KC * a.N;
        const uint4 *src = reinterpret_cast<const uint4 *>(a.wt);
        uint4 *dst = reinterpret_cast<uint4 *>(wsm);
        for (int i = tid; i < nv; i += blockDim.x) dst[i] = src[i];
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = taddr_s;
    const uint32_t halo_s = smem_u32(halo), w_s = smem_u32(wsm);
    const uint32_t idesc = idesc_bf16(128, a.N);
    const int tiles_x = a.W / TX, tiles_y = a.H / TY;
    const long long ntiles = (long long)a.B * a.D * tiles_y * tiles_x;
    uint32_t phase = 0;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = (int)(tile % tiles_x);
        const int ty = (int)((tile / tiles_x) % tiles_y);
        const int z0 = (int)((tile / ((long long)tiles_x * tiles_y)) % a.D);
        const int b = (int)(tile / ((long long)tiles_x * tiles_y * a.D));
        const int x0 = tx * TX, y0 = ty * TY;
        // ---- halo [chunk][lz][ly][lx][8], zero outside the volume
        for (int i = tid; i < KC * HCELLS; i += blockDim.x) {
            const int ch = i / HCELLS, cell = i % HCELLS;
            const int lz = cell / (HY * HX), ly = (cell / HX) % HY, lx = cell % HX;
            const int gz = z0 - 1 + lz, gy = y0 - 1 + ly, gx = x0 - 1 + lx;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gz >= 0 && gz < a.D && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) {
                const long long off = ((((long long)b * a.D + gz) * a.H + gy) * a.W + gx) * a.cin + ch * 8;
                v = *reinterpret_cast<const uint4 *>(a.x + off);
            }
            reinterpret_cast<uint4 *>(halo)[i] = v;
        }
        fence_proxy_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                for (int kk = 0; kk < KC / 2; ++kk) {
                    const uint32_t aa = halo_s + (uint32_t)(2 * kk) * CHB + (uint32_t)(((dz * HY + dy) * HX + dx) * 16);
                    const uint32_t bb = w_s + (uint32_t)((tap * KC + 2 * kk) * a.N) * 16;
                    umma_bf16(taddr, smem_desc(aa, CHB, HX * 16), smem_desc(bb, a.N * 16, 128), idesc,
                              (tap | kk) != 0);
                }
            }
            umma_commit(smem_u32(&mbar));
        }
        const bool ok = mbar_wait(smem_u32(&mbar), phase, MBAR_LIMIT);
        phase ^= 1;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
            break;
        }
        fence_after_sync();
        // ---- epilogue: row m = 32 warp + lane -> cell (x0 + m % 8, y0 + m / 8, z0)
        const int m = warp * 32 + lane;
        const int cx = x0 + (m & 7), cy = y0 + (m >> 3);
        const uint32_t lin = (uint32_t)(((long long)z0 * a.H + cy) * a.W + cx);
        __nv_bfloat16 *out = a.y + ((((long long)b * a.D + z0) * a.H + cy) * a.W + cx) * a.N;
        for (int h = 0; h < a.N / 16; ++h) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 16), v);
            __align__(16) __nv_bfloat16 o[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int ch = h * 16 + j;
                float s = v[j] + (a.bias ? a.bias[ch] : 0.0f);
                if (a.relu) s = fmaxf(s, 0.0f);
                if (a.drop_p > 0.0f)
                    s = dropout_keep(a.seed, a.pass, a.layer, (uint32_t)b, lin, ch, a.drop_p) ? s / (1.0f - a.drop_p)
                                                                                              : 0.0f;
                o[j] = __float2bfloat16_rn(s);
            }
            reinterpret_cast<uint4 *>(out + h * 16)[0] = reinterpret_cast<const uint4 *>(o)[0];
            reinterpret_cast<uint4 *>(out + h * 16)[1] = reinterpret_cast<const uint4 *>(o)[1];
        }
        fence_before_sync();
        __syncthreads();
    }
    fence_after_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 32);
}

hyb_status launch_conv3_tc(const ConvArgs &a, cudaStream_t st) {
    if (a.cin % 16 != 0 || (a.N != 16 && a.N != 32) || a.W % TX != 0 || a.H % TY != 0)
        return set_error(HYB_EINVAL, "conv shape: cin % 16, N in {16, 32}, W % 8, H % 16 required");
    const size_t smem = conv_smem_bytes(a.cin, a.N);
    cudaError_t e = cudaFuncSetAttribute(k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("conv smem attribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3_tc, 128, smem);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (long long)a.B * a.D * (a.H / TY) * (a.W / TX);
    const long long grid = std::min<long long>(ntiles, (long long)nsm * std::max(per_sm, 1));
    k_conv3_tc<<<(unsigned)grid, 128, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("conv launch: ") + cudaGetErrorString(e));
    return HYB_OK;
}

}  // namespace hyb
