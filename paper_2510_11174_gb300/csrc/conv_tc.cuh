// tcgen05 building blocks for the 3x3x3 convolution of the regime classifier
// (inline PTX; sm_100-family tensor cores with TMEM accumulators).
//
// Operand layout used throughout (K-major, no swizzle): a "core matrix" is 8
// rows of 16 bytes (8 BF16 values along K) stored contiguously (128 B).  A
// shared-memory matrix descriptor gives the start address, the byte offset
// between core matrices adjacent along K (leading byte offset) and along M/N
// (stride byte offset).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace hyb {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (tcgen05): start>>4 in bits [0,14), leading
// byte offset>>4 in [16,30), stride byte offset>>4 in [32,46), version 1 in
// [46,48), base offset 0, no swizzle (layout type 0 in [61,64))
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// K-major operand with the 32-byte swizzle (layout type 6 in [61,64)): rows
// of 32 bytes (16 BF16 along K), 8-row groups `sbo` bytes apart; the swizzle
// is taken from the absolute shared address (base offset 0), so the start may
// be any 32-byte row, not only a swizzle-pattern boundary
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t addr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;  // leading byte offset: unused when K fits the swizzle width
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

// instruction descriptor for kind::f16: FP32 accumulator (bits [4,6) = 1),
// BF16 A and B (bits [7,10) = 1, [10,13) = 1), both K-major, N>>3 in
// [17,23), M>>4 in [24,29)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols));
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar_smem) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_smem)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// wait for the phase `parity` of an mbarrier; gives up after `limit` polls
// and returns false (the caller records a timeout and stops issuing work)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// plain arrival (count 1) on an mbarrier
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// arrival that also announces `bytes` of asynchronous (TMA) transactions
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// tiled TMA load of a 5-D box into shared memory, completion counted on mbar
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void *tmap, int c0, int c1, int c2, int c3, int c4,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void *tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// 32 lanes x 32 bits, 8 consecutive columns
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// three loads of 32 lanes x 32 bits x 8 consecutive columns (at t0, t1, t2)
// under one wait: v[8 k + i] = column i of load k
__device__ __forceinline__ void tmem_ld8x3(uint32_t t0, uint32_t t1, uint32_t t2, float v[24]) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(t0), "r"(t1), "r"(t2)
        : "memory");
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 bits, 32 consecutive columns under one wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 bits, 16 consecutive columns: thread i of the warp gets lane (32w + i)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace hyb

#include "../../include/hyb.h"

namespace hyb {

// one 3x3x3 convolution layer on the tensor cores (see conv.cu)
struct ConvArgs {
    const __nv_bfloat16 *x;   // [B][D][H][W][cin] channels-last
    const __nv_bfloat16 *wt;  // [27][cin/8][N][8] core layout
    const float *bias;        // [N] or null
    __nv_bfloat16 *y;         // [B][D][H][W][N]
    float *y_f32;             // when set: FP32 output [B][D][H][W][N] instead of y
    int B, D, H, W, cin, N;   // cin: the channels one launch contracts (16 or 32)
    int cin_total;            // channel pitch of x (0: cin); a launch reads channels cin_off .. cin_off + cin - 1
    int cin_off;
    int out_pitch;            // channel pitch of y / y_f32 (0: N); a launch writes channels out_off .. out_off + N - 1
    int out_off;
    int accum;                // y_f32 += the raw sums (no bias, ReLU or dropout): the partial of one input chunk
    int relu;
    uint32_t drop_thr;        // dropout threshold round(p 2^16) on 16-bit Philox fields; 0: no dropout
    float drop_scale;         // 1 / (1 - drop_thr 2^-16)
    int scale_out;            // kept outputs are multiplied by drop_scale (set with dropout; alone: scaling only)
    uint32_t seed, pass, layer;
    int *status;
    int x_lo, x_hi;           // when x_hi > x_lo: only the tiles whose outputs meet x_lo <= x < x_hi
};
hyb_status launch_conv3_tc(const ConvArgs &a, cudaStream_t st);

// one dense layer on the tensor cores (see gemm.cu): y[r][off + n] = sum_k
// x[r][k] w[n][k] for r < rows, n < N, FP32 out
struct GemmArgs {
    const __nv_bfloat16 *x;   // [rows][K] BF16
    const __nv_bfloat16 *w;   // packed K-major core layout [K/8][N][8]
    float *y;                 // [rows][pitch] FP32
    long long rows;
    int K, N, pitch, off;
    int *status;
};
hyb_status launch_gemm_tc(const GemmArgs &a, cudaStream_t st);

// the last layer (16 -> 1 channel, 3x3x3) on the tensor cores (see conv.cu);
// mc_k = 0 writes the logit, mc_k = k >= 1 folds sigmoid(logit) into the
// running mean / M2 of the MC passes (k = 1 starts them)
struct LastArgs {
    const __nv_bfloat16 *x;   // [B][D][H][W][16] channels-last
    uint32_t w[256];          // BF16 weights as B operand: [ci / 8][tap (27, padded to 32)][ci % 8]
    float bias;
    int B, D, H, W;
    float *logit;             // [B][D][H][W] (mc_k = 0)
    int mc_k;
    float *pm, *m2;           // MC mean and M2 (mc_k >= 1)
    int *status;
    int x_lo, x_hi;           // when x_hi > x_lo: only the blocks whose outputs meet x_lo <= x < x_hi
};
hyb_status launch_conv_last_tc(const LastArgs &a, cudaStream_t st);

}  // namespace hyb
