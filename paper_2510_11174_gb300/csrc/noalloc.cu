// hyb_field_energy_noalloc: the FP64 field-energy reduction of hyb_diagnostics
// as a stand-alone entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that must not synchronise the
// device in the middle of its loop (cudaMalloc and cudaFree may do so), code
// whose device memory is entirely owned by another allocator (a caching
// allocator that has already reserved the free memory), and code with a fixed
// memory budget decided at start-up.  For them the block partial sums live in
// a file-scope device array of fixed size instead of a caller- or
// library-allocated buffer.  Every GPU that loads the library holds that array
// until the process exits.
#include <mutex>

#include "hyb_internal.cuh"

namespace hyb {

static constexpr int NA_THREADS = 256;
static constexpr long long NA_CHUNK = 16384;  // array elements reduced by one block
static constexpr int NA_MAX_BLOCKS = 4096;    // partial sums the static array holds per quantity

// two quantities (E, B) x NA_MAX_BLOCKS partial sums: 64 KiB
static __device__ __align__(256) double g_energy_scratch[2 * NA_MAX_BLOCKS];

static_assert(HYB_NOALLOC_MAX_CELLS * 3LL <= NA_CHUNK * NA_MAX_BLOCKS, "maximum size exceeds the static scratch");

__device__ __forceinline__ double na_block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// block b sums E^2 and B^2 over elements [b*NA_CHUNK, (b+1)*NA_CHUNK) of the
// 3*N-element component-major arrays and overwrites partial slot b
__global__ void __launch_bounds__(NA_THREADS) k_na_partials(const float *__restrict__ E, const float *__restrict__ B,
                                                            long long n3, double *__restrict__ scratch) {
    __shared__ double sh[NA_THREADS];
    const long long lo = (long long)blockIdx.x * NA_CHUNK;
    const long long hi = min(lo + NA_CHUNK, n3);
    double se = 0.0, sb = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NA_THREADS) {
        const double e = E[i], b = B[i];
        se += e * e;
        sb += b * b;
    }
    se = na_block_sum(se, sh);
    sb = na_block_sum(sb, sh);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = se;
        scratch[NA_MAX_BLOCKS + blockIdx.x] = sb;
    }
}

__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double *__restrict__ scratch, int nblocks,
                                                         double dvol_half, double *__restrict__ out) {
    __shared__ double sh[NA_THREADS];
    for (int q = 0; q < 2; ++q) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) acc += scratch[q * NA_MAX_BLOCKS + b];
        acc = na_block_sum(acc, sh);
        if (threadIdx.x == 0) out[q] = acc * dvol_half;
    }
}

// Device address of the static array, looked up once per device with that
// device current (in host code the array's name is only a host-side handle).
static std::mutex g_na_mutex;
static double *g_na_addr[64] = {};

static hyb_status na_scratch(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return set_error(HYB_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess)
            return set_error(HYB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_addr[dev] = (double *)p;
    }
    *out = g_na_addr[dev];
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" hyb_status hyb_field_energy_noalloc(const float *E_dev, const float *B_dev, long long n_cells, double dx,
                                               double dy, double dz, double *out_dev, void *stream) {
    if (!E_dev || !B_dev || !out_dev) return set_error(HYB_EINVAL, "null pointer");
    if (n_cells < 1) return set_error(HYB_EINVAL, "n_cells must be >= 1");
    if (n_cells > HYB_NOALLOC_MAX_CELLS)
        return set_error(HYB_EINVAL, "n_cells exceeds HYB_NOALLOC_MAX_CELLS (the fixed scratch of this entry point)");
    if (!(dx > 0.0 && dy > 0.0 && dz > 0.0)) return set_error(HYB_EINVAL, "cell size must be positive");
    double *scratch = nullptr;
    hyb_status s = na_scratch(&scratch);
    if (s != HYB_OK) return s;
    const long long n3 = 3 * n_cells;
    const int nblocks = (int)((n3 + NA_CHUNK - 1) / NA_CHUNK);
    cudaStream_t st = (cudaStream_t)stream;
    k_na_partials<<<nblocks, NA_THREADS, 0, st>>>(E_dev, B_dev, n3, scratch);
    k_na_final<<<1, NA_THREADS, 0, st>>>(scratch, nblocks, 0.5 * dx * dy * dz, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HYB_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return HYB_OK;
}
