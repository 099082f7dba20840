// Mass/momentum reduction that allocates nothing (declared in include/lbm.h
// as lbm_reduce_noalloc).
//
// Some callers cannot allocate device memory: code running while a memory
// pool is frozen or capped (an inference server that reserved all of HBM up
// front, a custom allocator that forbids cudaMalloc after start-up), or a
// host process that only borrows device pointers from another framework and
// must not create allocations of its own. They pass the populations, the
// mask and a 4-double output; the per-block partial sums live in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"

namespace {

// Lattice shape and velocity components, i = (cx+1) + 3(cy+1) [+ 9(cz+1)].
template <int LAT> struct Lat;
template <> struct Lat<0> { static constexpr int D = 2, Q = 9; };
template <> struct Lat<1> { static constexpr int D = 3, Q = 27; };
__device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__device__ constexpr int cz_of(int i) { return i / 9 - 1; }

__device__ __forceinline__ double warp_total(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kThreads = 256;
constexpr int kNodesPerBlock = 8192;                 // 32 nodes per thread
constexpr int kMaxBlocks = LBM_REDUCE_NOALLOC_MAX_NODES / kNodesPerBlock;
constexpr int kFinalThreads = 1024;
static_assert(LBM_REDUCE_NOALLOC_MAX_NODES % kNodesPerBlock == 0, "whole blocks");

// Partial sums (mass, jx, jy, jz) of each block: 8192 x 4 doubles = 256 KiB.
// Every call writes exactly the slots it then reads, so nothing is cleared.
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_partials_dev[kMaxDevices] = {nullptr};

// Device address of the partials on the current device, looked up once per
// device (host code may not use the array's name as a device pointer).
cudaError_t partials_on_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_dev[dev] = static_cast<double *>(p);
    }
    *out = g_partials_dev[dev];
    return cudaSuccess;
}

template <int LAT>
__global__ void __launch_bounds__(kThreads)
k_noalloc_partial(unsigned N, const uint8_t *__restrict__ mask, const double *__restrict__ f,
                  double *__restrict__ partial)
{
    constexpr int D = Lat<LAT>::D, Q = Lat<LAT>::Q;
    const unsigned lo = blockIdx.x * kNodesPerBlock;
    const unsigned hi = min(N, lo + kNodesPerBlock);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned n = lo + threadIdx.x; n < hi; n += kThreads) {
        if (mask && mask[n]) continue;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double fi = f[(size_t)i * N + n];
            acc[0] += fi;
            if (cx_of(i)) acc[1] += cx_of(i) * fi;
            if (cy_of(i)) acc[2] += cy_of(i) * fi;
            if (D == 3 && cz_of(i)) acc[3] += cz_of(i) * fi;
        }
    }
    __shared__ double sh[4][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_total(acc[k]);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double v = lane < kThreads / 32 ? sh[k][lane] : 0.0;
            v = warp_total(v);
            if (lane == 0) partial[4 * blockIdx.x + k] = v;
        }
    }
}

__global__ void __launch_bounds__(kFinalThreads)
k_noalloc_final(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kFinalThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += partial[4 * b + k];
    __shared__ double sh[4][kFinalThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_total(acc[k]);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double v = warp_total(sh[k][lane]);
            if (lane == 0) out[k] = v;
        }
    }
}

}  // namespace

extern "C" int lbm_reduce_noalloc(int lattice, int nx, int ny, int nz, const double *f_dev,
                                  const uint8_t *mask_dev, double *sums_dev, void *stream)
{
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return LBM_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == LBM_D2Q9 && nz != 1)) return LBM_EINVAL;
    if (!f_dev || !sums_dev) return LBM_EINVAL;
    const double N = (double)nx * ny * nz;
    if (N > (double)LBM_REDUCE_NOALLOC_MAX_NODES) return LBM_ETOOBIG;
    double *partial = nullptr;
    if (partials_on_current_device(&partial) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    const unsigned n = (unsigned)N;
    const int nblocks = (int)((n + kNodesPerBlock - 1) / kNodesPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (lattice == LBM_D2Q9)
        k_noalloc_partial<0><<<nblocks, kThreads, 0, s>>>(n, mask_dev, f_dev, partial);
    else
        k_noalloc_partial<1><<<nblocks, kThreads, 0, s>>>(n, mask_dev, f_dev, partial);
    k_noalloc_final<<<1, kFinalThreads, 0, s>>>(partial, nblocks, sums_dev);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}
