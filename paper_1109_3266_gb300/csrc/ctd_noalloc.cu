// ctd_noalloc.cu -- an allocation-free variant of the avg-RSD reduction.
//
// Some callers cannot allocate device memory at the moment they need the
// precision measure, such as hosts that hand all device memory to their own
// pool allocator and forbid libraries from calling cudaMalloc.  For them,
// ctd_avg_rsd_noalloc reduces dose and stddev arrays that already live on the
// device, using per-block partial sums kept in a fixed file-scope device array
// instead of library-allocated scratch.
//
// The array (g_rsd_scratch, 5 * kMaxBlocks + 8 doubles = 160 KB) is part of the
// library image: every GPU that loads the library holds it until the process
// exits.  All calls share it; each call overwrites every partial it reads, so
// nothing is carried over from the previous call, but calls that overlap on
// the GPU (on different streams, or from different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "ctd_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr size_t kVoxPerThread = 64;
constexpr size_t kVoxPerBlock = kThreads * kVoxPerThread;    // 16384 voxels per block
constexpr int kMaxBlocks = 4096;
constexpr size_t kMaxVoxels = kVoxPerBlock * kMaxBlocks;     // 67,108,864 voxels
constexpr int kScratchDoubles = 5 * kMaxBlocks + 8;          // partials: 1 max + 4 sums per block, + 8 cells
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_rsd_scratch[kScratchDoubles];

// layout inside the scratch array
constexpr int kOffMax = 0;                   // [kMaxBlocks] per-block maxima
constexpr int kOffSums = kMaxBlocks;         // [4][kMaxBlocks] per-block sums
constexpr int kOffCells = 5 * kMaxBlocks;    // [0] = d_max

// maximum dose over voxels with rho >= 0.1 in this block's tile
__global__ void na_dmax_kernel(const double *__restrict__ dose, const float *__restrict__ rho, size_t nvox,
                               double *scratch)
{
    const size_t begin = blockIdx.x * kVoxPerBlock;
    const size_t end = begin + kVoxPerBlock < nvox ? begin + kVoxPerBlock : nvox;
    double m = 0.0;
    for (size_t v = begin + threadIdx.x; v < end; v += kThreads)
        if (rho[v] >= 0.1f && dose[v] > m) m = dose[v];
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) b = fmax(b, sh[w]);
        scratch[kOffMax + blockIdx.x] = b;
    }
}

__global__ void na_dmax_final_kernel(int nblocks, double *scratch)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < nblocks; ++i) b = fmax(b, scratch[kOffMax + i]);
        scratch[kOffCells] = b;
    }
}

// sums of s/D over D > 0.1 D_max and of s over D > 0.2 D_max, with their counts
__global__ void na_rsd_kernel(const double *__restrict__ dose, const double *__restrict__ sd,
                              const float *__restrict__ rho, size_t nvox, double *scratch)
{
    const double dmax = scratch[kOffCells];
    const size_t begin = blockIdx.x * kVoxPerBlock;
    const size_t end = begin + kVoxPerBlock < nvox ? begin + kVoxPerBlock : nvox;
    double x[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t v = begin + threadIdx.x; v < end; v += kThreads) {
        if (!(rho[v] >= 0.1f)) continue;
        const double D = dose[v];
        if (D > 0.1 * dmax) {
            x[0] += sd[v] / D;
            x[1] += 1.0;
        }
        if (D > 0.2 * dmax) {
            x[2] += sd[v];
            x[3] += 1.0;
        }
    }
    __shared__ double sh[4][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_down_sync(0xffffffffu, x[k], o);
        if (lane == 0) sh[k][warp] = x[k];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += sh[k][w];
            scratch[kOffSums + k * kMaxBlocks + blockIdx.x] = s;
        }
}

__global__ void na_final_kernel(int nblocks, const double *scratch, double *result)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < nblocks; ++i) s[k] += scratch[kOffSums + k * kMaxBlocks + i];
        const double dmax = scratch[kOffCells];
        result[0] = s[1] > 0.0 ? s[0] / s[1] : 0.0;
        result[1] = (s[3] > 0.0 && dmax > 0.0) ? s[2] / (s[3] * dmax) : 0.0;
        result[2] = dmax;
    }
}

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices];   // device address of g_rsd_scratch, per device

int na_fail(int code, const char *msg)
{
    ctd::set_error(msg);
    return code;
}

}  // namespace

extern "C" {

int ctd_avg_rsd_noalloc(const double *dose_dev, const double *stddev_dev, const float *density_dev, size_t nvox,
                        double *result_dev, void *stream)
{
    ctd::set_error("");
    if (!dose_dev || !stddev_dev || !density_dev || !result_dev) return na_fail(CTD_EINVAL, "null device pointer");
    if (nvox == 0) return na_fail(CTD_EINVAL, "nvox must be positive");
    if (nvox > kMaxVoxels)
        return na_fail(CTD_EINVAL, "nvox exceeds the 67,108,864 voxels the fixed scratch array covers");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return na_fail(CTD_ECUDA, "no usable current CUDA device");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The scratch array's device address, looked up with the device current.  Outside
    // stream capture it is looked up on every call (a device reset reloads the module
    // and moves the array); during capture the address of this device's last lookup
    // is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;   // unknown: take the cached address
    }
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_rsd_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return na_fail(CTD_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    const int nblocks = static_cast<int>((nvox + kVoxPerBlock - 1) / kVoxPerBlock);
    na_dmax_kernel<<<nblocks, kThreads, 0, s>>>(dose_dev, density_dev, nvox, scratch);
    na_dmax_final_kernel<<<1, 32, 0, s>>>(nblocks, scratch);
    na_rsd_kernel<<<nblocks, kThreads, 0, s>>>(dose_dev, stddev_dev, density_dev, nvox, scratch);
    na_final_kernel<<<1, 32, 0, s>>>(nblocks, scratch, result_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(CTD_ECUDA, cudaGetErrorString(e));
    return CTD_OK;
}

}  // extern "C"
