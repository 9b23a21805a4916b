// ctd_stats.cu -- batch statistics of the dose engine (Sec. 2.2.1) and the
// precision measures of Sec. 3.1, as streaming kernels over the FP64 grids.
#include <cuda_runtime.h>

#include "ctd_internal.h"

namespace ctd {
namespace {

constexpr int kThreads = 256;

// Fold one batch: d = E_b / (m_v n_b) in Gy per history; accumulate d and d^2,
// keep the raw energy, clear the batch tally.  scale = keV->J * 1000 / (V n_b).
__global__ void fold_kernel(double *__restrict__ tally, const float *__restrict__ rho, double *__restrict__ sum_d,
                            double *__restrict__ sum_d2, double *__restrict__ edep, size_t nvox, double scale)
{
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const double t = tally[v];
        if (t == 0.0) continue;
        const float r = rho[v];
        edep[v] += t;
        tally[v] = 0.0;
        if (r > 0.0f) {
            const double d = t * scale / static_cast<double>(r);
            sum_d[v] += d;
            sum_d2[v] += d * d;
        }
    }
}

// The same fold for several requests at once, one tile of kFoldTile voxels per step.
__global__ void fold_multi_kernel(const FoldDesc *__restrict__ descs, const uint64_t *__restrict__ tile_off, int n,
                                  uint64_t total_tiles)
{
    for (uint64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= tile) lo = mid;
            else hi = mid - 1;
        }
        const FoldDesc d = descs[lo];
        const uint64_t base = (tile - tile_off[lo]) * static_cast<uint64_t>(kFoldTile);
        const uint64_t end = base + kFoldTile < d.nvox ? base + kFoldTile : d.nvox;
        for (uint64_t v = base + threadIdx.x; v < end; v += blockDim.x) {
            const double t = d.tally[v];
            if (t == 0.0) continue;
            const float r = d.rho[v];
            d.edep[v] += t;
            d.tally[v] = 0.0;
            if (r > 0.0f) {
                const double x = t * d.scale / static_cast<double>(r);
                d.sum_d[v] += x;
                d.sum_d2[v] += x * x;
            }
        }
    }
}

// Mean over nb batches and its standard error: s^2 = (sum d^2 - nb D^2) / (nb (nb - 1)).
__device__ __forceinline__ void mean_sd(double s1, double s2, int nb, double &D, double &sd)
{
    D = s1 / nb;
    double var = (s2 - nb * D * D) / (static_cast<double>(nb) * (nb - 1));
    sd = var > 0.0 ? sqrt(var) : 0.0;
}

__global__ void finalize_kernel(const double *__restrict__ sum_d, const double *__restrict__ sum_d2, int nb,
                                double *__restrict__ dose, double *__restrict__ sd, size_t nvox)
{
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
        double D, s;
        mean_sd(sum_d[v], sum_d2[v], nb, D, s);
        dose[v] = D;
        sd[v] = s;
    }
}

// Block-wide sums of K doubles; partials[k * n_parts + block].
template <int K>
__device__ __forceinline__ void block_sums(double (&x)[K], double *partials, int n_parts)
{
    __shared__ double sh[K][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_down_sync(0xffffffffu, x[k], o);
        if (lane == 0) sh[k][warp] = x[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += sh[k][w];
            partials[k * n_parts + blockIdx.x] = s;
        }
    }
}

// pass 1: maximum dose over voxels with rho >= 0.1 (per block)
__global__ void dmax_kernel(const double *__restrict__ dose, const float *__restrict__ rho, size_t nvox,
                            double *partials)
{
    double m = 0.0;
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x)
        if (rho[v] >= 0.1f && dose[v] > m) m = dose[v];
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) b = fmax(b, sh[w]);
        partials[blockIdx.x] = b;
    }
}

__global__ void max_final_kernel(const double *partials, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < n; ++i) b = fmax(b, partials[i]);
        *out = b;
    }
}

// pass 2: sums for avg RSD (s/D over D > 0.1 D_max) and the paper's sigma_bar
// (s/D_max over D > 0.2 D_max), both inside rho >= 0.1
__global__ void rsd_kernel(const double *__restrict__ dose, const double *__restrict__ sd,
                           const float *__restrict__ rho, size_t nvox, const double *dmax_p, double *partials,
                           int n_parts)
{
    const double dmax = *dmax_p;
    double x[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
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
    block_sums<4>(x, partials, n_parts);
}

__global__ void rsd_final_kernel(const double *partials, int n_parts, const double *dmax_p, double *result)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < n_parts; ++i) s[k] += partials[k * n_parts + i];
        const double dmax = *dmax_p;
        result[0] = s[1] > 0.0 ? s[0] / s[1] : 0.0;
        result[1] = (s[3] > 0.0 && dmax > 0.0) ? s[2] / (s[3] * dmax) : 0.0;
        result[2] = dmax;
    }
}

__global__ void sum_kernel(const double *__restrict__ x, size_t n, double *partials, int n_parts)
{
    double a[1] = {0.0};
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<size_t>(gridDim.x) * blockDim.x)
        a[0] += x[v];
    block_sums<1>(a, partials, n_parts);
}

__global__ void sum_final_kernel(const double *partials, int n_parts, double *result)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n_parts; ++i) s += partials[i];
        *result = s;
    }
}

// One pass over a new phantom's voxels (grid-stride): range checks and the
// per-material presence and largest density, reduced in shared memory, then one
// global atomic per block and quantity.  -0 densities count as +0.
__global__ void scan_phantom_kernel(const uint8_t *__restrict__ mat, const float *__restrict__ rho, size_t nvox,
                                    int n_mat, uint32_t *__restrict__ vox, PhantomScan *out)
{
    __shared__ unsigned int s_max[kMaxPhantomMaterials];
    __shared__ unsigned int s_mask;
    __shared__ unsigned long long s_bad_mat, s_bad_rho;
    if (threadIdx.x < kMaxPhantomMaterials) s_max[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        s_mask = 0u;
        s_bad_mat = ~0ull;
        s_bad_rho = ~0ull;
    }
    __syncthreads();
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int m = mat[v];
        const float r = rho[v];
        if (m >= n_mat) {
            atomicMin(&s_bad_mat, static_cast<unsigned long long>(v));
            continue;
        }
        const uint32_t f = __float_as_uint(r + 0.0f);   // -0 as +0
        const uint32_t ex = f >> 23;
        if (!(r >= 0.0f) || (f != 0u && (ex < kRhoExpLo || ex > kRhoExpHi))) {
            atomicMin(&s_bad_rho, static_cast<unsigned long long>(v));
            continue;
        }
        vox[v] = (static_cast<uint32_t>(m) << 28) | (f ? f - (kRhoExpBias << 23) : 0u);
        atomicMax(&s_max[m], f);
        atomicOr(&s_mask, 1u << m);
    }
    __syncthreads();
    if (threadIdx.x < n_mat && (s_mask >> threadIdx.x & 1u)) atomicMax(&out->max_bits[threadIdx.x], s_max[threadIdx.x]);
    if (threadIdx.x == 0) {
        if (s_mask) atomicOr(&out->present_mask, s_mask);
        if (s_bad_mat != ~0ull) atomicMin(&out->first_bad_mat, s_bad_mat);
        if (s_bad_rho != ~0ull) atomicMin(&out->first_bad_rho, s_bad_rho);
    }
}

int grid_for(size_t n)
{
    size_t g = (n + kThreads - 1) / kThreads;
    if (g > 152 * 16) g = 152 * 16;
    if (g == 0) g = 1;
    return static_cast<int>(g);
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA; }

}  // namespace

int launch_fold(double *tally, const float *rho, double *sum_d, double *sum_d2, double *edep, size_t nvox,
                double scale, void *stream)
{
    fold_kernel<<<grid_for(nvox), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(tally, rho, sum_d, sum_d2,
                                                                                      edep, nvox, scale);
    return ok();
}

int launch_fold_multi(const FoldDesc *descs, const uint64_t *tile_off, int n, uint64_t total_tiles, void *stream)
{
    if (total_tiles == 0) return CTD_OK;
    const int grid = total_tiles < 152 * 16 ? static_cast<int>(total_tiles) : 152 * 16;
    fold_multi_kernel<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(descs, tile_off, n, total_tiles);
    return ok();
}

int launch_finalize(const double *sum_d, const double *sum_d2, int nb, double *dose, double *sd, size_t nvox,
                    void *stream)
{
    finalize_kernel<<<grid_for(nvox), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(sum_d, sum_d2, nb, dose,
                                                                                         sd, nvox);
    return ok();
}

// partials: at least 5 * n_parts doubles; result: 3 doubles (avg rsd, sigma_bar, d_max)
int launch_rsd(const double *dose, const double *sd, const float *rho, size_t nvox, double *partials, int n_parts,
               double *result, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dmax_kernel<<<n_parts, kThreads, 0, s>>>(dose, rho, nvox, partials);
    max_final_kernel<<<1, 32, 0, s>>>(partials, n_parts, result + 2);
    rsd_kernel<<<n_parts, kThreads, 0, s>>>(dose, sd, rho, nvox, result + 2, partials + n_parts, n_parts);
    rsd_final_kernel<<<1, 32, 0, s>>>(partials + n_parts, n_parts, result + 2, result);
    return ok();
}

int launch_scan_phantom(const uint8_t *mat, const float *rho, size_t nvox, int n_mat, uint32_t *vox,
                        PhantomScan *out, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PhantomScan init{};
    init.first_bad_mat = ~0ull;
    init.first_bad_rho = ~0ull;
    if (cudaMemcpyAsync(out, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) return CTD_ECUDA;
    scan_phantom_kernel<<<grid_for(nvox), kThreads, 0, s>>>(mat, rho, nvox, n_mat, vox, out);
    return ok();
}

int launch_sum(const double *x, size_t n, double *partials, int n_parts, double *result, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sum_kernel<<<n_parts, kThreads, 0, s>>>(x, n, partials, n_parts);
    sum_final_kernel<<<1, 32, 0, s>>>(partials, n_parts, result);
    return ok();
}

}  // namespace ctd
