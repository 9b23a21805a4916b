// ctd_stats.cu -- batch statistics of the dose engine (Sec. 2.2.1) and the
// precision measures of Sec. 3.1, as streaming kernels over the FP64 grids.
#include <cuda_runtime.h>

#include "ctd_internal.h"

namespace ctd {
namespace {

constexpr int kThreads = 256;

// GB300's binary64 pipe is narrow, so these kernels divide by nothing per voxel:
// the fold multiplies by the voxel's 1/rho (correctly rounded once, when the
// phantom is created), the mean and variance by 1/nb and 1/(nb (nb - 1)) from
// the host, and the avg RSD's s/D by a Newton-Raphson reciprocal of D.

// 1/x for a positive x: the hardware's approximate reciprocal (relative error
// below 2^-22) and two Newton-Raphson steps y <- y + y (1 - x y), each of which
// squares the relative error, so the result is within an ulp or two of 1/x; a
// subnormal x (which the approximation flushes) takes the division.
__device__ __forceinline__ double recip(double x)
{
    if (x < 2.2250738585072014e-308) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// Fold one batch: d = E_b / (m_v n_b) in Gy per history; accumulate d and d^2,
// keep the raw energy, clear the batch tally.  scale = keV->J * 1000 / (V n_b),
// rinv = 1 / rho (0 where rho = 0).  Four voxels a grid stride apart per thread
// and pass, so that their loads are in flight together.
constexpr int kFoldUnroll = 4;

__device__ __forceinline__ void fold_voxel(double t, size_t v, double *__restrict__ tally,
                                           const double *__restrict__ rinv, double *__restrict__ sum_d,
                                           double *__restrict__ sum_d2, double *__restrict__ edep, double scale)
{
    const double d = (t * scale) * rinv[v];
    edep[v] += t;
    tally[v] = 0.0;
    sum_d[v] += d;
    sum_d2[v] += d * d;
}

__global__ void fold_kernel(double *__restrict__ tally, const double *__restrict__ rinv, double *__restrict__ sum_d,
                            double *__restrict__ sum_d2, double *__restrict__ edep, size_t nvox, double scale)
{
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t v0 = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v0 < nvox;
         v0 += kFoldUnroll * stride) {
        double t[kFoldUnroll];
#pragma unroll
        for (int k = 0; k < kFoldUnroll; ++k) {
            const size_t v = v0 + k * stride;
            t[k] = v < nvox ? tally[v] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kFoldUnroll; ++k)
            if (t[k] != 0.0) fold_voxel(t[k], v0 + k * stride, tally, rinv, sum_d, sum_d2, edep, scale);
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
            if (t != 0.0) fold_voxel(t, v, d.tally, d.rinv, d.sum_d, d.sum_d2, d.edep, d.scale);
        }
    }
}

// Mean over nb batches and its standard error: s^2 = (sum d^2 - nb D^2) / (nb (nb - 1)),
// with inv_nb = 1/nb and inv_nn = 1/(nb (nb - 1)).
__device__ __forceinline__ void mean_sd(double s1, double s2, int nb, double inv_nb, double inv_nn, double &D,
                                        double &sd)
{
    D = s1 * inv_nb;
    const double var = (s2 - nb * D * D) * inv_nn;
    sd = var > 0.0 ? sqrt(var) : 0.0;
}

__global__ void finalize_kernel(const double *__restrict__ sum_d, const double *__restrict__ sum_d2, int nb,
                                double inv_nb, double inv_nn, double *__restrict__ dose, double *__restrict__ sd,
                                size_t nvox)
{
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
        double D, s;
        mean_sd(sum_d[v], sum_d2[v], nb, inv_nb, inv_nn, D, s);
        dose[v] = D;
        sd[v] = s;
    }
}

// Sum of n partials in a fixed order by one warp: lane l adds partials l, l + 32,
// ... in turn, then the lanes' sums are added pairwise by shuffles.
__device__ __forceinline__ double warp_sum(const double *p, int n)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
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
    // doses are >= +0: their bit patterns order like their values (integer compares)
    long long m = 0;
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x)
        if (rho[v] >= 0.1f) {
            const long long b = __double_as_longlong(dose[v]);
            if (b > m) m = b;
        }
    __shared__ long long sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_down_sync(0xffffffffu, m, o);
        if (y > m) m = y;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int w = 0; w < kThreads / 32; ++w)
            if (sh[w] > b) b = sh[w];
        partials[blockIdx.x] = __longlong_as_double(b);
    }
}

__global__ void max_final_kernel(const double *partials, int n, double *out)
{
    double b = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) b = fmax(b, partials[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
    if (threadIdx.x == 0) *out = b;
}

// pass 2: sums for avg RSD (s/D over D > 0.1 D_max) and the paper's sigma_bar
// (s/D_max over D > 0.2 D_max), both inside rho >= 0.1
__global__ void rsd_kernel(const double *__restrict__ dose, const double *__restrict__ sd,
                           const float *__restrict__ rho, size_t nvox, const double *dmax_p, double *partials,
                           int n_parts)
{
    // doses are >= +0, and the bit patterns of non-negative doubles order like their
    // values: the thresholds are compared as integers, the voxels counted in integers
    const double dmax = *dmax_p;
    const long long lo1 = __double_as_longlong(0.1 * dmax), lo2 = __double_as_longlong(0.2 * dmax);
    double rel = 0.0, s2 = 0.0;
    unsigned n1 = 0, n2 = 0;
    for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < nvox;
         v += static_cast<size_t>(gridDim.x) * blockDim.x) {
        if (!(rho[v] >= 0.1f)) continue;
        const double D = dose[v];
        const long long b = __double_as_longlong(D);
        if (b > lo1) {
            rel += sd[v] * recip(D);
            ++n1;
        }
        if (b > lo2) {
            s2 += sd[v];
            ++n2;
        }
    }
    double x[4] = {rel, static_cast<double>(n1), s2, static_cast<double>(n2)};
    block_sums<4>(x, partials, n_parts);
}

__global__ void rsd_final_kernel(const double *partials, int n_parts, const double *dmax_p, double *result)
{
    double s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] = warp_sum(partials + k * n_parts, n_parts);
    if (threadIdx.x == 0) {
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
    const double s = warp_sum(partials, n_parts);
    if (threadIdx.x == 0) *result = s;
}

// One pass over a new phantom's voxels (grid-stride): range checks and the
// per-material presence and largest density, reduced in shared memory, then one
// global atomic per block and quantity.  -0 densities count as +0.
__global__ void scan_phantom_kernel(const uint8_t *__restrict__ mat, const float *__restrict__ rho, size_t nvox,
                                    int n_mat, uint32_t *__restrict__ vox, double *__restrict__ rinv,
                                    PhantomScan *out)
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
        rinv[v] = f ? 1.0 / static_cast<double>(r) : 0.0;
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

int launch_fold(double *tally, const double *rinv, double *sum_d, double *sum_d2, double *edep, size_t nvox,
                double scale, void *stream)
{
    const size_t per_pass = (nvox + kFoldUnroll - 1) / kFoldUnroll;
    fold_kernel<<<grid_for(per_pass), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(tally, rinv, sum_d, sum_d2,
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
    const double inv_nb = 1.0 / nb, inv_nn = 1.0 / (static_cast<double>(nb) * (nb - 1));
    finalize_kernel<<<grid_for(nvox), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(sum_d, sum_d2, nb, inv_nb,
                                                                                         inv_nn, dose, sd, nvox);
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

int launch_scan_phantom(const uint8_t *mat, const float *rho, size_t nvox, int n_mat, uint32_t *vox, double *rinv,
                        PhantomScan *out, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PhantomScan init{};
    init.first_bad_mat = ~0ull;
    init.first_bad_rho = ~0ull;
    if (cudaMemcpyAsync(out, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) return CTD_ECUDA;
    scan_phantom_kernel<<<grid_for(nvox), kThreads, 0, s>>>(mat, rho, nvox, n_mat, vox, rinv, out);
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
