// ctd_fluence.cu -- the paper's Metropolis-Hastings beamlet sampler (Algorithm A1)
// on the device, one chain per thread as the paper runs it, for its comparison
// with the alias-table draw the transport uses (ctd_mh_beamlets).
#include <cuda_runtime.h>

#include "ctd_device.cuh"
#include "ctd_host.h"

namespace {

using namespace ctd::dev;

constexpr uint32_t kStreamMh = 4;

// Chain c takes particles [lo_c, lo_c + len_c) (the first n mod chains chains one
// more), starts at beamlet i0; particle i: trial beamlet J from the first word of
// Philox block (i, 0, stream 4), zeta from the second, J kept if zeta < f_J / f_last
// (binary64, as the acceptance ratio is defined).
__global__ void mh_chain_kernel(int n_f, const double *__restrict__ f, int i0, uint64_t n, uint64_t seed,
                                uint64_t chains, unsigned long long *counts)
{
    const uint64_t per = n / chains, rem = n % chains;
    for (uint64_t c = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; c < chains;
         c += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t lo = per * c + (c < rem ? c : rem);
        const uint64_t len = per + (c < rem ? 1 : 0);
        int last = i0;
        for (uint64_t i = lo; i < lo + len; ++i) {
            const U4 b = block(seed, i, 0, kStreamMh);
            const int j = static_cast<int>((static_cast<uint64_t>(b.x) * static_cast<uint64_t>(n_f)) >> 32);
            const double zeta = static_cast<double>(2u * (b.y >> 9) + 1u) * 0x1p-24;
            const int cur = zeta < __ldg(&f[j]) / __ldg(&f[last]) ? j : last;
            atomicAdd(&counts[cur], 1ull);
            last = cur;
        }
    }
}

}  // namespace

using namespace ctd::host;

extern "C" int ctd_mh_beamlets(ctd_ctx *ctx, int n_f, const double *f, int i0, uint64_t n, uint64_t seed,
                               uint64_t chains, uint64_t *counts)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (!f || !counts || n_f < 1 || n_f > (1 << 24) || i0 < 0 || i0 >= n_f || chains < 1 || chains > (1ull << 32))
        return fail(CTD_EINVAL, "need 1 <= n_f <= 2^24 intensities, 0 <= i0 < n_f, 1 <= chains <= 2^32");
    for (int i = 0; i < n_f; ++i)
        if (!(f[i] >= 0.0) || !std::isfinite(f[i])) return fail(CTD_EINVAL, "intensity %d is not finite and >= 0", i);
    DevBuf<double> df;
    DevBuf<unsigned long long> dc;
    if ((rc = df.ensure(n_f)) || (rc = dc.ensure(n_f))) return rc;
    CK(cudaMemcpyAsync(df.p, f, n_f * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(dc.p, 0, n_f * sizeof(unsigned long long), ctx->stream));
    const int block = 128;
    const uint64_t want = (chains + block - 1) / block;
    const int grid = static_cast<int>(want < 65536 ? want : 65536);
    mh_chain_kernel<<<grid, block, 0, ctx->stream>>>(n_f, df.p, i0, n, seed, chains, dc.p);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(counts, dc.p, n_f * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CTD_OK;
}
