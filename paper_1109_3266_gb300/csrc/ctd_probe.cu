// ctd_probe.cu -- memory-system probes that bound the transport kernel: the
// rate of binary64 L2 reductions into random tally slots (the deposits of
// Sec. 2.1) and of random voxel gathers (the Woodcock step's fetch of material
// and density).  Measurement aids only; nothing on the transport path calls them.
#include <cuda_runtime.h>

#include "ctd_internal.h"

namespace ctd {
namespace {

// lowbias32 integer hash (C. Wellons' published 32-bit mixer)
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// slot of operation i, uniform on [0, n_slots) for n_slots < 2^32
__device__ __forceinline__ uint32_t slot(uint32_t i, uint32_t salt, uint32_t n_slots)
{
    return static_cast<uint32_t>((static_cast<uint64_t>(mix32(i ^ salt)) * n_slots) >> 32);
}

constexpr int kUnroll = 8;

__global__ void probe_red_kernel(double *__restrict__ buf, uint32_t n_slots, uint32_t rounds, uint32_t salt)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r = 0; r < rounds; ++r) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const uint32_t i = (r * kUnroll + k) * stride + t;
            asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(buf + slot(i, salt, n_slots))),
                         "d"(1.0)
                         : "memory");
        }
    }
}

__global__ void probe_gather4_kernel(const float *__restrict__ buf, uint32_t n_slots, uint32_t rounds, uint32_t salt,
                                     float *__restrict__ out)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    float acc = 0.0f;
    for (uint32_t r = 0; r < rounds; ++r) {
        float v[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) v[k] = __ldg(&buf[slot((r * kUnroll + k) * stride + t, salt, n_slots)]);
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) acc += v[k];
    }
    out[t] = acc;
}

__global__ void probe_voxel_kernel(const uint8_t *__restrict__ mat, const float *__restrict__ rho, uint32_t n_slots,
                                   uint32_t rounds, uint32_t salt, float *__restrict__ out)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    float acc = 0.0f;
    for (uint32_t r = 0; r < rounds; ++r) {
        float v[kUnroll];
        int m[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const uint32_t s = slot((r * kUnroll + k) * stride + t, salt, n_slots);
            m[k] = __ldg(&mat[s]);
            v[k] = __ldg(&rho[s]);
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) acc += v[k] * static_cast<float>(m[k] + 1);
    }
    out[t] = acc;
}

}  // namespace

// One probe launch of `rounds` x 8 operations per thread.  Buffers: kind 0
// `dbuf` (n_slots doubles); kind 1 `fbuf` (n_slots floats); kind 2 `mbuf`
// (n_slots bytes) and `fbuf`; `out` holds grid x block floats (kinds 1, 2).
int launch_probe(int kind, double *dbuf, float *fbuf, uint8_t *mbuf, float *out, uint32_t n_slots, uint32_t rounds,
                 uint32_t salt, int grid, int block, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0) probe_red_kernel<<<grid, block, 0, s>>>(dbuf, n_slots, rounds, salt);
    else if (kind == 1) probe_gather4_kernel<<<grid, block, 0, s>>>(fbuf, n_slots, rounds, salt, out);
    else probe_voxel_kernel<<<grid, block, 0, s>>>(mbuf, fbuf, n_slots, rounds, salt, out);
    return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
}

}  // namespace ctd
