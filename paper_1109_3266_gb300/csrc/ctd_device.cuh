// ctd_device.cuh -- device arithmetic of the transport (sm_103a), shared by the
// transport kernels: Philox4x32-10, the uniform mapping, the logarithm and
// sincos, float/double bit conversions, the binary64 direction
// renormalisation, the rotation after a scatter, the 1 keV node lookup and the
// R/C-surface lookup.  The transport compiles with fast binary32 arithmetic
// (hardware reciprocal, square root, logarithm and sincos; multiply-adds
// contracted): the decisions it takes are checked history by history against
// binary64 with bounds on these errors.  Binary64 stays exact.
#pragma once

#include <cuda_runtime.h>

#include "ctd_internal.h"

namespace ctd {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kStreamTransport = 0, kStreamSource = 1, kStreamSampler = 3;
constexpr uint32_t kMaxTrials = 1000;
constexpr uint32_t kMaxSteps = 100000000u;

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64 products,
// xor with the round key, key bumped by the Weyl constants.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                     uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// Philox4x32-10 with the ten round keys given (rk[2r], rk[2r+1] = key + r * Weyl)
__device__ __forceinline__ U4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
        const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ U4 block(uint64_t seed, uint64_t h, uint32_t step, uint32_t stream)
{
    return philox(static_cast<uint32_t>(h), static_cast<uint32_t>(h >> 32), step, stream,
                  static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// (2 (x >> 9) + 1) 2^-24: exact in binary32, never 0 or 1.  Built from bits:
// a = 1 + k 2^-23 (k = x >> 9 as the significand) minus (1 - 2^-24) is
// (2k + 1) 2^-24 exactly (2k + 1 < 2^24 fits the significand, so the one
// subtraction does not round): the same value without an integer conversion.
__device__ __forceinline__ float uni(uint32_t x)
{
    return __uint_as_float((x >> 9) | 0x3f800000u) - 0x1.fffffep-1f;
}

// ---------------------------------------------------------------- log and sincos
// The hardware approximations (the SFU's base-2 logarithm and sine/cosine).
// Measured against binary64 over every uniform the transport draws: ln u within
// 1.9e-6 absolutely (a free path -ln(u)/mu_max is then off by at most
// 1.9e-6/mu_max cm), cos and sin of 2 pi t within 3.4e-7.
__device__ __forceinline__ float log32(float x) { return __logf(x); }

// cos and sin of 2 pi t for t in [0, 1): of 2 pi (t - 1/2) in [-pi, pi), where
// the approximation holds its accuracy, negated
__device__ __forceinline__ void sincos_turns(float t, float &c, float &s)
{
    float sn, cs;
    __sincosf((t - 0.5f) * 6.2831853071795865f, &sn, &cs);
    c = -cs;
    s = -sn;
}

// Exact binary32 -> binary64 widening with integer instructions (GB300's FP64
// pipe is narrow; this keeps conversions off it).  Zeros keep their sign;
// subnormals, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double(static_cast<int>(u & 0x80000000u), 0);
    if (ex == 0u || ex == 0xffu) return static_cast<double>(f);
    const uint32_t hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
}

// binary64 -> binary32 by truncating the significand to 23 bits (round toward
// zero); magnitudes below 2^-126 give 0.
__device__ __forceinline__ float trunc32(double d)
{
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(d));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(d));
    const uint32_t ex = (hi >> 20) & 0x7ffu;
    if (ex < 897u) return 0.0f;
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float((hi & 0x80000000u) | (((ex - 896u) & 0xffu) << 23) | m);
}

// Back to unit length after a scatter: d = n2 - 1, the squared norm's excess,
// in binary64 with three fused multiply-adds, ((y^2 - 1) + x^2) + z^2, from the
// widened components (each square is exact in binary64); the correction
// e = -d/2 of one Newton step c = 1.5 - 0.5 n2 for 1/sqrt(n2) from 1 is d
// truncated to binary32 times -1/2, applied to each component with one fused
// multiply-add.
__device__ __forceinline__ void renorm(float &ux, float &uy, float &uz)
{
    const double dx = widen(ux), dy = widen(uy), dz = widen(uz);
    const double d = __fma_rn(dz, dz, __fma_rn(dx, dx, __fma_rn(dy, dy, -1.0)));
    const float ef = trunc32(d) * -0.5f;
    ux = __fmaf_rn(ux, ef, ux);
    uy = __fmaf_rn(uy, ef, uy);
    uz = __fmaf_rn(uz, ef, uz);
}

// E 2^23 as an integer: exact for 1 keV <= E < 2^40 keV (every photon energy of
// the transport is at least the node floor e_min >= 1 keV)
__device__ __forceinline__ unsigned long long kev_fixed(float e)
{
    const uint32_t u = __float_as_uint(e);
    const int ex = static_cast<int>((u >> 23) & 0xffu) - 127;
    const unsigned long long m = (u & 0x7fffffu) | 0x800000u;
    return ex >= 0 ? (m << ex) : (m >> -ex);
}

// binary32 -> binary64 for positive normal numbers only: the exponent rebiased and
// the significand moved into place (the general widen() without its branches)
__device__ __forceinline__ double widen_normal(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t hi = (((u >> 23) + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
}

// Tally deposit of a non-negative binary32 energy into the binary64 grid, as a
// global reduction that returns nothing (a fire-and-forget L2 atomic), also
// when the grid's address was read from shared memory.  A positive deposit is a
// normal number: a photon energy (at least 1 keV) or the difference of two
// energies of at least 1 keV, which is a multiple of their binary32 ulp.
__device__ __forceinline__ void deposit(double *tally, size_t idx, float e)
{
    if (e > 0.0f)
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(tally + idx)),
                     "d"(widen_normal(e))
                     : "memory");
}

// New direction after a scatter of polar cosine mu and azimuth 2 pi tphi.
__device__ __forceinline__ void rotate(float &ux, float &uy, float &uz, float mu, float tphi)
{
    float st2 = __fmaf_rn(-mu, mu, 1.0f);
    if (st2 < 0.0f) st2 = 0.0f;
    const float st = sqrtf(st2);
    float cp, sp;
    sincos_turns(tphi, cp, sp);
    const float a2 = __fmaf_rn(ux, ux, uy * uy);
    float nx, ny, nz;
    if (a2 < static_cast<float>(1e-12)) {
        nx = st * cp;
        ny = st * sp;
        nz = uz > 0.0f ? mu : -mu;
    } else {
        const float a = sqrtf(a2);
        const float rr = st / a;
        nx = __fmaf_rn(rr, __fmaf_rn(ux * uz, cp, -(uy * sp)), ux * mu);
        ny = __fmaf_rn(rr, __fmaf_rn(uy * uz, cp, ux * sp), uy * mu);
        nz = __fmaf_rn(-(a * st), cp, uz * mu);
    }
    ux = nx;
    uy = ny;
    uz = nz;
    renorm(ux, uy, uz);
}

// energy node j and fraction te on the 1 keV grid
__device__ __forceinline__ int enode(float e, int e_min, int n_e, float &te)
{
    const float fe = e - static_cast<float>(e_min);
    int j = static_cast<int>(fe);
    if (j > n_e - 2) j = n_e - 2;
    if (j < 0) j = 0;
    te = fe - static_cast<float>(j);
    return j;
}

// bilinear lookup of mu(zeta, E) on a surface (Sec. 2.2.2); S holds the surface as
// cells of the four corners of a lookup, [n_e - 1][n_zeta - 1] float4, so one
// 16-byte read fetches them
__device__ __forceinline__ float surface(const float *__restrict__ S, int n_zeta, int j, float te, float z)
{
    const float zf = __fmul_rn(z, static_cast<float>(n_zeta - 1));   // rounded on its own, never fused
    int i = static_cast<int>(zf);
    if (i > n_zeta - 2) i = n_zeta - 2;
    const float a = zf - static_cast<float>(i);
    const float4 c = __ldg(reinterpret_cast<const float4 *>(S) + (static_cast<size_t>(j) * (n_zeta - 1) + i));
    const float a0 = c.x, a1 = c.y, b0 = c.z, b1 = c.w;
    const float lo = __fmaf_rn(a, a1 - a0, a0);
    const float hi = __fmaf_rn(a, b1 - b0, b0);
    float mu = __fmaf_rn(te, hi - lo, lo);
    if (mu > 1.0f) mu = 1.0f;
    if (mu < -1.0f) mu = -1.0f;
    return mu;
}

}  // namespace dev
}  // namespace ctd
