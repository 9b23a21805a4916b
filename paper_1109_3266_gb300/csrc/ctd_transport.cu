// ctd_transport.cu -- photon transport kernel of the dose engine (sm_103a).
//
// One persistent grid per batch.  Each lane holds one photon history until it
// ends (photoelectric absorption, cutoff, escape, termination) and then takes
// the next history of its warp's claim; warps claim runs of consecutive
// histories from a global counter, so a warp's lanes work on one 1 keV
// spectrum interval at a time (Sec. 2.2.5).  Per history (Fig. 2, Sec. 2.1):
// source sampling, Woodcock steps against mu_max(E), the interaction choice,
// R/C-surface polar angles (Sec. 2.2.2-2.2.3) and local deposition into the
// FP64 batch tally with L2 atomics.
//
// Numerics: binary32 transport compiled with --fmad=false, so every multiply
// and add rounds on its own; fused multiply-adds appear only as explicit
// __fmaf_rn.  Logarithm and sincos are the series defined below, identical on
// every platform.  Direction renormalisation after a scatter is binary64.
#include <cuda_runtime.h>

#include "ctd_internal.h"

namespace ctd {
namespace {

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

__device__ __forceinline__ U4 block(uint64_t seed, uint64_t h, uint32_t step, uint32_t stream)
{
    return philox(static_cast<uint32_t>(h), static_cast<uint32_t>(h >> 32), step, stream,
                  static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// (2 (x >> 9) + 1) 2^-24: exact in binary32, never 0 or 1
__device__ __forceinline__ float uni(uint32_t x)
{
    return static_cast<float>(2u * (x >> 9) + 1u) * 0x1p-24f;
}

// ---------------------------------------------------------------- binary32 log and sincos
// ln x: x = 2^e m with m in (sqrt(1/2), sqrt(2)], ln m = 2 atanh(s), s = (m-1)/(m+1),
// atanh series through s^11 in Horner form, then + e ln 2 with ln 2 split in two.
__device__ __forceinline__ float log32(float x)
{
    uint32_t bits = __float_as_uint(x);
    int e = static_cast<int>((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float f = m - 1.0f;
    const float s = f / (2.0f + f);
    const float z = s * s;
    float p = __fmaf_rn(z, 0x1.745d18p-4f, 0x1.c71c72p-4f);
    p = __fmaf_rn(z, p, 0x1.24924ap-3f);
    p = __fmaf_rn(z, p, 0x1.99999ap-3f);
    p = __fmaf_rn(z, p, 0x1.555556p-2f);
    const float r = z * p;
    const float s2 = s + s;
    const float lnm = __fmaf_rn(s2, r, s2);
    const float ef = static_cast<float>(e);
    return __fmaf_rn(ef, 0x1.62e430p-1f, __fmaf_rn(ef, -0x1.05c610p-29f, lnm));
}

// cos and sin of 2 pi t: exact reduction in turns to a quarter-turn offset in
// [-1/8, 1/8], Taylor polynomials of sin (to x^9) and cos (to x^10).
__device__ __forceinline__ void sincos_turns(float t, float &c, float &s)
{
    const float w = t - floorf(t);
    int q = static_cast<int>(w * 4.0f);
    float r = w - static_cast<float>(q) * 0.25f;
    if (r > 0.125f) {
        r = r - 0.25f;
        q = q + 1;
    }
    const float x = r * 0x1.921fb6p+2f;
    const float x2 = x * x;
    float ps = __fmaf_rn(x2, 0x1.71de3ap-19f, -0x1.a01a02p-13f);
    ps = __fmaf_rn(x2, ps, 0x1.111112p-7f);
    ps = __fmaf_rn(x2, ps, -0x1.555556p-3f);
    const float sn = __fmaf_rn(x * x2, ps, x);
    float pc = __fmaf_rn(x2, -0x1.27e4fcp-22f, 0x1.a01a02p-16f);
    pc = __fmaf_rn(x2, pc, -0x1.6c16c2p-10f);
    pc = __fmaf_rn(x2, pc, 0x1.555556p-5f);
    pc = __fmaf_rn(x2, pc, -0.5f);
    const float cs = __fmaf_rn(x2, pc, 1.0f);
    switch (q & 3) {
    case 0: c = cs; s = sn; break;
    case 1: c = -sn; s = cs; break;
    case 2: c = -cs; s = -sn; break;
    default: c = sn; s = -cs; break;
    }
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

// Back to unit length after a scatter: the squared norm n2 and the correction
// e = c - 1 of one Newton step c = 1.5 - 0.5 n2 for 1/sqrt(n2) from 1 are
// binary64 (the products of widened floats are exact, so the fused forms equal
// the separately rounded ones); e, truncated to binary32, is applied to each
// component with one fused multiply-add.
__device__ __forceinline__ void renorm(float &ux, float &uy, float &uz)
{
    const double dx = widen(ux), dy = widen(uy), dz = widen(uz);
    const double n2 = __fma_rn(dz, dz, __fma_rn(dx, dx, __dmul_rn(dy, dy)));
    const double e = __fma_rn(-0.5, n2, 0.5);
    const float ef = trunc32(e);
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

// tally deposit of a non-negative binary32 energy into the binary64 grid
__device__ __forceinline__ void deposit(double *tally, size_t idx, float e)
{
    if (e > 0.0f) atomicAdd(tally + idx, widen(e));
}

// New direction after a scatter of polar cosine mu and azimuth 2 pi tphi.
__device__ __forceinline__ void rotate(float &ux, float &uy, float &uz, float mu, float tphi)
{
    float st2 = 1.0f - mu * mu;
    if (st2 < 0.0f) st2 = 0.0f;
    const float st = sqrtf(st2);
    float cp, sp;
    sincos_turns(tphi, cp, sp);
    const float a2 = ux * ux + uy * uy;
    float nx, ny, nz;
    if (a2 < static_cast<float>(1e-12)) {
        nx = st * cp;
        ny = st * sp;
        nz = uz > 0.0f ? mu : -mu;
    } else {
        const float a = sqrtf(a2);
        const float rr = st / a;
        nx = ux * mu + rr * ((ux * uz) * cp - uy * sp);
        ny = uy * mu + rr * ((uy * uz) * cp + ux * sp);
        nz = uz * mu - (a * st) * cp;
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

// bilinear lookup of mu(zeta, E) on a surface (Sec. 2.2.2)
__device__ __forceinline__ float surface(const float *__restrict__ S, int n_zeta, int j, float te, float z)
{
    const float zf = z * static_cast<float>(n_zeta - 1);
    int i = static_cast<int>(zf);
    if (i > n_zeta - 2) i = n_zeta - 2;
    const float a = zf - static_cast<float>(i);
    const float *r0 = S + static_cast<size_t>(j) * n_zeta + i;
    const float *r1 = r0 + n_zeta;
    const float a0 = __ldg(r0), a1 = __ldg(r0 + 1), b0 = __ldg(r1), b1 = __ldg(r1 + 1);
    const float lo = a0 + a * (a1 - a0);
    const float hi = b0 + a * (b1 - b0);
    float mu = lo + te * (hi - lo);
    if (mu > 1.0f) mu = 1.0f;
    if (mu < -1.0f) mu = -1.0f;
    return mu;
}

struct Photon {
    float x, y, z, ux, uy, uz, e;
    uint64_t h;
    uint32_t step;
    int nreal;
};

struct LaneCounts {
    uint32_t n[10];
    unsigned long long e_emitted, e_escaped;   // keV * 2^23
};

// Source sampling (Secs. 2.2.5-2.2.6).  Returns true if the photon enters the phantom.
__device__ __forceinline__ int bin_search(const TransportParams &P, uint64_t local)
{
    // largest bin j with pref[j] <= local
    int lo = 0, hi = P.nbins - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&P.pref[mid]) <= local) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Source photon of local history `local` (global index h); `bin` is the 1 keV
// interval of the warp's claim start, a lower bound for this history's interval.
__device__ __forceinline__ bool source(const TransportParams &P, uint64_t h, uint64_t local, int bin, Photon &ph,
                                       LaneCounts &cnt)
{
    while (bin < P.nbins - 1 && __ldg(&P.pref[bin + 1]) <= local) ++bin;
    const U4 b0 = block(P.seed, h, 0, kStreamSource);
    const float elo = __ldg(&P.bin_lo[bin]), ehi = __ldg(&P.bin_hi[bin]);
    const float e = elo + (ehi - elo) * uni(b0.x);
    cnt.e_emitted += kev_fixed(e);
    float cb = 1.0f, sb = 0.0f;
    if (P.src_kind == CTD_SRC_ARC) {
        if (P.continuous) {
            sincos_turns(P.a0t + P.awt * uni(b0.y), cb, sb);
        } else {
            const uint32_t k = static_cast<uint32_t>((static_cast<uint64_t>(b0.y) * static_cast<uint64_t>(P.n_proj)) >> 32);
            cb = __ldg(&P.cb[k]);
            sb = __ldg(&P.sb[k]);
        }
    }
    // uniform in solid angle over the field: uniform point, accepted with cos^3
    bool accepted = false;
    float uu = 0.0f, vv = 0.0f, q = 0.0f;
    for (uint32_t t = 1; t <= kMaxTrials; ++t) {
        const U4 b = block(P.seed, h, t, kStreamSource);
        uu = P.ulo + P.uw * uni(b.x);
        vv = P.vlo + P.vw * uni(b.y);
        q = (P.D2 + uu * uu) + vv * vv;
        const float c2 = P.D2 / q;
        const float acc = c2 * sqrtf(c2);
        if (uni(b.z) < acc) {
            accepted = true;
            break;
        }
    }
    if (!accepted) {
        cnt.n[kCntAborted]++;
        cnt.e_escaped += kev_fixed(e);
        return false;
    }
    const float inv = 1.0f / sqrtf(q);
    float ux, uy, uz, rx, ry, rz;
    if (P.src_kind == CTD_SRC_ARC) {
        ux = (uu * cb - P.D * sb) * inv;
        uy = ((-uu) * sb - P.D * cb) * inv;
        uz = vv * inv;
        rx = P.D * sb;
        ry = P.D * cb;
        rz = 0.0f;
    } else {
        ux = uu * inv;
        uy = vv * inv;
        uz = P.D * inv;
        rx = 0.0f;
        ry = 0.0f;
        rz = -P.D;
    }
    renorm(ux, uy, uz);
    // entry into the box (slab method); outside is vacuum
    const float t0x = (P.bx0 - rx) / ux, t1x = (P.bx1 - rx) / ux;
    const float t0y = (P.by0 - ry) / uy, t1y = (P.by1 - ry) / uy;
    const float t0z = (P.bz0 - rz) / uz, t1z = (P.bz1 - rz) / uz;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fminf(t0z, t1z));
    const float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fmaxf(t0z, t1z));
    if (!(tn < tf) || !(tf > 0.0f)) {
        cnt.n[kCntMissed]++;
        cnt.e_escaped += kev_fixed(e);
        return false;
    }
    if (tn < 0.0f) tn = 0.0f;
    ph.x = rx + tn * ux;
    ph.y = ry + tn * uy;
    ph.z = rz + tn * uz;
    ph.ux = ux;
    ph.uy = uy;
    ph.uz = uz;
    ph.e = e;
    ph.h = h;
    ph.step = 0;
    ph.nreal = 0;
    return true;
}

// Site of a real interaction found by a flight
struct Hit {
    size_t idx;       // voxel
    int m;            // material
    int j;            // energy node
    float te;         // energy fraction
    int type;         // 0 photoelectric, 1 Compton, 2 Rayleigh
    uint32_t rz, rw;  // the step's random words for zeta and phi
};

enum { kEnded = 0, kFictitious = 1, kReal = 2 };

// One Woodcock flight (Sec. 2.1): free path against mu_max(E), the move, the
// escape test, the voxel and the interaction type.
__device__ __forceinline__ int flight(const TransportParams &P, const float4 *__restrict__ s_tab,
                                      const float *__restrict__ s_mm, Photon &ph, LaneCounts &cnt, Hit &hit)
{
    if (ph.step >= kMaxSteps) {
        cnt.n[kCntAborted]++;
        cnt.e_escaped += kev_fixed(ph.e);
        return kEnded;
    }
    const U4 b = block(P.seed, ph.h, ph.step, kStreamTransport);
    ph.step++;
    cnt.n[kCntSteps]++;
    float te;
    const int j = enode(ph.e, P.e_min, P.n_e, te);
    const float m0 = s_mm[j], m1 = s_mm[j + 1];
    const float mmax = m0 + te * (m1 - m0);
    const float path = (-log32(uni(b.x))) / mmax;
    ph.x = ph.x + path * ph.ux;
    ph.y = ph.y + path * ph.uy;
    ph.z = ph.z + path * ph.uz;
    const float fx = (ph.x - P.bx0) * P.ix, fy = (ph.y - P.by0) * P.iy, fz = (ph.z - P.bz0) * P.iz;
    if (!(fx >= 0.0f && fx < static_cast<float>(P.nx) && fy >= 0.0f && fy < static_cast<float>(P.ny) &&
          fz >= 0.0f && fz < static_cast<float>(P.nz))) {
        cnt.n[kCntEscaped]++;
        cnt.e_escaped += kev_fixed(ph.e);
        return kEnded;
    }
    const size_t idx = static_cast<size_t>(static_cast<int>(fx)) +
                       static_cast<size_t>(P.nx) *
                           (static_cast<size_t>(static_cast<int>(fy)) + static_cast<size_t>(P.ny) * static_cast<size_t>(static_cast<int>(fz)));
    const int m = __ldg(&P.mat[idx]);
    const float rho = __ldg(&P.rho[idx]);
    const float4 A = s_tab[m * P.n_e + j], B = s_tab[m * P.n_e + j + 1];
    const float c1 = A.x + te * (B.x - A.x);
    const float c2 = A.y + te * (B.y - A.y);
    const float c3 = A.z + te * (B.z - A.z);
    // interaction type with probabilities mu_i / mu_max
    const float y = uni(b.y) * mmax;
    int type;
    if (y < rho * c1) type = 0;
    else if (y < rho * c2) type = 1;
    else if (y < rho * c3) type = 2;
    else type = 3;
    if (type == 3) {
        cnt.n[kCntFict]++;
        return kFictitious;
    }
    hit.idx = idx;
    hit.m = m;
    hit.j = j;
    hit.te = te;
    hit.type = type;
    hit.rz = b.z;
    hit.rw = b.w;
    return kReal;
}

// A real interaction: local deposition, C/R-surface polar angle, rotation.
// Returns false when the history has ended.
__device__ __forceinline__ bool interact(const TransportParams &P, Photon &ph, const Hit &hit, LaneCounts &cnt)
{
    ph.nreal++;
    if (hit.type == 0) {
        // photoelectric absorption: the electron deposits E here
        cnt.n[kCntPe]++;
        deposit(P.tally, hit.idx, ph.e);
        return false;
    }
    const float *S = hit.type == 1 ? P.csurf : P.rsurf + static_cast<size_t>(hit.m) * P.n_e * P.n_zeta;
    const float mu = surface(S, P.n_zeta, hit.j, hit.te, uni(hit.rz));
    if (hit.type == 1) {
        // Compton: E' = E / (1 + (E/mc^2)(1 - mu)), the electron gets E - E'
        cnt.n[kCntCompton]++;
        const float k = ph.e / static_cast<float>(kMec2);
        const float ep = ph.e / (1.0f + k * (1.0f - mu));
        if (ep < static_cast<float>(P.e_min)) {
            cnt.n[kCntCutoff]++;
            deposit(P.tally, hit.idx, ph.e);
            return false;
        }
        deposit(P.tally, hit.idx, ph.e - ep);
        ph.e = ep;
    } else {
        cnt.n[kCntRayleigh]++;
    }
    if (P.mode == CTD_MODE_MAX_REAL && ph.nreal >= P.max_real) {
        cnt.n[kCntTerminated]++;
        cnt.e_escaped += kev_fixed(ph.e);
        return false;
    }
    rotate(ph.ux, ph.uy, ph.uz, mu, uni(hit.rw));
    return true;
}

// Flights until a real interaction, the escape, or flight_cap fictitious
// flights; then the interaction.  Returns false when the history has ended.
__device__ __forceinline__ bool walk(const TransportParams &P, const float4 *__restrict__ s_tab,
                                     const float *__restrict__ s_mm, Photon &ph, LaneCounts &cnt)
{
    Hit hit;
    int f, k = 0;
    do {
        f = flight(P, s_tab, s_mm, ph, cnt, hit);
    } while (f == kFictitious && ++k < P.flight_cap);
    if (f == kEnded) return false;
    if (f == kFictitious) return true;
    return interact(P, ph, hit, cnt);
}

// Per-warp photon queue in shared memory: source photons are made 32 at a
// time by the whole warp and taken by lanes whose history has ended.
constexpr int kQueue = 64;
constexpr size_t kQueueBytes = kQueue * (7 * sizeof(float) + sizeof(uint64_t));

template <int kMinBlocks>
__global__ void __launch_bounds__(256, kMinBlocks) transport_kernel(const TransportParams P)
{
    extern __shared__ float4 smem[];
    float4 *s_tab = smem;
    const int ntab = P.n_mat * P.n_e;
    float *s_mm = reinterpret_cast<float *>(smem + ntab);
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) s_tab[i] = reinterpret_cast<const float4 *>(P.tab)[i];
    for (int i = threadIdx.x; i < P.n_e; i += blockDim.x) s_mm[i] = P.mmax[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *qbase = reinterpret_cast<unsigned char *>(smem + ntab + (P.n_e + 3) / 4) + warp * kQueueBytes;
    uint64_t *qh = reinterpret_cast<uint64_t *>(qbase);
    float *qf = reinterpret_cast<float *>(qh + kQueue);   // [7][kQueue]: x y z ux uy uz e
    __syncthreads();

    const unsigned lt_mask = (1u << lane) - 1u;
    LaneCounts cnt;
#pragma unroll
    for (int i = 0; i < 10; ++i) cnt.n[i] = 0;
    cnt.e_emitted = 0;
    cnt.e_escaped = 0;

    Photon ph;
    bool alive = false;
    uint64_t pool_next = 0, pool_end = 0;   // warp-uniform claim of local history indices
    int pool_bin = 0;                       // 1 keV interval of the claim's first history
    bool drained = false;
    int qcount = 0;                         // photons waiting in the warp's queue
    for (;;) {
        // top the queue up with one round of 32 source photons
        if (qcount < 32 && !drained) {
            if (pool_next >= pool_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(P.work, static_cast<unsigned long long>(P.chunk));
                base = __shfl_sync(kFull, base, 0);
                const uint64_t b = P.local_begin + base;
                if (b >= P.local_end) {
                    drained = true;
                } else {
                    pool_next = b;
                    pool_end = b + P.chunk < P.local_end ? b + P.chunk : P.local_end;
                    pool_bin = bin_search(P, pool_next);
                }
            }
            if (!drained) {
                const uint64_t avail = pool_end - pool_next;
                const unsigned take = avail < 32 ? static_cast<unsigned>(avail) : 32u;
                Photon np;
                bool ok = false;
                if (lane < take) {
                    const uint64_t local = pool_next + lane;
                    ok = source(P, P.h_base + local, local, pool_bin, np, cnt);
                }
                const unsigned okm = __ballot_sync(kFull, ok);
                if (ok) {
                    const int slot = qcount + __popc(okm & lt_mask);
                    qh[slot] = np.h;
                    qf[0 * kQueue + slot] = np.x;
                    qf[1 * kQueue + slot] = np.y;
                    qf[2 * kQueue + slot] = np.z;
                    qf[3 * kQueue + slot] = np.ux;
                    qf[4 * kQueue + slot] = np.uy;
                    qf[5 * kQueue + slot] = np.uz;
                    qf[6 * kQueue + slot] = np.e;
                }
                qcount += __popc(okm);
                pool_next += take;
            }
            __syncwarp();
        }
        // lanes without a photon take one from the queue
        const unsigned need = __ballot_sync(kFull, !alive);
        const int npop = __popc(need) < qcount ? __popc(need) : qcount;
        if (!alive) {
            const int rank = __popc(need & lt_mask);
            if (rank < npop) {
                const int slot = qcount - 1 - rank;
                ph.h = qh[slot];
                ph.x = qf[0 * kQueue + slot];
                ph.y = qf[1 * kQueue + slot];
                ph.z = qf[2 * kQueue + slot];
                ph.ux = qf[3 * kQueue + slot];
                ph.uy = qf[4 * kQueue + slot];
                ph.uz = qf[5 * kQueue + slot];
                ph.e = qf[6 * kQueue + slot];
                ph.step = 0;
                ph.nreal = 0;
                alive = true;
            }
        }
        qcount -= npop;
        __syncwarp();
        if (!__any_sync(kFull, alive)) {
            if (drained && qcount == 0) break;
            continue;
        }
        if (alive) alive = walk(P, s_tab, s_mm, ph, cnt);
    }

    // flush the lane counters: warp sums, one atomic per warp
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        unsigned long long v = cnt.n[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
        if (lane == 0 && v) atomicAdd(&P.counts->n[i], v);
    }
    // energies: 128-bit fixed-point totals (lo, hi) so that no run can overflow them
    unsigned long long em = cnt.e_emitted, es = cnt.e_escaped;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        em += __shfl_down_sync(kFull, em, o);
        es += __shfl_down_sync(kFull, es, o);
    }
    if (lane == 0) {
        const unsigned long long o1 = atomicAdd(&P.counts->e_fix[0], em);
        if (o1 + em < o1) atomicAdd(&P.counts->e_fix[1], 1ull);
        const unsigned long long o2 = atomicAdd(&P.counts->e_fix[2], es);
        if (o2 + es < o2) atomicAdd(&P.counts->e_fix[3], 1ull);
    }
}

__global__ void sample_mu_kernel(const float *surf, int n_zeta, int n_e, int e_min, float e, uint64_t seed,
                                 uint64_t n, double *out)
{
    float te;
    const int j = enode(e, e_min, n_e, te);
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const U4 b = block(seed, i, 0, kStreamSampler);
        out[i] = static_cast<double>(surface(surf, n_zeta, j, te, uni(b.x)));
    }
}

__global__ void eval_math_kernel(int fn, const float *x, float *out, size_t n)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        if (fn == 0) {
            out[i] = log32(x[i]);
        } else {
            float c, s;
            sincos_turns(x[i], c, s);
            out[2 * i] = c;
            out[2 * i + 1] = s;
        }
    }
}

}  // namespace

size_t transport_smem_bytes(int n_mat, int n_e, int threads)
{
    return static_cast<size_t>(n_mat) * n_e * sizeof(float4) + static_cast<size_t>((n_e + 3) / 4) * sizeof(float4) +
           static_cast<size_t>(threads / 32) * kQueueBytes;
}

// The register budget follows the residency asked for: 4 or more blocks of
// 256 threads per SM cap the kernel at 64 registers, fewer at 85.
template <int kMinBlocks>
int launch_transport_t(const TransportParams &p, int grid, int block, size_t smem, cudaStream_t stream)
{
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(transport_kernel<kMinBlocks>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem)) != cudaSuccess)
            return CTD_ECUDA;
    }
    transport_kernel<kMinBlocks><<<grid, block, smem, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
}

int launch_transport(const TransportParams &p, int grid, int block, int threads_per_sm, size_t smem, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (threads_per_sm >= 1024) return launch_transport_t<4>(p, grid, block, smem, s);
    return launch_transport_t<3>(p, grid, block, smem, s);
}

int launch_sample_mu(const float *surf, int n_zeta, int n_e, int e_min, float e, uint64_t seed, uint64_t n,
                     double *out, void *stream)
{
    sample_mu_kernel<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(surf, n_zeta, n_e, e_min, e, seed, n, out);
    return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
}

int launch_eval_math(int fn, const float *x, float *out, size_t n, void *stream)
{
    eval_math_kernel<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(fn, x, out, n);
    return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
}

}  // namespace ctd
