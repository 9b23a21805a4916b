// ctd_transport.cu -- photon transport kernel of the dose engine (sm_103a).
//
// Persistent grid.  Warps claim runs of consecutive histories from a global
// counter, so a warp works on one 1 keV spectrum interval at a time
// (Sec. 2.2.5).  Each warp keeps a queue of source photons in shared memory,
// filled 32 at a time by the whole warp (source sampling, Secs. 2.2.5-2.2.6);
// a lane whose history has ended takes the next photon from the queue.  A lane
// then runs up to flight_cap Woodcock flights against mu_max(E) (Sec. 2.1),
// stopping at a real interaction, which it carries out: photoelectric or
// Compton deposition into the FP64 tally with L2 atomics, polar angle from the
// C or R surface (Secs. 2.2.2-2.2.3), rotation.
//
// One kernel template serves one request (its parameters in the kernel's
// parameter space, its tables in shared memory) and many requests at once (a
// request table in device memory, each photon carrying its request index,
// the union of the requests' material tables in shared memory).
#include "ctd_device.cuh"

namespace ctd {
namespace {

using namespace dev;

struct Photon {
    float x, y, z, ux, uy, uz, e;
    uint64_t h;
    uint32_t step;
    int nreal;
    int r;            // request index (multi-request launches)
};

struct LaneCounts {
    uint32_t n[10];
    unsigned long long e_emitted, e_escaped;   // keV * 2^23
};

__device__ __forceinline__ void clear(LaneCounts &c)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) c.n[i] = 0;
    c.e_emitted = 0;
    c.e_escaped = 0;
}

// Add a lane's counts to a request's totals (energies as 128-bit fixed point).
__device__ __forceinline__ void flush_lane(DeviceCounts *dst, LaneCounts &c)
{
#pragma unroll
    for (int i = 0; i < 10; ++i)
        if (c.n[i]) atomicAdd(&dst->n[i], static_cast<unsigned long long>(c.n[i]));
    if (c.e_emitted) {
        const unsigned long long o = atomicAdd(&dst->e_fix[0], c.e_emitted);
        if (o + c.e_emitted < o) atomicAdd(&dst->e_fix[1], 1ull);
    }
    if (c.e_escaped) {
        const unsigned long long o = atomicAdd(&dst->e_fix[2], c.e_escaped);
        if (o + c.e_escaped < o) atomicAdd(&dst->e_fix[3], 1ull);
    }
    clear(c);
}

// Counts of a lane belong to one request at a time; switching flushes them.
template <bool kMulti>
struct Counter {
    LaneCounts c;
    int owner;
    __device__ __forceinline__ void begin()
    {
        clear(c);
        owner = 0;
    }
    __device__ __forceinline__ LaneCounts &to(const LaunchParams &P, int r)
    {
        if (kMulti && r != owner) {
            flush_lane(P.reqs[owner].counts, c);
            owner = r;
        }
        return c;
    }
};

template <bool kMulti>
__device__ __forceinline__ const RequestDesc &req(const LaunchParams &P, int r)
{
    return kMulti ? P.reqs[r] : P.one;
}

__device__ __forceinline__ int bin_search(const RequestDesc &q, uint64_t local)
{
    // largest bin j with pref[j] <= local
    int lo = 0, hi = q.nbins - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&q.pref[mid]) <= local) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Source photon of local history `local` (global index h) of request q;
// `bin` is a lower bound of its 1 keV interval.  Returns true if the photon
// enters the phantom.
__device__ __forceinline__ bool source(const RequestDesc &q, uint64_t h, uint64_t local, int bin, Photon &ph,
                                       LaneCounts &cnt)
{
    while (bin < q.nbins - 1 && __ldg(&q.pref[bin + 1]) <= local) ++bin;
    const U4 b0 = block(q.seed, h, 0, kStreamSource);
    const float elo = __ldg(&q.bin_lo[bin]), ehi = __ldg(&q.bin_hi[bin]);
    const float e = elo + (ehi - elo) * uni(b0.x);
    cnt.e_emitted += kev_fixed(e);
    float cb = 1.0f, sb = 0.0f;
    if (q.src_kind == CTD_SRC_ARC) {
        if (q.continuous) {
            sincos_turns(q.a0t + q.awt * uni(b0.y), cb, sb);
        } else {
            const uint32_t k =
                static_cast<uint32_t>((static_cast<uint64_t>(b0.y) * static_cast<uint64_t>(q.n_proj)) >> 32);
            cb = __ldg(&q.cb[k]);
            sb = __ldg(&q.sb[k]);
        }
    }
    // uniform in solid angle over the field: uniform point, accepted with cos^3
    const float D = q.D, D2 = q.D2;
    bool accepted = false;
    float uu = 0.0f, vv = 0.0f, qq = 0.0f;
    for (uint32_t t = 1; t <= kMaxTrials; ++t) {
        const U4 b = block(q.seed, h, t, kStreamSource);
        uu = q.ulo + q.uw * uni(b.x);
        vv = q.vlo + q.vw * uni(b.y);
        qq = (D2 + uu * uu) + vv * vv;
        const float c2 = D2 / qq;
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
    const float inv = 1.0f / sqrtf(qq);
    float ux, uy, uz, rx, ry, rz;
    if (q.src_kind == CTD_SRC_ARC) {
        ux = (uu * cb - D * sb) * inv;
        uy = ((-uu) * sb - D * cb) * inv;
        uz = vv * inv;
        rx = D * sb;
        ry = D * cb;
        rz = 0.0f;
    } else {
        ux = uu * inv;
        uy = vv * inv;
        uz = D * inv;
        rx = 0.0f;
        ry = 0.0f;
        rz = -D;
    }
    renorm(ux, uy, uz);
    // entry into the box (slab method); outside is vacuum
    const float t0x = (q.bx0 - rx) / ux, t1x = (q.bx1 - rx) / ux;
    const float t0y = (q.by0 - ry) / uy, t1y = (q.by1 - ry) / uy;
    const float t0z = (q.bz0 - rz) / uz, t1z = (q.bz1 - rz) / uz;
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
    return true;
}

// Site of a real interaction found by a flight
struct Hit {
    size_t idx;       // voxel
    int m;            // row of the tables
    int j;            // energy node
    float te;         // energy fraction
    int type;         // 0 photoelectric, 1 Compton, 2 Rayleigh
    uint32_t rz, rw;  // the step's random words for zeta and phi
};

enum { kEnded = 0, kFictitious = 1, kReal = 2 };

struct Smem {
    const float4 *tab;    // [n_mat][n_e]
    const float *mm;      // [n_e] majorant of a single-request launch
};

// One Woodcock flight (Sec. 2.1): free path against mu_max(E), the move, the
// escape test, the voxel and the interaction type.
template <bool kMulti>
__device__ __forceinline__ int flight(const LaunchParams &P, const RequestDesc &q, const Smem &sm, Photon &ph,
                                      LaneCounts &cnt, Hit &hit)
{
    if (ph.step >= kMaxSteps) {
        cnt.n[kCntAborted]++;
        cnt.e_escaped += kev_fixed(ph.e);
        return kEnded;
    }
    const U4 b = block(q.seed, ph.h, ph.step, kStreamTransport);
    ph.step++;
    cnt.n[kCntSteps]++;
    float te;
    const int n_e = P.sh.n_e;
    const int j = enode(ph.e, P.sh.e_min, n_e, te);
    float m0, m1;
    if (kMulti) {
        m0 = __ldg(&q.mmax[j]);
        m1 = __ldg(&q.mmax[j + 1]);
    } else {
        m0 = sm.mm[j];
        m1 = sm.mm[j + 1];
    }
    const float mmax = m0 + te * (m1 - m0);
    const float path = (-log32(uni(b.x))) / mmax;
    ph.x = ph.x + path * ph.ux;
    ph.y = ph.y + path * ph.uy;
    ph.z = ph.z + path * ph.uz;
    const float fx = (ph.x - q.bx0) * q.ix, fy = (ph.y - q.by0) * q.iy, fz = (ph.z - q.bz0) * q.iz;
    if (!(fx >= 0.0f && fx < static_cast<float>(q.nx) && fy >= 0.0f && fy < static_cast<float>(q.ny) &&
          fz >= 0.0f && fz < static_cast<float>(q.nz))) {
        cnt.n[kCntEscaped]++;
        cnt.e_escaped += kev_fixed(ph.e);
        return kEnded;
    }
    const size_t idx = static_cast<size_t>(static_cast<int>(fx)) +
                       static_cast<size_t>(q.nx) * (static_cast<size_t>(static_cast<int>(fy)) +
                                                    static_cast<size_t>(q.ny) * static_cast<size_t>(static_cast<int>(fz)));
    int m = __ldg(&q.mat[idx]);
    if (kMulti) m = q.mat_map[m];
    const float rho = __ldg(&q.rho[idx]);
    const float4 A = sm.tab[m * n_e + j], B = sm.tab[m * n_e + j + 1];
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
__device__ __forceinline__ bool interact(const LaunchParams &P, const RequestDesc &q, Photon &ph, const Hit &hit,
                                         LaneCounts &cnt)
{
    ph.nreal++;
    if (hit.type == 0) {
        // photoelectric absorption: the electron deposits E here
        cnt.n[kCntPe]++;
        deposit(q.tally, hit.idx, ph.e);
        return false;
    }
    const float *S = hit.type == 1 ? P.sh.csurf : P.sh.rsurf + static_cast<size_t>(hit.m) * P.sh.n_e * P.sh.n_zeta;
    const float mu = surface(S, P.sh.n_zeta, hit.j, hit.te, uni(hit.rz));
    if (hit.type == 1) {
        // Compton: E' = E / (1 + (E/mc^2)(1 - mu)), the electron gets E - E'
        cnt.n[kCntCompton]++;
        const float k = ph.e / static_cast<float>(kMec2);
        const float ep = ph.e / (1.0f + k * (1.0f - mu));
        if (ep < static_cast<float>(P.sh.e_min)) {
            cnt.n[kCntCutoff]++;
            deposit(q.tally, hit.idx, ph.e);
            return false;
        }
        deposit(q.tally, hit.idx, ph.e - ep);
        ph.e = ep;
    } else {
        cnt.n[kCntRayleigh]++;
    }
    if (q.mode == CTD_MODE_MAX_REAL && ph.nreal >= q.max_real) {
        cnt.n[kCntTerminated]++;
        cnt.e_escaped += kev_fixed(ph.e);
        return false;
    }
    rotate(ph.ux, ph.uy, ph.uz, mu, uni(hit.rw));
    return true;
}

// Flights until a real interaction, the escape, or flight_cap flights; then the
// interaction.  Returns false when the history has ended.
template <bool kMulti>
__device__ __forceinline__ bool walk(const LaunchParams &P, const Smem &sm, Photon &ph, LaneCounts &cnt)
{
    const RequestDesc &q = req<kMulti>(P, ph.r);
    Hit hit;
    int f, k = 0;
    do {
        f = flight<kMulti>(P, q, sm, ph, cnt, hit);
    } while (f == kFictitious && ++k < P.flight_cap);
    if (f == kEnded) return false;
    if (f == kFictitious) return true;
    return interact(P, q, ph, hit, cnt);
}

// Per-warp photon queue in shared memory: source photons are made 32 at a
// time by the whole warp and taken by lanes whose history has ended.
constexpr int kQueue = 64;
constexpr size_t kQueueBytes = kQueue * (7 * sizeof(float) + sizeof(uint64_t) + sizeof(int));

template <int kMinBlocks, bool kMulti>
__global__ void __launch_bounds__(256, kMinBlocks) transport_kernel(const LaunchParams P)
{
    extern __shared__ float4 smem[];
    float4 *s_tab = smem;
    const int ntab = P.sh.n_mat * P.sh.n_e;
    float *s_mm = reinterpret_cast<float *>(smem + ntab);
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) s_tab[i] = reinterpret_cast<const float4 *>(P.sh.tab)[i];
    if (!kMulti)
        for (int i = threadIdx.x; i < P.sh.n_e; i += blockDim.x) s_mm[i] = P.one.mmax[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *qbase =
        reinterpret_cast<unsigned char *>(smem + ntab + (kMulti ? 0 : (P.sh.n_e + 3) / 4)) + warp * kQueueBytes;
    uint64_t *qh = reinterpret_cast<uint64_t *>(qbase);
    float *qf = reinterpret_cast<float *>(qh + kQueue);   // [7][kQueue]: x y z ux uy uz e
    int *qr = reinterpret_cast<int *>(qf + 7 * kQueue);
    __syncthreads();
    const Smem sm{s_tab, s_mm};

    const unsigned lt_mask = (1u << lane) - 1u;
    Counter<kMulti> cnt;
    cnt.begin();

    Photon ph;
    ph.r = 0;
    bool alive = false;
    uint64_t pool_next = 0, pool_end = 0;   // warp-uniform claim (multi: over all requests' histories)
    int pool_bin = 0;                       // 1 keV interval of the round's first history
    int pool_req = 0;                       // request of pool_next (multi)
    bool drained = false;
    int qcount = 0;                         // photons waiting in the warp's queue
    const uint64_t range_begin = kMulti ? 0 : P.one.local_begin;
    const uint64_t range_end = kMulti ? P.req_off[P.n_req] : P.one.local_end;
    for (;;) {
        // top the queue up with one round of up to 32 source photons of one request
        if (qcount < 32 && !drained) {
            if (pool_next >= pool_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(P.work, static_cast<unsigned long long>(P.chunk));
                base = __shfl_sync(kFull, base, 0);
                const uint64_t b = range_begin + base;
                if (b >= range_end) {
                    drained = true;
                } else {
                    pool_next = b;
                    pool_end = b + P.chunk < range_end ? b + P.chunk : range_end;
                    if (!kMulti) pool_bin = bin_search(P.one, pool_next);
                }
            }
            if (!drained) {
                uint64_t avail = pool_end - pool_next;
                uint64_t local = pool_next;
                if (kMulti) {
                    // the request holding pool_next; a round stops at its end
                    int lo = 0, hi = P.n_req - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (__ldg(&P.req_off[mid]) <= pool_next) lo = mid;
                        else hi = mid - 1;
                    }
                    pool_req = lo;
                    const uint64_t rend = __ldg(&P.req_off[lo + 1]);
                    if (rend - pool_next < avail) avail = rend - pool_next;
                    local = P.reqs[lo].local_begin + (pool_next - __ldg(&P.req_off[lo]));
                    pool_bin = bin_search(P.reqs[lo], local);
                }
                const unsigned take = avail < 32 ? static_cast<unsigned>(avail) : 32u;
                const RequestDesc &q = req<kMulti>(P, pool_req);
                Photon np;
                bool ok = false;
                if (lane < take) {
                    LaneCounts &c = cnt.to(P, pool_req);
                    ok = source(q, q.h_base + local + lane, local + lane, pool_bin, np, c);
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
                    qr[slot] = pool_req;
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
                ph.r = qr[slot];
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
        if (alive) alive = walk<kMulti>(P, sm, ph, cnt.to(P, ph.r));
    }

    if (kMulti) {
        flush_lane(P.reqs[cnt.owner].counts, cnt.c);
        return;
    }
    // single request: warp sums, one atomic per warp
    LaneCounts &c = cnt.c;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        unsigned long long v = c.n[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
        if (lane == 0 && v) atomicAdd(&P.one.counts->n[i], v);
    }
    unsigned long long em = c.e_emitted, es = c.e_escaped;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        em += __shfl_down_sync(kFull, em, o);
        es += __shfl_down_sync(kFull, es, o);
    }
    if (lane == 0) {
        const unsigned long long o1 = atomicAdd(&P.one.counts->e_fix[0], em);
        if (o1 + em < o1) atomicAdd(&P.one.counts->e_fix[1], 1ull);
        const unsigned long long o2 = atomicAdd(&P.one.counts->e_fix[2], es);
        if (o2 + es < o2) atomicAdd(&P.one.counts->e_fix[3], 1ull);
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

template <int kMinBlocks, bool kMulti>
int launch_t(const LaunchParams &p, int grid, int block, size_t smem, cudaStream_t stream)
{
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(transport_kernel<kMinBlocks, kMulti>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem)) != cudaSuccess)
            return CTD_ECUDA;
    }
    transport_kernel<kMinBlocks, kMulti><<<grid, block, smem, stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
}

}  // namespace

size_t transport_smem_bytes(const LaunchParams &p, int threads)
{
    const bool multi = p.n_req > 0;
    return static_cast<size_t>(p.sh.n_mat) * p.sh.n_e * sizeof(float4) +
           (multi ? 0 : static_cast<size_t>((p.sh.n_e + 3) / 4) * sizeof(float4)) +
           static_cast<size_t>(threads / 32) * kQueueBytes;
}

// The register budget follows the residency asked for: 4 or more blocks of
// 256 threads per SM cap the kernel at 64 registers, fewer at 85.
int launch_transport(const LaunchParams &p, int grid, int block, int threads_per_sm, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = transport_smem_bytes(p, block);
    const bool multi = p.n_req > 0;
    if (threads_per_sm >= 1024)
        return multi ? launch_t<4, true>(p, grid, block, smem, s) : launch_t<4, false>(p, grid, block, smem, s);
    return multi ? launch_t<3, true>(p, grid, block, smem, s) : launch_t<3, false>(p, grid, block, smem, s);
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
