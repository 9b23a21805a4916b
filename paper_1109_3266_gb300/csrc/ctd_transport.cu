// ctd_transport.cu -- photon transport kernel of the dose engine (sm_103a).
//
// Persistent grid.  Warps claim runs of consecutive histories from a global
// counter, so a warp works on one 1 keV spectrum interval at a time
// (Sec. 2.2.5).  Each warp keeps a queue of source photons in shared memory,
// filled 32 at a time by the whole warp (source sampling, Secs. 2.2.4-2.2.6);
// a lane whose history has ended takes the next photon from the queue.  A lane
// then runs up to flight_cap Woodcock flights against mu_max(E) (Sec. 2.1),
// stopping at a real interaction, which it carries out: photoelectric or
// Compton deposition into the FP64 tally as L2 reductions, polar angle from the
// C or R surface (Secs. 2.2.2-2.2.3), rotation and binary64 renormalisation.
// Per-step event counts live in registers, the rest of a lane's counts in its
// shared-memory slot.
//
// One kernel template, four forms: one request without a fluence map, one
// request with one (its source path compiled only there), both with the request
// in the kernel's parameter space; and many requests at once, without or with
// maps (warps walk through a request table, one request at a time, its
// descriptor in shared memory, its tables read through L1).
#include "ctd_device.cuh"

namespace ctd {
namespace {

using namespace dev;

struct Photon {
    float x, y, z;    // position in voxel units: (r - box origin) / voxel size per axis
    float ux, uy, uz, e;
    uint64_t h;
    uint32_t step;
    int j;            // energy node of e, its fraction and 1 / the majorant there;
    float te, imax;   // they change only with e
};

// Philox block of (history, step, stream) of request q: the round keys are
// taken from q when it sits in the kernel's parameter space (kKeys), else
// derived from the seed.
template <bool kKeys>
__device__ __forceinline__ U4 draw(const RequestDesc &q, uint64_t h, uint32_t step, uint32_t stream)
{
    if (kKeys)
        return philox_rk(static_cast<uint32_t>(h), static_cast<uint32_t>(h >> 32), step, stream, q.rk);
    return block(q.seed, h, step, stream);
}

// energy node, fraction and inverse majorant of the photon's energy
__device__ __forceinline__ void set_energy(Photon &ph, const SharedTables &sh, const float *__restrict__ s_mm)
{
    ph.j = enode(ph.e, sh.e_min, sh.n_e, ph.te);
    const float m0 = s_mm[ph.j], m1 = s_mm[ph.j + 1];
    ph.imax = 1.0f / __fmaf_rn(ph.te, m1 - m0, m0);
}

// A lane's once-per-history event counts, energy totals and the real
// interactions of its current photon, in shared memory: they change at most a
// few times per history, and registers are what bounds the kernel's residency.
struct LaneSlot {
    unsigned long long e_emitted, e_escaped;   // keV * 2^23
    uint32_t ev[6];                            // PE, escaped, missed, cutoff, terminated, aborted
    uint32_t nreal;                            // real interactions of the current photon
    uint32_t pad;
};
static_assert(sizeof(LaneSlot) == 48, "LaneSlot layout");

// Event counts of a lane: the per-step events (fictitious, Compton, Rayleigh)
// in registers, the rest in the lane's slot.  Woodcock steps are not counted:
// each ends in exactly one of escape, fictitious, PE, Compton or Rayleigh.
struct LaneCounts {
    uint32_t fict, compton, rayleigh;
    LaneSlot *me;
    __device__ __forceinline__ void clear()
    {
        fict = compton = rayleigh = 0;
        me->e_emitted = 0;
        me->e_escaped = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i) me->ev[i] = 0;
    }
    // k is a constant at every call site, so the switch folds away
    __device__ __forceinline__ void event(int k)
    {
        switch (k) {
        case kCntFict: ++fict; break;
        case kCntCompton: ++compton; break;
        case kCntRayleigh: ++rayleigh; break;
        case kCntPe: ++me->ev[0]; break;
        case kCntEscaped: ++me->ev[1]; break;
        case kCntMissed: ++me->ev[2]; break;
        case kCntCutoff: ++me->ev[3]; break;
        case kCntTerminated: ++me->ev[4]; break;
        default: ++me->ev[5]; break;   // kCntAborted
        }
    }
    __device__ __forceinline__ void emitted(float e) { me->e_emitted += kev_fixed(e); }
    __device__ __forceinline__ void escaped(float e) { me->e_escaped += kev_fixed(e); }
};

// Per-history records of a trace launch (kTrace instantiations only): each
// history writes its own record, so no two lanes write the same one.
struct Tracer {
    uint4 *rec;
    uint64_t h0, n;
    // the last real interaction: its type and voxel
    __device__ __forceinline__ void last(uint64_t h, int type, uint32_t idx) const
    {
        const uint64_t i = h - h0;
        if (i < n) {
            rec[i].x = (rec[i].x & 0xffu) | (static_cast<uint32_t>(type + 1) << 8);
            rec[i].z = idx;
        }
    }
    // how the history ended, its steps and the energy the ending event deposited
    __device__ __forceinline__ void end(uint64_t h, int code, uint32_t steps, float e) const
    {
        const uint64_t i = h - h0;
        if (i < n) {
            rec[i].x = (rec[i].x & 0xff00u) | static_cast<uint32_t>(code + 1);
            rec[i].y = steps;
            rec[i].w = __float_as_uint(e);
        }
    }
};

// A warp's counts added to a request's totals: warp sums, one atomic per
// counter (energies as 128-bit fixed-point totals).  Leaves the counts cleared.
__device__ __forceinline__ void flush_warp(DeviceCounts *dst, LaneCounts &c, int lane)
{
    __syncwarp();
    const LaneSlot &m = *c.me;
    uint32_t v[10];
    v[kCntPe] = m.ev[0];
    v[kCntCompton] = c.compton;
    v[kCntRayleigh] = c.rayleigh;
    v[kCntFict] = c.fict;
    v[kCntEscaped] = m.ev[1];
    v[kCntMissed] = m.ev[2];
    v[kCntCutoff] = m.ev[3];
    v[kCntTerminated] = m.ev[4];
    v[kCntAborted] = m.ev[5];
    v[kCntSteps] = m.ev[1] + c.fict + m.ev[0] + c.compton + c.rayleigh;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        unsigned long long x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
        if (lane == 0 && x) atomicAdd(&dst->n[i], x);
    }
    unsigned long long em = m.e_emitted, es = m.e_escaped;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        em += __shfl_down_sync(kFull, em, o);
        es += __shfl_down_sync(kFull, es, o);
    }
    if (lane == 0) {
        const unsigned long long o1 = atomicAdd(&dst->e_fix[0], em);
        if (o1 + em < o1) atomicAdd(&dst->e_fix[1], 1ull);
        const unsigned long long o2 = atomicAdd(&dst->e_fix[2], es);
        if (o2 + es < o2) atomicAdd(&dst->e_fix[3], 1ull);
    }
    c.clear();
    __syncwarp();
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
template <bool kKeys, bool kFluence, bool kTrace>
__device__ __forceinline__ bool source(const RequestDesc &q, uint64_t h, uint64_t local, int bin, Photon &ph,
                                       LaneCounts &cnt, const Tracer &tr)
{
    while (bin < q.nbins - 1 && __ldg(&q.pref[bin + 1]) <= local) ++bin;
    const U4 b0 = draw<kKeys>(q, h, 0, kStreamSource);
    const float elo = __ldg(&q.bin_lo[bin]), ehi = __ldg(&q.bin_hi[bin]);
    const float e = __fmaf_rn(ehi - elo, uni(b0.x), elo);
    cnt.emitted(e);
    float cb = 1.0f, sb = 0.0f, zs = 0.0f;
    if (q.src_kind == CTD_SRC_ARC) {
        if (q.continuous) {
            // the angle in turns, reduced to [0, 1) (arcs may span several turns)
            const float turns = __fmaf_rn(q.awt, uni(b0.y), q.a0t);
            sincos_turns(turns - floorf(turns), cb, sb);
            zs = __fmaf_rn(q.hdz, uni(b0.y), q.hz0);
        } else {
            const uint32_t k =
                static_cast<uint32_t>((static_cast<uint64_t>(b0.y) * static_cast<uint64_t>(q.n_proj)) >> 32);
            cb = __ldg(&q.cb[k]);
            sb = __ldg(&q.sb[k]);
            zs = __ldg(&q.zb[k]);
        }
    }
    // uniform in solid angle over the field: uniform point, accepted with cos^3;
    // with a fluence map (Sec. 2.2.4): beamlet from the alias table, point uniform in it
    const float D = q.D, D2 = q.D2;
    bool accepted = false;
    float uu = 0.0f, vv = 0.0f, qq = 0.0f;
    if (kFluence && q.fl_n > 0) {
        const U4 b = draw<kKeys>(q, h, 1, kStreamSource);
        const uint32_t k =
            static_cast<uint32_t>((static_cast<uint64_t>(b.x) * static_cast<uint64_t>(static_cast<uint32_t>(q.fl_n))) >> 32);
        const uint32_t beam = b.y < __ldg(&q.fl_thr[k]) ? k : static_cast<uint32_t>(__ldg(&q.fl_alias[k]));
        const uint32_t iv = static_cast<uint32_t>((static_cast<uint64_t>(beam) * q.fl_magic) >> 40);
        const uint32_t iu = beam - iv * static_cast<uint32_t>(q.fl_nu);
        uu = __fmaf_rn(q.fl_du, static_cast<float>(iu) + uni(b.z), q.ulo);
        vv = __fmaf_rn(q.fl_dv, static_cast<float>(iv) + uni(b.w), q.vlo);
        qq = __fmaf_rn(vv, vv, __fmaf_rn(uu, uu, D2));
        accepted = true;
    }
    for (uint32_t t = 1; t <= kMaxTrials && !accepted; ++t) {
        const U4 b = draw<kKeys>(q, h, t, kStreamSource);
        uu = __fmaf_rn(q.uw, uni(b.x), q.ulo);
        vv = __fmaf_rn(q.vw, uni(b.y), q.vlo);
        qq = __fmaf_rn(vv, vv, __fmaf_rn(uu, uu, D2));
        const float c2 = D2 / qq;
        const float acc = c2 * sqrtf(c2);
        if (uni(b.z) < acc) {
            accepted = true;
            break;
        }
    }
    if (!accepted) {
        cnt.event(kCntAborted);
        cnt.escaped(e);
        if (kTrace) tr.end(h, kEndAborted, 0, 0.0f);
        return false;
    }
    const float inv = 1.0f / sqrtf(qq);
    float ux, uy, uz, rx, ry, rz;
    if (q.src_kind == CTD_SRC_ARC) {
        ux = __fmaf_rn(uu, cb, -(D * sb)) * inv;
        uy = __fmaf_rn(-uu, sb, -(D * cb)) * inv;
        uz = vv * inv;
        rx = D * sb;
        ry = D * cb;
        rz = zs;
    } else {
        ux = uu * inv;
        uy = vv * inv;
        uz = D * inv;
        rx = 0.0f;
        ry = 0.0f;
        rz = -D;
    }
    // (the source direction is normalised in binary32; binary64 renormalisation
    // is for the directions made by scatters)
    // entry into the box (slab method, with the direction's reciprocals); outside is vacuum
    const float iux = 1.0f / ux, iuy = 1.0f / uy, iuz = 1.0f / uz;
    const float t0x = (q.bx0 - rx) * iux, t1x = (q.bx1 - rx) * iux;
    const float t0y = (q.by0 - ry) * iuy, t1y = (q.by1 - ry) * iuy;
    const float t0z = (q.bz0 - rz) * iuz, t1z = (q.bz1 - rz) * iuz;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fminf(t0z, t1z));
    const float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fmaxf(t0z, t1z));
    if (!(tn < tf) || !(tf > 0.0f)) {
        cnt.event(kCntMissed);
        cnt.escaped(e);
        if (kTrace) tr.end(h, kEndMissed, 0, 0.0f);
        return false;
    }
    if (tn < 0.0f) tn = 0.0f;
    // the entry point in voxel units, clamped into the box (it lies on the box's
    // surface; rounding can leave it just outside): [0, the number below n]
    ph.x = fminf(fmaxf((__fmaf_rn(tn, ux, rx) - q.bx0) * q.ix, 0.0f), __uint_as_float(__float_as_uint(q.fnx) - 1u));
    ph.y = fminf(fmaxf((__fmaf_rn(tn, uy, ry) - q.by0) * q.iy, 0.0f), __uint_as_float(__float_as_uint(q.fny) - 1u));
    ph.z = fminf(fmaxf((__fmaf_rn(tn, uz, rz) - q.bz0) * q.iz, 0.0f), __uint_as_float(__float_as_uint(q.fnz) - 1u));
    ph.ux = ux;
    ph.uy = uy;
    ph.uz = uz;
    ph.e = e;
    ph.h = h;
    return true;
}

// Site of a real interaction found by a flight
struct Hit {
    uint32_t idx;     // voxel (phantoms hold fewer than 2^32 voxels)
    int m;            // material
    int type;         // 0 photoelectric, 1 Compton, 2 Rayleigh
    uint32_t rz, rw;  // the step's random words for zeta and phi
};

enum { kEscaped = 0, kFictitious = 1, kReal = 2 };

// One Woodcock flight (Sec. 2.1): free path against mu_max(E), the move, the
// escape test, the voxel and the interaction type.  s_tab is the request's
// attenuation table in shared memory.  An escape is counted by the caller,
// outside the loop of flights, and the caller keeps ph.step below kMaxSteps
// (the history's step limit).
template <bool kKeys>
__device__ __forceinline__ int flight(const SharedTables &sh, const RequestDesc &q, const float4 *__restrict__ s_tab,
                                      Photon &ph, LaneCounts &cnt, Hit &hit)
{
    const U4 b = draw<kKeys>(q, ph.h, ph.step, kStreamTransport);
    ph.step++;
    const int n_e = sh.n_e;
    const int j = ph.j;
    const float te = ph.te, imax = ph.imax;
    const float path = (-log32(uni(b.x))) * imax;
    // the move in voxel units: each displacement s u_k times 1/d_k, added fused
    ph.x = __fmaf_rn(path * ph.ux, q.ix, ph.x);
    ph.y = __fmaf_rn(path * ph.uy, q.iy, ph.y);
    ph.z = __fmaf_rn(path * ph.uz, q.iz, ph.z);
    const float fx = ph.x, fy = ph.y, fz = ph.z;
    // 0 <= f < n on each axis, as one unsigned compare of the bit patterns: for
    // floats other than -0 it is the same test (negative floats and NaNs have the
    // sign bit or an all-ones exponent, so larger patterns than n), and a position
    // is never -0 (the entry point is clamped to +0 at least, and adding a nonzero
    // or +0 displacement to a value other than -0 never gives -0)
    if (!(__float_as_uint(fx) < __float_as_uint(q.fnx) && __float_as_uint(fy) < __float_as_uint(q.fny) &&
          __float_as_uint(fz) < __float_as_uint(q.fnz)))
        return kEscaped;
    const uint32_t idx = static_cast<uint32_t>(static_cast<int>(fx)) +
                         static_cast<uint32_t>(q.nx) *
                             (static_cast<uint32_t>(static_cast<int>(fy)) +
                              static_cast<uint32_t>(q.ny) * static_cast<uint32_t>(static_cast<int>(fz)));
    // one gather: the material in the top 4 bits, the density's exponent rebased
    const uint32_t w = __ldg(&q.vox[idx]);
    const int m = static_cast<int>(w >> 28);
    const uint32_t rb = w & 0x0fffffffu;
    const float rho = rb ? __uint_as_float(rb + (kRhoExpBias << 23)) : 0.0f;
    // interaction type with probabilities mu_i / mu_max: fictitious when u1 is at or
    // above the total share; otherwise the first cumulative share above u1.  The
    // table's fourth column is the total share's node difference, so a fictitious
    // step reads one node; a real one reads the next node's c1 and c2 as well.
    const float4 A = s_tab[m * n_e + j];
    const float y = uni(b.y);
    const float sr = rho * imax;
    const float c3 = __fmaf_rn(te, A.w, A.z);
    if (!(y < sr * c3)) {
        cnt.event(kCntFict);
        return kFictitious;
    }
    const float2 B = *reinterpret_cast<const float2 *>(&s_tab[m * n_e + j + 1]);
    const float c1 = __fmaf_rn(te, B.x - A.x, A.x);
    const float c2 = __fmaf_rn(te, B.y - A.y, A.y);
    int type;
    if (y < sr * c1) type = 0;
    else if (y < sr * c2) type = 1;
    else type = 2;
    hit.idx = idx;
    hit.m = m;
    hit.type = type;
    hit.rz = b.z;
    hit.rw = b.w;
    return kReal;
}

// A real interaction: local deposition, C/R-surface polar angle, rotation.
// Returns false when the history has ended.
template <bool kTrace>
__device__ __forceinline__ bool interact(const SharedTables &sh, const RequestDesc &q, const float *__restrict__ s_mm,
                                         Photon &ph, const Hit &hit, LaneCounts &cnt, const Tracer &tr)
{
    if (kTrace) tr.last(ph.h, hit.type, hit.idx);
    if (hit.type == 0) {
        // photoelectric absorption: the electron deposits E here
        cnt.event(kCntPe);
        deposit(q.tally, hit.idx, ph.e);
        if (kTrace) tr.end(ph.h, kEndPe, ph.step, ph.e);
        return false;
    }
    const float *S = hit.type == 1
                         ? q.csurf + static_cast<size_t>(hit.m) * q.cs_stride * 4
                         : q.rsurf + static_cast<size_t>(hit.m) * (sh.n_e - 1) * (sh.n_zeta - 1) * 4;
    const float mu = surface(S, sh.n_zeta, ph.j, ph.te, uni(hit.rz));
    if (hit.type == 1) {
        // Compton: E' = E / (1 + (E/mc^2)(1 - mu)), the electron gets E - E'
        cnt.event(kCntCompton);
        const float k = ph.e * static_cast<float>(1.0 / kMec2);
        const float ep = ph.e / __fmaf_rn(k, 1.0f - mu, 1.0f);
        if (ep < static_cast<float>(sh.e_min)) {
            cnt.event(kCntCutoff);
            deposit(q.tally, hit.idx, ph.e);
            if (kTrace) tr.end(ph.h, kEndCutoff, ph.step, ph.e);
            return false;
        }
        deposit(q.tally, hit.idx, ph.e - ep);
        if (kTrace) tr.end(ph.h, kEndTerminated, ph.step, ph.e - ep);   // kept if the history ends here
        ph.e = ep;
        set_energy(ph, sh, s_mm);
    } else {
        cnt.event(kCntRayleigh);
        if (kTrace) tr.end(ph.h, kEndTerminated, ph.step, 0.0f);
    }
    if (q.mode == CTD_MODE_MAX_REAL && ++cnt.me->nreal >= static_cast<uint32_t>(q.max_real)) {
        cnt.event(kCntTerminated);
        cnt.escaped(ph.e);
        return false;
    }
    rotate(ph.ux, ph.uy, ph.uz, mu, uni(hit.rw));
    return true;
}

// Per-warp photon queue in shared memory: source photons are made 32 at a
// time by the whole warp and taken by lanes whose history has ended.
constexpr int kQueue = 64;
constexpr size_t kQueueBytes = kQueue * (7 * sizeof(float) + sizeof(uint64_t));

// A warp's claim of local history indices [next, end) and the 1 keV interval
// of its first history, kept in shared memory (read only when the queue is
// topped up).
struct WarpPool {
    uint64_t next, end;
    int bin;
    int pad[3];
};

struct Queue {
    uint64_t *h;
    float *f;   // [7][kQueue]: x y z (voxel units) ux uy uz e
    WarpPool *pool;
};

constexpr size_t kWarpBytes = kQueueBytes + sizeof(WarpPool) + 32 * sizeof(LaneSlot);
static_assert(kWarpBytes % 16 == 0, "a warp's shared-memory area must keep 16-byte alignment");

// All histories [q.local_begin, q.local_end) of one request, claimed by warps
// from q.work in runs of `chunk`.  Returns when the warp has no photon left.
template <bool kKeys, bool kFluence, bool kTrace>
__device__ __forceinline__ void run_request(const LaunchParams &P, const RequestDesc &q, const float4 *s_tab,
                                            const float *s_mm, const Queue &Q, int lane, LaneCounts &cnt)
{
    Tracer tr;
    tr.rec = P.trace;
    tr.h0 = P.trace_h0;
    tr.n = kTrace ? P.trace_n : 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    Photon ph;
    bool alive = false;
    bool drained = false;
    int qcount = 0;                         // photons waiting in the warp's queue
    if (lane == 0) {
        Q.pool->next = 0;
        Q.pool->end = 0;
        Q.pool->bin = 0;
    }
    __syncwarp();
    for (;;) {
        // top the queue up with one round of up to 32 source photons
        if (qcount < 32 && !drained) {
            uint64_t pool_next = Q.pool->next, pool_end = Q.pool->end;
            int pool_bin = Q.pool->bin;
            if (pool_next >= pool_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(q.work, static_cast<unsigned long long>(P.chunk));
                base = __shfl_sync(kFull, base, 0);
                const uint64_t b = q.local_begin + base;
                if (b >= q.local_end) {
                    drained = true;
                } else {
                    pool_next = b;
                    pool_end = b + P.chunk < q.local_end ? b + P.chunk : q.local_end;
                    pool_bin = bin_search(q, pool_next);
                }
            }
            if (!drained) {
                const uint64_t avail = pool_end - pool_next;
                const unsigned take = avail < 32 ? static_cast<unsigned>(avail) : 32u;
                Photon np;
                bool ok = false;
                if (lane < take) {
                    const uint64_t local = pool_next + lane;
                    ok = source<kKeys, kFluence, kTrace>(q, q.h_base + local, local, pool_bin, np, cnt, tr);
                }
                const unsigned okm = __ballot_sync(kFull, ok);
                if (ok) {
                    const int slot = qcount + __popc(okm & lt_mask);
                    Q.h[slot] = np.h;
                    Q.f[0 * kQueue + slot] = np.x;
                    Q.f[1 * kQueue + slot] = np.y;
                    Q.f[2 * kQueue + slot] = np.z;
                    Q.f[3 * kQueue + slot] = np.ux;
                    Q.f[4 * kQueue + slot] = np.uy;
                    Q.f[5 * kQueue + slot] = np.uz;
                    Q.f[6 * kQueue + slot] = np.e;
                }
                qcount += __popc(okm);
                pool_next += take;
            }
            __syncwarp();
            if (lane == 0) {
                Q.pool->next = pool_next;
                Q.pool->end = pool_end;
                Q.pool->bin = pool_bin;
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
                ph.h = Q.h[slot];
                ph.x = Q.f[0 * kQueue + slot];
                ph.y = Q.f[1 * kQueue + slot];
                ph.z = Q.f[2 * kQueue + slot];
                ph.ux = Q.f[3 * kQueue + slot];
                ph.uy = Q.f[4 * kQueue + slot];
                ph.uz = Q.f[5 * kQueue + slot];
                ph.e = Q.f[6 * kQueue + slot];
                ph.step = 0;
                cnt.me->nreal = 0;
                set_energy(ph, P.sh, s_mm);
                alive = true;
            }
        }
        qcount -= npop;
        __syncwarp();
        if (!__any_sync(kFull, alive)) {
            if (drained && qcount == 0) break;
            continue;
        }
        if (alive) {
            // flights until a real interaction, the escape or flight_cap flights; then the
            // interaction.  A run stops short of the history's step limit; a history that
            // has reached it is aborted when its next run would start.
            const uint32_t room = kMaxSteps - ph.step;
            const int lim = room < static_cast<uint32_t>(P.flight_cap) ? static_cast<int>(room) : P.flight_cap;
            if (lim == 0) {
                cnt.event(kCntAborted);
                cnt.escaped(ph.e);
                if (kTrace) tr.end(ph.h, kEndAborted, ph.step, 0.0f);
                alive = false;
            } else {
                Hit hit;
                int f, k = 0;
                do {
                    f = flight<kKeys>(P.sh, q, s_tab, ph, cnt, hit);
                } while (f == kFictitious && ++k < lim);
                if (f == kEscaped) {
                    cnt.event(kCntEscaped);
                    cnt.escaped(ph.e);
                    if (kTrace) tr.end(ph.h, kEndEscaped, ph.step, 0.0f);
                    alive = false;
                } else if (f == kReal) {
                    alive = interact<kTrace>(P.sh, q, s_mm, ph, hit, cnt, tr);
                }
            }
        }
    }
}

__device__ __forceinline__ void load_tables(const RequestDesc &q, int n_e, float4 *s_tab, float *s_mm)
{
    const int ntab = q.n_mat * n_e;
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) s_tab[i] = reinterpret_cast<const float4 *>(q.tab)[i];
    for (int i = threadIdx.x; i < n_e; i += blockDim.x) s_mm[i] = q.mmax[i];
}

// Single request (kForm 0 or 1): the request lives in the kernel's parameter
// space, its attenuation table and majorant are copied into shared memory.
// Several requests: each warp works on one request at a time with a copy of its
// descriptor in shared memory and its tables read through L1, and when that
// request has no history left to claim the warp moves on to the next one by
// itself, so that one request's tail overlaps the next one's start without the
// block waiting for its slowest warp.
// kForm: 0 one request without a fluence map, 1 one request with a fluence map
// (the map's source path is compiled only into this form, so that it does not
// cost the open-field form registers), 2 several requests without maps, 3 several
// requests of which some have a map (checked per request).  The multi-request
// forms take each request's Philox round keys from its descriptor in shared
// memory.
// kTrace (single-request forms): also write each history's record to P.trace.
constexpr int kReqWords = sizeof(RequestDesc) / 16;

template <int kMaxThreads, int kMinBlocks, int kForm, bool kTrace = false>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) transport_kernel(const LaunchParams P)
{
    extern __shared__ float4 smem[];
    const int n_e = P.sh.n_e;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool kMulti = kForm >= 2;
    // single: the tables, then the warps' queues; several: per warp, a descriptor and
    // the queue
    float4 *s_tab = smem;
    float *s_mm = reinterpret_cast<float *>(smem + P.sh.max_n_mat * n_e);
    float4 *w_req4 = smem + warp * (kReqWords + kWarpBytes / 16);
    unsigned char *wbase = kMulti ? reinterpret_cast<unsigned char *>(w_req4 + kReqWords)
                                  : reinterpret_cast<unsigned char *>(smem + P.sh.max_n_mat * n_e + (n_e + 3) / 4) +
                                        warp * kWarpBytes;
    Queue Q;
    Q.h = reinterpret_cast<uint64_t *>(wbase);
    Q.f = reinterpret_cast<float *>(Q.h + kQueue);
    Q.pool = reinterpret_cast<WarpPool *>(wbase + kQueueBytes);
    LaneCounts cnt;
    cnt.me = reinterpret_cast<LaneSlot *>(wbase + kQueueBytes + sizeof(WarpPool)) + lane;
    cnt.clear();

    if (!kMulti) {
        load_tables(P.one, n_e, s_tab, s_mm);
        __syncthreads();
        run_request<true, kForm == 1, kTrace>(P, P.one, s_tab, s_mm, Q, lane, cnt);
        flush_warp(P.one.counts, cnt, lane);
        return;
    }
    // every warp starts at the first request and walks forward to the next request
    // with histories left, so that the warps of an SM mostly work on one request
    // (its phantom and tally stay in L2) and a request's tail overlaps the next one's
    // start
    const RequestDesc &q = *reinterpret_cast<const RequestDesc *>(w_req4);
    int r = 0;
    for (;;) {
        int found = -1;
        if (lane == 0) {
            for (int rr = r; rr < P.n_req; ++rr) {
                const RequestDesc &c = P.reqs[rr];
                const unsigned long long claimed = *reinterpret_cast<volatile unsigned long long *>(c.work);
                if (c.local_begin + claimed < c.local_end) {
                    found = rr;
                    break;
                }
            }
        }
        found = __shfl_sync(kFull, found, 0);
        if (found < 0) break;
        const float4 *src = reinterpret_cast<const float4 *>(P.reqs + found);
        for (int i = lane; i < kReqWords; i += 32) w_req4[i] = src[i];
        __syncwarp();
        run_request<true, kForm == 3, false>(P, q, reinterpret_cast<const float4 *>(q.tab), q.mmax, Q, lane, cnt);
        flush_warp(q.counts, cnt, lane);
        __syncwarp();
        // the same request is exhausted now; continue the walk from it
        r = found;
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
        } else if (fn == 2) {
            out[i] = uni(__float_as_uint(x[i]));
        } else {
            float c, s;
            sincos_turns(x[i], c, s);
            out[2 * i] = c;
            out[2 * i + 1] = s;
        }
    }
}

template <int kMaxThreads, int kMinBlocks, int kForm, bool kTrace = false>
int launch_t(const LaunchParams &p, int grid, int block, size_t smem, cudaStream_t stream,
             const L2Window *win = nullptr)
{
    auto *k = transport_kernel<kMaxThreads, kMinBlocks, kForm, kTrace>;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
            return CTD_ECUDA;
    }
    if (!win) {
        k<<<grid, block, smem, stream>>>(p);
        return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
    }
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeAccessPolicyWindow;
    attr.val.accessPolicyWindow.base_ptr = win->base;
    attr.val.accessPolicyWindow.num_bytes = win->bytes;
    attr.val.accessPolicyWindow.hitRatio = win->hit_ratio;
    attr.val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr.val.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k, p) != cudaSuccess) return CTD_ECUDA;
    return cudaGetLastError() == cudaSuccess ? CTD_OK : CTD_ECUDA;
}

template <int kForm>
int launch_m(const LaunchParams &p, int grid, int block, int threads_per_sm, size_t smem, cudaStream_t s,
             const L2Window *win)
{
    // the register budget follows the residency asked for (65536 registers per SM)
    if (block <= 128 && threads_per_sm >= 896) return launch_t<128, 7, kForm>(p, grid, block, smem, s, win);
    if (threads_per_sm >= 1024) return launch_t<256, 4, kForm>(p, grid, block, smem, s, win);
    return launch_t<256, 3, kForm>(p, grid, block, smem, s, win);
}

}  // namespace

size_t transport_smem_bytes(const LaunchParams &p, int threads)
{
    // several requests: per warp, a descriptor and the queue
    if (p.n_req > 0) return static_cast<size_t>(threads / 32) * (kReqWords * sizeof(float4) + kWarpBytes);
    return (static_cast<size_t>(p.sh.max_n_mat) * p.sh.n_e + (p.sh.n_e + 3) / 4) * sizeof(float4) +
           static_cast<size_t>(threads / 32) * kWarpBytes;
}

// persistent grids: a few blocks per SM
constexpr int kMaxGrid = 1 << 16;

// Kernel variants by residency: 4 blocks of 256 threads per SM cap it at 64
// registers, 7 blocks of 128 at 73, fewer at 85.
int launch_transport(const LaunchParams &p, int grid, int block, int threads_per_sm, void *stream,
                     const L2Window *win)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid <= 0 || grid > kMaxGrid || block <= 0 || block > 256 || block % 32 != 0) {
        set_error("transport launch shape out of range");
        return CTD_EINVAL;
    }
    const size_t smem = transport_smem_bytes(p, block);
    if (p.trace) {
        // trace launches (validation): one instantiation per source form, at 64 registers
        if (p.n_req > 0) {
            set_error("trace launches take one request");
            return CTD_EINVAL;
        }
        return p.one.fl_n > 0 ? launch_t<256, 4, 1, true>(p, grid, block, smem, s)
                              : launch_t<256, 4, 0, true>(p, grid, block, smem, s);
    }
    if (p.n_req > 0) return p.any_fluence ? launch_m<3>(p, grid, block, threads_per_sm, smem, s, win)
                                           : launch_m<2>(p, grid, block, threads_per_sm, smem, s, win);
    return p.one.fl_n > 0 ? launch_m<1>(p, grid, block, threads_per_sm, smem, s, win)
                          : launch_m<0>(p, grid, block, threads_per_sm, smem, s, win);
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
