// ctd_capi.cu -- the C ABI of include/ctd.h: contexts, resident phantoms,
// source/spectrum/physics set-up, the batch loop of Sec. 2.2.1 and results.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ctd_internal.h"

namespace {

thread_local std::string g_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(CTD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

#define CKS(call)                                                                                         \
    do {                                                                                                  \
        int s_ = (call);                                                                                  \
        if (s_ != CTD_OK) {                                                                               \
            if (g_error.empty()) fail(s_, "%s failed: %s", #call, cudaGetErrorString(cudaGetLastError())); \
            return s_;                                                                                    \
        }                                                                                                 \
    } while (0)

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    int ensure(size_t count)
    {
        if (count <= n && p) return CTD_OK;
        release();
        if (count == 0) count = 1;
        if (cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(CTD_ENOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
        }
        n = count;
        return CTD_OK;
    }
};

struct Phantom {
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dy = 0, dz = 0;
    size_t nvox = 0;
    std::vector<ctd_material> mats;
    std::vector<double> rho_max;
    std::vector<int> present;
    ctd_physics phys{};
    ctd_source src{};
    bool has_src = false;
    std::vector<double> e_lo, e_hi, w;
    bool has_spec = false;

    DevBuf<uint8_t> mat;
    DevBuf<float> rho;
    // tables
    bool tables_ok = false;
    int n_e = 0;
    std::vector<float> h_tab, h_mm, h_cs, h_rs;
    DevBuf<float> tab, mm, cs, rs;
    // per-run state
    DevBuf<double> tally, sum_d, sum_d2, edep, dose, sd, partials, result;
    DevBuf<ctd::DeviceCounts> counts;
    DevBuf<unsigned long long> work;
    DevBuf<uint64_t> pref;     // [2][nbins+1]: batch of n_lo+1, batch of n_lo
    DevBuf<float> bins;        // [2][nbins]: lo, hi
    DevBuf<float> proj;        // [2][n_proj]: cos, sin
    uint64_t alloc_n = ~0ull;
    int alloc_nb = -1;
    ctd_run_stats stats{};
    bool have_result = false;
    int64_t busy_req = 0;      // served request using this phantom, 0 if none
    // fluence map (Sec. 2.2.4): alias table over fl_nu x fl_nv beamlets (fl_nu = 0: none)
    int fl_nu = 0, fl_nv = 0;
    std::vector<uint32_t> h_thr;
    std::vector<int32_t> h_alias;
    DevBuf<uint32_t> fl_thr;
    DevBuf<int32_t> fl_alias;
};

struct Staged {
    ctd::DeviceCounts c;
    double res[4];    // avg RSD, sigma_bar, D_max, deposited energy
};

struct ServeReq {
    int64_t id = 0;
    int ph = 0;
    ctd_request req{};
    int state = CTD_REQ_QUEUED;
    int batches = 0;
    uint64_t histories = 0;
    double avg_rsd = 0.0, sigma_bar = 0.0;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    bool cancel = false;
};

}  // namespace

namespace ctd {
void set_error(const char *msg) { g_error = msg; }
}  // namespace ctd

struct ctd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int blocks_per_sm = 4;
    int multi_blocks_per_sm = 3;   // multi-request launches hold more state per lane
    int threads = 256;
    int chunk = 256;
    int flight_cap = 4;
    std::map<int, std::unique_ptr<Phantom>> phantoms;
    int next_id = 1;
    std::vector<cudaEvent_t> events;
    // multi-request launches: request and fold descriptors, claim counters
    DevBuf<ctd::RequestDesc> u_reqs;
    DevBuf<uint64_t> u_tiles;
    DevBuf<ctd::FoldDesc> u_folds;
    DevBuf<unsigned long long> u_work;
    // served form: all requests by id, the admission queue and the running set
    std::map<int64_t, ServeReq> sreqs;
    std::vector<int64_t> pending, active;
    int64_t next_req = 1;
    int max_active = 64;
    double round_histories = 1e8;   // admission stops once a round would exceed this
    // batched form: the captured batch loop and what it was captured for
    cudaGraphExec_t batch_graph = nullptr;
    std::vector<unsigned char> batch_graph_key;
    cudaStream_t capture_stream = nullptr;
    double reserve_bytes = 1.0 * (1ull << 30);
    // batched and served forms: 0 runs each request as its own chain of
    // single-request launches on its own stream (the device overlaps the chains),
    // 1 shares one multi-request launch per batch among all requests
    int shared_launch = 0;
    Staged *staged = nullptr;      // pinned read-back of counts and results
    size_t staged_n = 0;
    // angular surfaces by (kind, q0, e_min, n_e, n_zeta): they do not depend on the phantom
    std::map<std::array<double, 5>, std::vector<float>> surfaces;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fork_event = nullptr;
};

namespace {

constexpr int kRsdParts = 1024;

int use_device(ctd_ctx *ctx)
{
    if (!ctx) return fail(CTD_EINVAL, "null context");
    g_error.clear();
    CK(cudaSetDevice(ctx->device));
    return CTD_OK;
}

Phantom *find(ctd_ctx *ctx, ctd_phantom id)
{
    auto it = ctx->phantoms.find(id);
    return it == ctx->phantoms.end() ? nullptr : it->second.get();
}

int busy(Phantom *P)
{
    return P->busy_req ? fail(CTD_EBUSY, "phantom is in use by served request %lld",
                              static_cast<long long>(P->busy_req))
                       : CTD_OK;
}

// Klein-Nishina C (kind 0), Rayleigh R (kind 1, form-factor width q0) or
// Waller-Hartree C (kind 2, scattering-function width q0) surface in binary32,
// built once per context and node grid.
const std::vector<float> &angular_surface(ctd_ctx *ctx, int kind, double q0, int e_min, int n_e, int n_zeta)
{
    const std::array<double, 5> key{static_cast<double>(kind), kind ? (q0 > 0.0 ? q0 : 0.0) : 0.0,
                                    static_cast<double>(e_min), static_cast<double>(n_e), static_cast<double>(n_zeta)};
    auto it = ctx->surfaces.find(key);
    if (it != ctx->surfaces.end()) return it->second;
    if (ctx->surfaces.size() >= 64) ctx->surfaces.clear();
    const size_t row = static_cast<size_t>(n_e) * n_zeta;
    std::vector<double> tmp(row);
    ctd::build_surface(kind, q0, e_min, n_e, n_zeta, tmp.data());
    std::vector<float> f(row);
    for (size_t i = 0; i < row; ++i) f[i] = static_cast<float>(tmp[i]);
    return ctx->surfaces.emplace(key, std::move(f)).first->second;
}

int build_tables(ctd_ctx *ctx, Phantom &P)
{
    if (P.tables_ok) return CTD_OK;
    const ctd_physics &ph = P.phys;
    const int n_e = ph.e_max_kev - ph.e_min_kev + 1;
    const int nm = static_cast<int>(P.mats.size());
    std::vector<double> cum, mmax;
    ctd::build_tables(P.mats, P.rho_max, P.present, ph.e_min_kev, n_e, ph.majorant_scale, ph.compton_model, cum,
                      mmax);
    P.h_tab.assign(static_cast<size_t>(nm) * n_e * 4, 0.0f);
    for (size_t i = 0; i < static_cast<size_t>(nm) * n_e; ++i)
        for (int c = 0; c < 3; ++c) P.h_tab[i * 4 + c] = static_cast<float>(cum[i * 3 + c]);
    P.h_mm.resize(n_e);
    for (int j = 0; j < n_e; ++j) P.h_mm[j] = static_cast<float>(mmax[j]);
    const size_t row = static_cast<size_t>(n_e) * ph.n_zeta;
    if (ph.compton_model == CTD_COMPTON_WH) {
        // one Waller-Hartree C surface per material
        P.h_cs.resize(row * nm);
        for (int m = 0; m < nm; ++m) {
            const std::vector<float> &c = angular_surface(ctx, 2, P.mats[m].sq0, ph.e_min_kev, n_e, ph.n_zeta);
            std::copy(c.begin(), c.end(), P.h_cs.begin() + m * row);
        }
    } else {
        P.h_cs = angular_surface(ctx, 0, 0.0, ph.e_min_kev, n_e, ph.n_zeta);
    }
    P.h_rs.resize(row * nm);
    for (int m = 0; m < nm; ++m) {
        const std::vector<float> &r = angular_surface(ctx, 1, P.mats[m].q0, ph.e_min_kev, n_e, ph.n_zeta);
        std::copy(r.begin(), r.end(), P.h_rs.begin() + m * row);
    }
    int rc;
    if ((rc = P.tab.ensure(P.h_tab.size())) || (rc = P.mm.ensure(n_e)) || (rc = P.cs.ensure(P.h_cs.size())) ||
        (rc = P.rs.ensure(row * nm)))
        return rc;
    CK(cudaMemcpyAsync(P.tab.p, P.h_tab.data(), P.h_tab.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P.mm.p, P.h_mm.data(), n_e * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P.cs.p, P.h_cs.data(), P.h_cs.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P.rs.p, P.h_rs.data(), row * nm * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    P.n_e = n_e;
    P.tables_ok = true;
    return CTD_OK;
}

// stratified allocation for batches of n_lo + 1 and n_lo histories (Sec. 2.2.5)
int upload_allocation(ctd_ctx *ctx, Phantom &P, uint64_t n, int nb)
{
    if (P.alloc_n == n && P.alloc_nb == nb) return CTD_OK;
    const int nbins = static_cast<int>(P.w.size());
    const uint64_t n_lo = n / static_cast<uint64_t>(nb);
    std::vector<uint64_t> pref(2 * (nbins + 1), 0), a;
    for (int which = 0; which < 2; ++which) {
        const uint64_t size = which == 0 ? n_lo + 1 : n_lo;
        if (!ctd::allocate(size, P.w, a)) return fail(CTD_EINVAL, "spectrum weights cannot be allocated");
        uint64_t *pr = &pref[which * (nbins + 1)];
        for (int j = 0; j < nbins; ++j) pr[j + 1] = pr[j] + a[j];
    }
    int rc;
    if ((rc = P.pref.ensure(pref.size()))) return rc;
    CK(cudaMemcpyAsync(P.pref.p, pref.data(), pref.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    P.alloc_n = n;
    P.alloc_nb = nb;
    return CTD_OK;
}

int ensure_run_buffers(Phantom &P)
{
    int rc;
    if ((rc = P.tally.ensure(P.nvox)) || (rc = P.sum_d.ensure(P.nvox)) || (rc = P.sum_d2.ensure(P.nvox)) ||
        (rc = P.edep.ensure(P.nvox)) || (rc = P.dose.ensure(P.nvox)) || (rc = P.sd.ensure(P.nvox)) ||
        (rc = P.partials.ensure(6 * kRsdParts)) || (rc = P.result.ensure(8)) || (rc = P.counts.ensure(1)) ||
        (rc = P.work.ensure(1)))
        return rc;
    return CTD_OK;
}

int check_ready(Phantom &P)
{
    if (!P.has_src) return fail(CTD_EINVAL, "no source set");
    if (!P.has_spec) return fail(CTD_EINVAL, "no spectrum set");
    for (size_t j = 0; j < P.w.size(); ++j)
        if (!(P.e_lo[j] >= P.phys.e_min_kev && P.e_hi[j] <= P.phys.e_max_kev))
            return fail(CTD_EINVAL, "spectrum bin %zu outside the node grid [%d, %d] keV", j, P.phys.e_min_kev,
                        P.phys.e_max_kev);
    return CTD_OK;
}

// The per-request part of a transport launch (geometry, source, spectrum, outputs).
void fill_request(Phantom &P, uint64_t seed, ctd::RequestDesc &q)
{
    std::memset(&q, 0, sizeof(q));
    q.mat = P.mat.p;
    q.rho = P.rho.p;
    q.tab = P.tab.p;
    q.mmax = P.mm.p;
    q.rsurf = P.rs.p;
    q.csurf = P.cs.p;
    q.cs_stride = P.phys.compton_model == CTD_COMPTON_WH ? P.n_e * P.phys.n_zeta : 0;
    if (P.fl_nu > 0) {
        q.fl_thr = P.fl_thr.p;
        q.fl_alias = P.fl_alias.p;
        q.fl_n = P.fl_nu * P.fl_nv;
        q.fl_nu = P.fl_nu;
        q.fl_magic = ((1ull << 40) / static_cast<uint64_t>(P.fl_nu)) + 1;
        q.fl_du = static_cast<float>((P.src.u_hi_cm - P.src.u_lo_cm) / static_cast<double>(P.fl_nu));
        q.fl_dv = static_cast<float>((P.src.v_hi_cm - P.src.v_lo_cm) / static_cast<double>(P.fl_nv));
    }
    q.n_mat = static_cast<int>(P.mats.size());
    q.work = P.work.p;
    q.nbins = static_cast<int>(P.w.size());
    q.bin_lo = P.bins.p;
    q.bin_hi = P.bins.p + q.nbins;
    q.cb = P.proj.p;
    q.sb = P.proj.p + (P.src.n_proj > 0 ? P.src.n_proj : 1);
    q.zb = P.proj.p + 2 * (P.src.n_proj > 0 ? P.src.n_proj : 1);
    q.hz0 = static_cast<float>(P.src.z0_cm);
    q.hdz = static_cast<float>(P.src.z1_cm - P.src.z0_cm);
    q.counts = P.counts.p;
    q.seed = seed;
    q.nx = P.nx;
    q.ny = P.ny;
    q.nz = P.nz;
    const double hx = static_cast<double>(P.nx) * P.dx / 2.0, hy = static_cast<double>(P.ny) * P.dy / 2.0,
                 hz = static_cast<double>(P.nz) * P.dz / 2.0;
    q.bx0 = static_cast<float>(-hx);
    q.by0 = static_cast<float>(-hy);
    q.bz0 = static_cast<float>(-hz);
    q.bx1 = static_cast<float>(hx);
    q.by1 = static_cast<float>(hy);
    q.bz1 = static_cast<float>(hz);
    q.ix = static_cast<float>(1.0 / P.dx);
    q.iy = static_cast<float>(1.0 / P.dy);
    q.iz = static_cast<float>(1.0 / P.dz);
    q.src_kind = P.src.kind;
    q.n_proj = P.src.n_proj;
    q.continuous = P.src.continuous;
    q.D = static_cast<float>(P.src.sad_cm);
    q.D2 = q.D * q.D;
    q.ulo = static_cast<float>(P.src.u_lo_cm);
    q.uw = static_cast<float>(P.src.u_hi_cm) - q.ulo;
    q.vlo = static_cast<float>(P.src.v_lo_cm);
    q.vw = static_cast<float>(P.src.v_hi_cm) - q.vlo;
    q.a0t = static_cast<float>(P.src.arc0_rad / (2.0 * ctd::kPi));
    q.awt = static_cast<float>((P.src.arc1_rad - P.src.arc0_rad) / (2.0 * ctd::kPi));
    q.mode = P.phys.mode;
    q.max_real = P.phys.max_real;
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        q.rk[2 * r] = k0;
        q.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

void fill_shared(Phantom &P, ctd::SharedTables &sh)
{
    sh.n_e = P.n_e;
    sh.n_zeta = P.phys.n_zeta;
    sh.e_min = P.phys.e_min_kev;
    sh.max_n_mat = static_cast<int>(P.mats.size());
}

cudaEvent_t event_at(ctd_ctx *ctx, size_t i)
{
    while (ctx->events.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->events.push_back(e);
    }
    return ctx->events[i];
}

// Streams for independent request chains; chain r runs on lane r % kMaxLanes.
constexpr int kMaxLanes = 64;

int ensure_lanes(ctd_ctx *ctx, int n)
{
    n = std::min(n, kMaxLanes);
    while (static_cast<int>(ctx->lanes.size()) < n) {
        cudaStream_t s;
        cudaEvent_t e;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(s);
            return fail(CTD_ECUDA, "cudaEventCreate failed");
        }
        ctx->lanes.push_back(s);
        ctx->lane_done.push_back(e);
    }
    if (!ctx->fork_event) CK(cudaEventCreateWithFlags(&ctx->fork_event, cudaEventDisableTiming));
    return CTD_OK;
}

// the first min(n, kMaxLanes) lanes start after everything issued so far on origin
int fork_lanes(ctd_ctx *ctx, cudaStream_t origin, int n)
{
    CK(cudaEventRecord(ctx->fork_event, origin));
    for (int i = 0; i < std::min(n, kMaxLanes); ++i) CK(cudaStreamWaitEvent(ctx->lanes[i], ctx->fork_event, 0));
    return CTD_OK;
}

// origin continues after everything issued on those lanes
int join_lanes(ctd_ctx *ctx, cudaStream_t origin, int n)
{
    for (int i = 0; i < std::min(n, kMaxLanes); ++i) {
        CK(cudaEventRecord(ctx->lane_done[i], ctx->lanes[i]));
        CK(cudaStreamWaitEvent(origin, ctx->lane_done[i], 0));
    }
    return CTD_OK;
}

cudaStream_t lane(ctd_ctx *ctx, int r) { return ctx->lanes[r % kMaxLanes]; }

// One single-request launch of q (its tables from P) on stream s, at the
// context's launch shape.
int launch_one(ctd_ctx *ctx, Phantom &P, const ctd::RequestDesc &q, cudaStream_t s)
{
    ctd::LaunchParams L;
    std::memset(&L, 0, sizeof(L));
    fill_shared(P, L.sh);
    L.one = q;
    L.chunk = ctx->chunk;
    L.flight_cap = ctx->flight_cap;
    return ctd::launch_transport(L, ctx->num_sms * ctx->blocks_per_sm, ctx->threads,
                                 ctx->threads * ctx->blocks_per_sm, s);
}

// Mean, standard error, avg RSD and deposited energy of a finished run of nb
// batches, on stream s.
int finish_stats(Phantom &P, int nb, cudaStream_t s)
{
    int e = ctd::launch_finalize(P.sum_d.p, P.sum_d2.p, nb, P.dose.p, P.sd.p, P.nvox, s);
    if (e == CTD_OK) e = ctd::launch_rsd(P.dose.p, P.sd.p, P.rho.p, P.nvox, P.partials.p, kRsdParts, P.result.p, s);
    if (e == CTD_OK)
        e = ctd::launch_sum(P.edep.p, P.nvox, P.partials.p + 5 * kRsdParts, kRsdParts, P.result.p + 3, s);
    return e;
}

// One transport launch over local histories [lb, le) of a batch starting at global h_base.
int transport(ctd_ctx *ctx, Phantom &P, ctd::RequestDesc &q, int which_size, uint64_t h_base, uint64_t lb,
              uint64_t le, double *tally, size_t ev_index)
{
    ctd::LaunchParams L;
    std::memset(&L, 0, sizeof(L));
    fill_shared(P, L.sh);
    q.pref = P.pref.p + which_size * (q.nbins + 1);
    q.h_base = h_base;
    q.local_begin = lb;
    q.local_end = le;
    q.tally = tally;
    q.work = P.work.p;
    L.one = q;
    L.chunk = ctx->chunk;
    L.flight_cap = ctx->flight_cap;
    CK(cudaMemsetAsync(P.work.p, 0, sizeof(unsigned long long), ctx->stream));
    cudaEvent_t e0 = event_at(ctx, 2 * ev_index), e1 = event_at(ctx, 2 * ev_index + 1);
    if (!e0 || !e1) return fail(CTD_ECUDA, "cudaEventCreate failed");
    CK(cudaEventRecord(e0, ctx->stream));
    const int grid = ctx->num_sms * ctx->blocks_per_sm;
    CKS(ctd::launch_transport(L, grid, ctx->threads, ctx->threads * ctx->blocks_per_sm, ctx->stream));
    CK(cudaEventRecord(e1, ctx->stream));
    return CTD_OK;
}

int prepare_run(ctd_ctx *ctx, Phantom &P, uint64_t n, int nb)
{
    int rc;
    if ((rc = check_ready(P))) return rc;
    if ((rc = build_tables(ctx, P))) return rc;
    if ((rc = upload_allocation(ctx, P, n, nb))) return rc;
    if ((rc = ensure_run_buffers(P))) return rc;
    return CTD_OK;
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device time of launches [0, n_launch) from their event pairs.
int transport_time(ctd_ctx *ctx, size_t n_launch, double &t)
{
    t = 0.0;
    for (size_t i = 0; i < n_launch; ++i) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->events[2 * i], ctx->events[2 * i + 1]));
        t += ms * 1e-3;
    }
    return CTD_OK;
}

// Counts, energies and precision figures of several phantoms read back in one
// go (copies into pinned staging, one synchronisation).
int collect_many(ctd_ctx *ctx, Phantom *const *ps, int n, size_t n_launch, double t0_wall,
                 const double *t0_each = nullptr)
{
    if (static_cast<size_t>(n) > ctx->staged_n) {
        if (ctx->staged) cudaFreeHost(ctx->staged);
        ctx->staged = nullptr;
        ctx->staged_n = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&ctx->staged), n * sizeof(Staged)) != cudaSuccess) {
            cudaGetLastError();
            return fail(CTD_ENOMEM, "cudaMallocHost failed");
        }
        ctx->staged_n = n;
    }
    for (int i = 0; i < n; ++i) {
        CK(cudaMemcpyAsync(&ctx->staged[i].c, ps[i]->counts.p, sizeof(ctd::DeviceCounts), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->staged[i].res, ps[i]->result.p, sizeof(ctx->staged[i].res), cudaMemcpyDeviceToHost,
                           ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    const double t_now = now_s();
    double t_transport;
    int rc;
    if ((rc = transport_time(ctx, n_launch, t_transport))) return rc;
    for (int i = 0; i < n; ++i) {
        const ctd::DeviceCounts &c = ctx->staged[i].c;
        const double *res = ctx->staged[i].res;
        ctd_run_stats &s = ps[i]->stats;
        s.pe = c.n[ctd::kCntPe];
        s.compton = c.n[ctd::kCntCompton];
        s.rayleigh = c.n[ctd::kCntRayleigh];
        s.fictitious = c.n[ctd::kCntFict];
        s.escaped = c.n[ctd::kCntEscaped];
        s.missed = c.n[ctd::kCntMissed];
        s.cutoff = c.n[ctd::kCntCutoff];
        s.terminated = c.n[ctd::kCntTerminated];
        s.aborted = c.n[ctd::kCntAborted];
        s.steps = c.n[ctd::kCntSteps];
        s.e_emitted_kev = ctd::fixed_kev(c.e_fix[0], c.e_fix[1]);
        s.e_escaped_kev = ctd::fixed_kev(c.e_fix[2], c.e_fix[3]);
        s.avg_rsd = res[0];
        s.paper_sigma_bar = res[1];
        s.d_max = res[2];
        s.e_deposited_kev = res[3];
        s.t_transport_s = t_transport;
        s.transport_launches = static_cast<int>(n_launch);
        s.t_total_s = t_now - (t0_each ? t0_each[i] : t0_wall);
    }
    return CTD_OK;
}

int collect(ctd_ctx *ctx, Phantom &P, size_t n_launch, double t0_wall)
{
    Phantom *ps[1] = {&P};
    return collect_many(ctx, ps, 1, n_launch, t0_wall);
}

}  // namespace

extern "C" {

const char *ctd_last_error(void) { return g_error.c_str(); }

int ctd_abi_version(void) { return CTD_ABI_VERSION; }

int ctd_create(ctd_ctx **out, const ctd_options *opt)
{
    g_error.clear();
    if (!out) return fail(CTD_EINVAL, "null output pointer");
    *out = nullptr;
    std::unique_ptr<ctd_ctx> ctx(new ctd_ctx());
    if (opt) {
        ctx->device = opt->device;
        if (opt->blocks_per_sm > 0) ctx->blocks_per_sm = opt->blocks_per_sm;
        if (opt->multi_blocks_per_sm > 0) ctx->multi_blocks_per_sm = opt->multi_blocks_per_sm;
        if (opt->serve_max_active > 0) ctx->max_active = opt->serve_max_active;
        if (opt->serve_round_histories > 0) ctx->round_histories = opt->serve_round_histories;
        if (opt->threads_per_block > 0) ctx->threads = opt->threads_per_block;
        if (opt->chunk > 0) ctx->chunk = opt->chunk;
        if (opt->flight_cap > 0) ctx->flight_cap = opt->flight_cap;
        ctx->shared_launch = opt->shared_launch != 0;
    }
    if (ctx->threads % 32 != 0 || ctx->threads > 256) return fail(CTD_EINVAL, "threads_per_block must be a multiple of 32 and at most 256");
    if (ctx->blocks_per_sm > 64 || ctx->multi_blocks_per_sm > 64) return fail(CTD_EINVAL, "blocks_per_sm at most 64");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (ctx->device < 0 || ctx->device >= ndev) return fail(CTD_EINVAL, "device %d out of range (%d devices)", ctx->device, ndev);
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (opt && opt->stream) {
        ctx->stream = static_cast<cudaStream_t>(opt->stream);
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    *out = ctx.release();
    return CTD_OK;
}

int ctd_destroy(ctd_ctx *ctx)
{
    if (!ctx) return CTD_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->phantoms.clear();
    if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
    for (auto e : ctx->events) cudaEventDestroy(e);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (auto l : ctx->lanes) cudaStreamDestroy(l);
    for (auto e : ctx->lane_done) cudaEventDestroy(e);
    if (ctx->fork_event) cudaEventDestroy(ctx->fork_event);
    if (ctx->staged) cudaFreeHost(ctx->staged);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return CTD_OK;
}

int ctd_create_phantom(ctd_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz, const uint8_t *mat,
                       const float *density, int n_mat, const ctd_material *mats, ctd_phantom *out)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (!out || !mat || !density || !mats) return fail(CTD_EINVAL, "null pointer argument");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(CTD_EINVAL, "voxel counts must be positive");
    if (!(dx > 0 && dy > 0 && dz > 0)) return fail(CTD_EINVAL, "voxel sizes must be positive");
    if (n_mat <= 0 || n_mat > ctd::kMaxPhantomMaterials) return fail(CTD_EINVAL, "n_mat must be 1..16");
    for (int m = 0; m < n_mat; ++m)
        if (!(mats[m].z_over_a > 0 && mats[m].a_mol > 0 && mats[m].z_eff > 0) || !std::isfinite(mats[m].q0) ||
            !std::isfinite(mats[m].sq0))
            return fail(CTD_EINVAL, "material %d has non-positive or non-finite parameters", m);
    const size_t nvox = static_cast<size_t>(nx) * ny * nz;
    if (nvox > (static_cast<size_t>(1) << 40)) return fail(CTD_EINVAL, "phantom too large");
    std::unique_ptr<Phantom> P(new Phantom());
    P->nx = nx; P->ny = ny; P->nz = nz;
    P->dx = dx; P->dy = dy; P->dz = dz;
    P->nvox = nvox;
    P->mats.assign(mats, mats + n_mat);
    P->rho_max.assign(n_mat, 0.0);
    P->present.assign(n_mat, 0);
    for (size_t v = 0; v < nvox; ++v) {
        const int m = mat[v];
        const double r = density[v];
        if (m >= n_mat) return fail(CTD_EINVAL, "voxel %zu has material %d >= n_mat", v, m);
        if (!(r >= 0.0) || !std::isfinite(r)) return fail(CTD_EINVAL, "voxel %zu has an invalid density", v);
        if (!P->present[m] || r > P->rho_max[m]) P->rho_max[m] = r;
        P->present[m] = 1;
    }
    P->phys.e_min_kev = 1;
    P->phys.e_max_kev = 150;
    P->phys.n_zeta = 1024;
    P->phys.majorant_scale = 1.0;
    P->phys.mode = CTD_MODE_FULL;
    P->phys.max_real = 0;
    P->phys.compton_model = CTD_COMPTON_KN;
    if ((rc = P->mat.ensure(nvox)) || (rc = P->rho.ensure(nvox))) return rc;
    CK(cudaMemcpyAsync(P->mat.p, mat, nvox, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P->rho.p, density, nvox * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int id = ctx->next_id++;
    ctx->phantoms[id] = std::move(P);
    *out = id;
    return CTD_OK;
}

int ctd_destroy_phantom(ctd_ctx *ctx, ctd_phantom ph)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    auto it = ctx->phantoms.find(ph);
    if (it == ctx->phantoms.end()) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if ((rc = busy(it->second.get()))) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->phantoms.erase(it);
    return CTD_OK;
}

int ctd_set_physics(ctd_ctx *ctx, ctd_phantom ph, const ctd_physics *phys)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!phys) return fail(CTD_EINVAL, "null physics");
    if ((rc = busy(P))) return rc;
    if (phys->e_min_kev < 1 || phys->e_max_kev <= phys->e_min_kev || phys->e_max_kev > 100000)
        return fail(CTD_EINVAL, "node grid must satisfy 1 <= e_min < e_max");
    if (phys->n_zeta < 2 || phys->n_zeta > (1 << 20)) return fail(CTD_EINVAL, "n_zeta must be 2..2^20");
    if (!(phys->majorant_scale >= 1.0) || !std::isfinite(phys->majorant_scale))
        return fail(CTD_EINVAL, "majorant_scale must be >= 1");
    if (phys->mode != CTD_MODE_FULL && phys->mode != CTD_MODE_MAX_REAL) return fail(CTD_EINVAL, "unknown mode");
    if (phys->mode == CTD_MODE_MAX_REAL && phys->max_real < 1) return fail(CTD_EINVAL, "max_real must be >= 1");
    if (phys->compton_model != CTD_COMPTON_KN && phys->compton_model != CTD_COMPTON_WH)
        return fail(CTD_EINVAL, "unknown Compton model");
    P->phys = *phys;
    P->tables_ok = false;
    return CTD_OK;
}

int ctd_set_source(ctd_ctx *ctx, ctd_phantom ph, const ctd_source *src)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!src) return fail(CTD_EINVAL, "null source");
    if ((rc = busy(P))) return rc;
    if (src->kind != CTD_SRC_STATIC && src->kind != CTD_SRC_ARC) return fail(CTD_EINVAL, "unknown source kind");
    if (!(src->sad_cm > 0) || !(src->u_hi_cm >= src->u_lo_cm) || !(src->v_hi_cm >= src->v_lo_cm))
        return fail(CTD_EINVAL, "source distance must be positive and field bounds ordered");
    const double hx = P->nx * P->dx / 2.0, hy = P->ny * P->dy / 2.0, hz = P->nz * P->dz / 2.0;
    if (src->kind == CTD_SRC_STATIC && !(src->sad_cm > hz))
        return fail(CTD_EINVAL, "static source must lie outside the phantom");
    if (src->kind == CTD_SRC_ARC && !(src->sad_cm > std::sqrt(hx * hx + hy * hy)))
        return fail(CTD_EINVAL, "arc radius must clear the phantom");
    const int np = src->kind == CTD_SRC_ARC && !src->continuous ? src->n_proj : 1;
    if (src->kind == CTD_SRC_ARC && !src->continuous && (src->n_proj < 1 || src->n_proj > (1 << 24)))
        return fail(CTD_EINVAL, "n_proj must be 1..2^24");
    if (!std::isfinite(src->z0_cm) || !std::isfinite(src->z1_cm)) return fail(CTD_EINVAL, "source heights must be finite");
    std::vector<float> tab(3 * np);
    for (int k = 0; k < np; ++k) {
        // projection angles b_k = arc0 + (arc1 - arc0) k / n_proj, heights z0 + (z1 - z0) k / n_proj
        const double b = src->arc0_rad + (src->arc1_rad - src->arc0_rad) * static_cast<double>(k) / static_cast<double>(np);
        tab[k] = static_cast<float>(std::cos(b));
        tab[np + k] = static_cast<float>(std::sin(b));
        tab[2 * np + k] =
            static_cast<float>(src->z0_cm + (src->z1_cm - src->z0_cm) * static_cast<double>(k) / static_cast<double>(np));
    }
    if ((rc = P->proj.ensure(tab.size()))) return rc;
    CK(cudaMemcpyAsync(P->proj.p, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    P->src = *src;
    P->src.n_proj = np;
    P->has_src = true;
    return CTD_OK;
}

int ctd_set_fluence(ctd_ctx *ctx, ctd_phantom ph, int n_u, int n_v, const double *f)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if ((rc = busy(P))) return rc;
    if (n_u == 0) {
        P->fl_nu = P->fl_nv = 0;
        return CTD_OK;
    }
    if (n_u < 0 || n_u > 65535 || n_v <= 0 || static_cast<int64_t>(n_u) * n_v > (1 << 24) || !f)
        return fail(CTD_EINVAL, "fluence map: n_u <= 65535, 1 <= n_u * n_v <= 2^24 beamlets and a host array");
    const int n = n_u * n_v;
    std::vector<uint32_t> thr(n);
    std::vector<int32_t> al(n);
    if (!ctd::alias_build(n, f, thr.data(), al.data()))
        return fail(CTD_EINVAL, "fluence map needs finite intensities >= 0 with a positive sum");
    if ((rc = P->fl_thr.ensure(n)) || (rc = P->fl_alias.ensure(n))) return rc;
    CK(cudaMemcpyAsync(P->fl_thr.p, thr.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P->fl_alias.p, al.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    P->h_thr.swap(thr);
    P->h_alias.swap(al);
    P->fl_nu = n_u;
    P->fl_nv = n_v;
    return CTD_OK;
}

int ctd_get_fluence_table(ctd_ctx *ctx, ctd_phantom ph, int *n, uint32_t *thr, int32_t *alias)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    const int m = P->fl_nu * P->fl_nv;
    if (n) *n = m;
    if (thr) std::copy(P->h_thr.begin(), P->h_thr.begin() + m, thr);
    if (alias) std::copy(P->h_alias.begin(), P->h_alias.begin() + m, alias);
    return CTD_OK;
}

int ctd_set_spectrum(ctd_ctx *ctx, ctd_phantom ph, const double *e_lo, const double *e_hi, const double *w, int nbins)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!e_lo || !e_hi || !w || nbins <= 0 || nbins > 100000) return fail(CTD_EINVAL, "bad spectrum arrays");
    if ((rc = busy(P))) return rc;
    double total = 0.0;
    for (int j = 0; j < nbins; ++j) {
        if (!(e_hi[j] >= e_lo[j]) || !(e_lo[j] > 0) || !(w[j] >= 0) || !std::isfinite(w[j]) || !std::isfinite(e_hi[j]))
            return fail(CTD_EINVAL, "spectrum bin %d is invalid", j);
        total += w[j];
    }
    if (!(total > 0)) return fail(CTD_EINVAL, "spectrum weights sum to zero");
    P->e_lo.assign(e_lo, e_lo + nbins);
    P->e_hi.assign(e_hi, e_hi + nbins);
    P->w.assign(w, w + nbins);
    std::vector<float> b(2 * nbins);
    for (int j = 0; j < nbins; ++j) {
        b[j] = static_cast<float>(e_lo[j]);
        b[nbins + j] = static_cast<float>(e_hi[j]);
    }
    if ((rc = P->bins.ensure(b.size()))) return rc;
    CK(cudaMemcpyAsync(P->bins.p, b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    P->alloc_n = ~0ull;
    P->alloc_nb = -1;
    P->has_spec = true;
    return CTD_OK;
}

int ctd_run(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (n_batches < 2 || static_cast<uint64_t>(n_batches) > n_histories)
        return fail(CTD_EINVAL, "need 2 <= n_batches <= n_histories");
    if ((rc = busy(P))) return rc;
    const double t0 = now_s();
    if ((rc = prepare_run(ctx, *P, n_histories, n_batches))) return rc;
    P->have_result = false;
    const size_t nv = P->nvox;
    CK(cudaMemsetAsync(P->tally.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->sum_d.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->sum_d2.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->edep.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
    ctd::RequestDesc T;
    fill_request(*P, seed, T);
    const uint64_t n_lo = n_histories / n_batches, rem = n_histories % n_batches;
    const double vol = P->dx * P->dy * P->dz;
    uint64_t h = 0;
    for (int b = 0; b < n_batches; ++b) {
        const uint64_t nb = static_cast<uint64_t>(b) < rem ? n_lo + 1 : n_lo;
        const int which = static_cast<uint64_t>(b) < rem ? 0 : 1;
        if ((rc = transport(ctx, *P, T, which, h, 0, nb, P->tally.p, b))) return rc;
        // d = E / (m n_b) with m = rho V / 1000 kg
        const double scale = ctd::kKevToJ * 1000.0 / (vol * static_cast<double>(nb));
        CKS(ctd::launch_fold(P->tally.p, P->rho.p, P->sum_d.p, P->sum_d2.p, P->edep.p, nv, scale, ctx->stream));
        h += nb;
    }
    CKS(ctd::launch_finalize(P->sum_d.p, P->sum_d2.p, n_batches, P->dose.p, P->sd.p, nv, ctx->stream));
    CKS(ctd::launch_rsd(P->dose.p, P->sd.p, P->rho.p, nv, P->partials.p, kRsdParts, P->result.p, ctx->stream));
    CKS(ctd::launch_sum(P->edep.p, nv, P->partials.p + 5 * kRsdParts, kRsdParts, P->result.p + 3, ctx->stream));
    if ((rc = collect(ctx, *P, n_batches, t0))) return rc;
    P->stats.histories = n_histories;
    P->stats.n_batches = n_batches;
    P->have_result = true;
    return CTD_OK;
}

}  // extern "C"

namespace {

}  // namespace

extern "C" {

int ctd_run_batch(ctd_ctx *ctx, int n_req, const ctd_phantom *phantoms, const uint64_t *n_histories,
                  const uint64_t *seeds, int n_batches)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (n_req <= 0 || !phantoms || !n_histories || !seeds) return fail(CTD_EINVAL, "bad request arrays");
    if (n_batches < 2) return fail(CTD_EINVAL, "need n_batches >= 2");
    const double t0 = now_s();
    std::vector<Phantom *> ps(n_req);
    for (int r = 0; r < n_req; ++r) {
        ps[r] = find(ctx, phantoms[r]);
        if (!ps[r]) return fail(CTD_ENOTFOUND, "unknown phantom %d", phantoms[r]);
        for (int k = 0; k < r; ++k)
            if (ps[k] == ps[r]) return fail(CTD_EINVAL, "phantom %d appears twice in one batch", phantoms[r]);
        if (static_cast<uint64_t>(n_batches) > n_histories[r])
            return fail(CTD_EINVAL, "request %d has fewer histories than batches", r);
        if ((rc = busy(ps[r]))) return rc;
        if ((rc = prepare_run(ctx, *ps[r], n_histories[r], n_batches))) return rc;
        // one shared launch holds one node grid and one angular surface size
        const ctd_physics &a = ps[0]->phys, &b = ps[r]->phys;
        if (ctx->shared_launch && (a.e_min_kev != b.e_min_kev || a.e_max_kev != b.e_max_kev || a.n_zeta != b.n_zeta))
            return fail(CTD_EINVAL, "request %d has another node grid than request 0", r);
    }
    int max_n_mat = 0;
    for (int r = 0; r < n_req; ++r) max_n_mat = std::max(max_n_mat, static_cast<int>(ps[r]->mats.size()));
    if ((rc = ctx->u_work.ensure(static_cast<size_t>(n_batches) * n_req))) return rc;
    // descriptors for every batch of every request, the history and tile offsets
    std::vector<ctd::RequestDesc> descs(static_cast<size_t>(n_batches) * n_req);
    std::vector<ctd::FoldDesc> folds(static_cast<size_t>(n_batches) * n_req);
    std::vector<uint64_t> tiles(n_req + 1, 0);
    for (int r = 0; r < n_req; ++r)
        tiles[r + 1] = tiles[r] + (ps[r]->nvox + ctd::kFoldTile - 1) / ctd::kFoldTile;
    for (int r = 0; r < n_req; ++r) {
        Phantom &P = *ps[r];
        const size_t nv = P.nvox;
        CK(cudaMemsetAsync(P.tally.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P.sum_d.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P.sum_d2.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P.edep.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P.counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
        P.have_result = false;
        const uint64_t n = n_histories[r], n_lo = n / n_batches, rem = n % n_batches;
        const double vol = P.dx * P.dy * P.dz;
        uint64_t h = 0;
        for (int b = 0; b < n_batches; ++b) {
            const uint64_t nb = static_cast<uint64_t>(b) < rem ? n_lo + 1 : n_lo;
            const int which = static_cast<uint64_t>(b) < rem ? 0 : 1;
            ctd::RequestDesc &q = descs[static_cast<size_t>(b) * n_req + r];
            fill_request(P, seeds[r], q);
            q.work = ctx->u_work.p + static_cast<size_t>(b) * n_req + r;
            q.pref = P.pref.p + which * (q.nbins + 1);
            q.h_base = h;
            q.local_begin = 0;
            q.local_end = nb;
            q.tally = P.tally.p;
            ctd::FoldDesc &f = folds[static_cast<size_t>(b) * n_req + r];
            f.tally = P.tally.p;
            f.rho = P.rho.p;
            f.sum_d = P.sum_d.p;
            f.sum_d2 = P.sum_d2.p;
            f.edep = P.edep.p;
            f.nvox = nv;
            f.scale = ctd::kKevToJ * 1000.0 / (vol * static_cast<double>(nb));
            h += nb;
        }
    }
    std::vector<unsigned char> key;
    auto put = [&key](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        key.insert(key.end(), c, c + n);
    };
    put(descs.data(), descs.size() * sizeof(ctd::RequestDesc));
    put(folds.data(), folds.size() * sizeof(ctd::FoldDesc));
    const int shape[8] = {n_batches, ctx->shared_launch, ctx->num_sms, ctx->blocks_per_sm, ctx->multi_blocks_per_sm,
                          ctx->threads, ctx->chunk, ctx->flight_cap};
    put(shape, sizeof(shape));
    size_t n_launch = 1;
    std::function<int(cudaStream_t)> body;
    if (!ctx->shared_launch) {
        // every request is its own chain (claim counters cleared, then transport
        // and fold of each batch in turn) on its own stream; the chains overlap
        for (int r = 0; r < n_req; ++r) {
            ctd::SharedTables sh;
            std::memset(&sh, 0, sizeof(sh));
            fill_shared(*ps[r], sh);
            put(&sh, sizeof(sh));
        }
        if ((rc = ensure_lanes(ctx, n_req))) return rc;
        if (!event_at(ctx, 0) || !event_at(ctx, 1)) return fail(CTD_ECUDA, "cudaEventCreate failed");
        body = [&](cudaStream_t cs) {
            if (cudaMemsetAsync(ctx->u_work.p, 0, static_cast<size_t>(n_batches) * n_req * sizeof(unsigned long long),
                                cs) != cudaSuccess ||
                cudaEventRecordWithFlags(ctx->events[0], cs, cudaEventRecordExternal) != cudaSuccess)
                return static_cast<int>(CTD_ECUDA);
            int e = fork_lanes(ctx, cs, n_req);
            for (int r = 0; r < n_req && e == CTD_OK; ++r) {
                Phantom &P = *ps[r];
                for (int b = 0; b < n_batches && e == CTD_OK; ++b) {
                    const size_t k = static_cast<size_t>(b) * n_req + r;
                    e = launch_one(ctx, P, descs[k], lane(ctx, r));
                    if (e == CTD_OK)
                        e = ctd::launch_fold(P.tally.p, P.rho.p, P.sum_d.p, P.sum_d2.p, P.edep.p, P.nvox, folds[k].scale,
                                             lane(ctx, r));
                }
                if (e == CTD_OK) e = finish_stats(P, n_batches, lane(ctx, r));
            }
            if (e == CTD_OK) e = join_lanes(ctx, cs, n_req);
            if (e == CTD_OK && cudaEventRecordWithFlags(ctx->events[1], cs, cudaEventRecordExternal) != cudaSuccess)
                e = CTD_ECUDA;
            return e;
        };
    } else {
        // batch b of every request in one launch, then one fold over every grid
        if ((rc = ctx->u_reqs.ensure(descs.size())) || (rc = ctx->u_folds.ensure(folds.size())) ||
            (rc = ctx->u_tiles.ensure(tiles.size())))
            return rc;
        CK(cudaMemcpyAsync(ctx->u_reqs.p, descs.data(), descs.size() * sizeof(ctd::RequestDesc),
                           cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->u_folds.p, folds.data(), folds.size() * sizeof(ctd::FoldDesc), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->u_tiles.p, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                           ctx->stream));
        put(tiles.data(), tiles.size() * sizeof(uint64_t));
        const void *bufs[3] = {ctx->u_reqs.p, ctx->u_folds.p, ctx->u_tiles.p};
        put(bufs, sizeof(bufs));
        ctd::LaunchParams L;
        std::memset(&L, 0, sizeof(L));
        fill_shared(*ps[0], L.sh);
        L.sh.max_n_mat = max_n_mat;
        L.n_req = n_req;
        L.chunk = ctx->chunk;
        L.flight_cap = ctx->flight_cap;
        put(&L, sizeof(L));
        const int mgrid = ctx->num_sms * ctx->multi_blocks_per_sm;
        for (int b = 0; b < n_batches; ++b)
            if (!event_at(ctx, 2 * b) || !event_at(ctx, 2 * b + 1)) return fail(CTD_ECUDA, "cudaEventCreate failed");
        n_launch = n_batches;
        body = [&, L, mgrid](cudaStream_t cs) mutable {
            int e = CTD_OK;
            if (cudaMemsetAsync(ctx->u_work.p, 0, static_cast<size_t>(n_batches) * n_req * sizeof(unsigned long long),
                                cs) != cudaSuccess)
                e = CTD_ECUDA;
            for (int b = 0; b < n_batches && e == CTD_OK; ++b) {
                L.reqs = ctx->u_reqs.p + static_cast<size_t>(b) * n_req;
                if (cudaEventRecordWithFlags(ctx->events[2 * b], cs, cudaEventRecordExternal) != cudaSuccess)
                    e = CTD_ECUDA;
                if (e == CTD_OK)
                    e = ctd::launch_transport(L, mgrid, ctx->threads, ctx->threads * ctx->multi_blocks_per_sm, cs);
                if (e == CTD_OK &&
                    cudaEventRecordWithFlags(ctx->events[2 * b + 1], cs, cudaEventRecordExternal) != cudaSuccess)
                    e = CTD_ECUDA;
                if (e == CTD_OK)
                    e = ctd::launch_fold_multi(ctx->u_folds.p + static_cast<size_t>(b) * n_req, ctx->u_tiles.p, n_req,
                                               tiles[n_req], cs);
            }
            for (int r = 0; r < n_req && e == CTD_OK; ++r) e = finish_stats(*ps[r], n_batches, cs);
            return e;
        };
    }
    const void *work = ctx->u_work.p;
    put(&work, sizeof(work));
    for (int r = 0; r < n_req; ++r) {
        const void *out[4] = {ps[r]->dose.p, ps[r]->sd.p, ps[r]->partials.p, ps[r]->result.p};
        put(out, sizeof(out));
    }
    // The batch loop is captured once into a CUDA graph and replayed while the
    // descriptors, buffers and launch shape stay the same.
    if (!ctx->batch_graph || key != ctx->batch_graph_key) {
        if (ctx->batch_graph) {
            cudaGraphExecDestroy(ctx->batch_graph);
            ctx->batch_graph = nullptr;
        }
        if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = ctx->capture_stream;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const int crc = body(cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (crc != CTD_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(CTD_ECUDA, "capturing the batched launches failed");
        }
        const cudaError_t ie = cudaGraphInstantiate(&ctx->batch_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            ctx->batch_graph = nullptr;
            return fail(CTD_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ie));
        }
        ctx->batch_graph_key.swap(key);
    }
    CK(cudaGraphLaunch(ctx->batch_graph, ctx->stream));
    if ((rc = collect_many(ctx, ps.data(), n_req, n_launch, t0))) return rc;
    for (int r = 0; r < n_req; ++r) {
        ps[r]->stats.histories = n_histories[r];
        ps[r]->stats.n_batches = n_batches;
        ps[r]->have_result = true;
    }
    return CTD_OK;
}

int ctd_run_range(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches, uint64_t h_begin,
                  uint64_t h_end, int clear)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (n_batches < 1 || static_cast<uint64_t>(n_batches) > n_histories)
        return fail(CTD_EINVAL, "need 1 <= n_batches <= n_histories");
    if (h_begin > h_end || h_end > n_histories) return fail(CTD_EINVAL, "history range outside [0, n_histories]");
    if ((rc = busy(P))) return rc;
    const double t0 = now_s();
    if ((rc = prepare_run(ctx, *P, n_histories, n_batches))) return rc;
    const size_t nv = P->nvox;
    if (clear) {
        CK(cudaMemsetAsync(P->edep.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
    }
    P->have_result = false;
    ctd::RequestDesc T;
    fill_request(*P, seed, T);
    const uint64_t n_lo = n_histories / n_batches, rem = n_histories % n_batches;
    uint64_t h = 0;
    size_t launches = 0;
    for (int b = 0; b < n_batches; ++b) {
        const uint64_t nb = static_cast<uint64_t>(b) < rem ? n_lo + 1 : n_lo;
        const uint64_t lo = h_begin > h ? h_begin : h, hi = h_end < h + nb ? h_end : h + nb;
        if (lo < hi) {
            if ((rc = transport(ctx, *P, T, static_cast<uint64_t>(b) < rem ? 0 : 1, h, lo - h, hi - h, P->edep.p, launches)))
                return rc;
            ++launches;
        }
        h += nb;
    }
    CK(cudaMemsetAsync(P->result.p, 0, 3 * sizeof(double), ctx->stream));
    CKS(ctd::launch_sum(P->edep.p, nv, P->partials.p + 5 * kRsdParts, kRsdParts, P->result.p + 3, ctx->stream));
    if ((rc = collect(ctx, *P, launches, t0))) return rc;
    P->stats.histories = h_end - h_begin;
    P->stats.n_batches = n_batches;
    return CTD_OK;
}

int ctd_get_dose_and_stddev(ctd_ctx *ctx, ctd_phantom ph, double *dose, double *stddev, size_t nvox,
                            ctd_run_stats *stats)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if ((dose || stddev) && !P->have_result) return fail(CTD_EINVAL, "no completed ctd_run on this phantom");
    if ((dose || stddev) && nvox != P->nvox) return fail(CTD_EINVAL, "nvox %zu != phantom's %zu", nvox, P->nvox);
    if (dose) CK(cudaMemcpyAsync(dose, P->dose.p, nvox * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (stddev) CK(cudaMemcpyAsync(stddev, P->sd.p, nvox * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (stats) *stats = P->stats;
    return CTD_OK;
}

int ctd_get_edep(ctd_ctx *ctx, ctd_phantom ph, double *edep_kev, size_t nvox)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!edep_kev || nvox != P->nvox) return fail(CTD_EINVAL, "edep buffer must hold the phantom's voxels");
    if (!P->edep.p) return fail(CTD_EINVAL, "nothing has run on this phantom");
    CK(cudaMemcpyAsync(edep_kev, P->edep.p, nvox * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CTD_OK;
}

int ctd_get_tables(ctd_ctx *ctx, ctd_phantom ph, int *n_e, int *n_zeta, int *n_mat, double *mu_cum, double *mu_max,
                   double *c_surf, double *r_surf)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if ((rc = build_tables(ctx, *P))) return rc;
    const int nm = static_cast<int>(P->mats.size());
    if (n_e) *n_e = P->n_e;
    if (n_zeta) *n_zeta = P->phys.n_zeta;
    if (n_mat) *n_mat = nm;
    if (mu_cum)
        for (size_t i = 0; i < static_cast<size_t>(nm) * P->n_e; ++i)
            for (int c = 0; c < 3; ++c) mu_cum[i * 3 + c] = P->h_tab[i * 4 + c];
    if (mu_max)
        for (int j = 0; j < P->n_e; ++j) mu_max[j] = P->h_mm[j];
    if (c_surf)
        for (size_t i = 0; i < P->h_cs.size(); ++i) c_surf[i] = P->h_cs[i];
    if (r_surf)
        for (size_t i = 0; i < P->h_rs.size(); ++i) r_surf[i] = P->h_rs[i];
    return CTD_OK;
}

int ctd_sample_mu(ctd_ctx *ctx, ctd_phantom ph, int kind, int material, double e_kev, uint64_t seed, uint64_t n,
                  double *out)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!out && n) return fail(CTD_EINVAL, "null output");
    if (kind != 0 && kind != 1) return fail(CTD_EINVAL, "kind is 0 (Compton) or 1 (Rayleigh)");
    if (material < 0 || material >= static_cast<int>(P->mats.size())) return fail(CTD_EINVAL, "material out of range");
    if (!(e_kev >= P->phys.e_min_kev && e_kev <= P->phys.e_max_kev)) return fail(CTD_EINVAL, "energy outside the node grid");
    if ((rc = build_tables(ctx, *P))) return rc;
    if (n == 0) return CTD_OK;
    DevBuf<double> buf;
    if ((rc = buf.ensure(n))) return rc;
    const size_t row = static_cast<size_t>(P->n_e) * P->phys.n_zeta;
    const float *surf = kind == 1 ? P->rs.p + material * row
                                  : P->cs.p + (P->phys.compton_model == CTD_COMPTON_WH ? material * row : 0);
    CKS(ctd::launch_sample_mu(surf, P->phys.n_zeta, P->n_e, P->phys.e_min_kev, static_cast<float>(e_kev), seed, n,
                              buf.p, ctx->stream));
    CK(cudaMemcpyAsync(out, buf.p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CTD_OK;
}

int ctd_eval_math(ctd_ctx *ctx, int fn, const float *x, float *out, size_t n)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (fn != 0 && fn != 1) return fail(CTD_EINVAL, "fn is 0 (log) or 1 (sincos of 2 pi x)");
    if (n == 0) return CTD_OK;
    if (!x || !out) return fail(CTD_EINVAL, "null buffer");
    DevBuf<float> bx, bo;
    const size_t no = fn == 0 ? n : 2 * n;
    if ((rc = bx.ensure(n)) || (rc = bo.ensure(no))) return rc;
    CK(cudaMemcpyAsync(bx.p, x, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CKS(ctd::launch_eval_math(fn, bx.p, bo.p, n, ctx->stream));
    CK(cudaMemcpyAsync(out, bo.p, no * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CTD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- served form
namespace {

double elapsed_since(double t) { return now_s() - t; }

// Admit queued requests in order while memory and slots allow.
int admit(ctd_ctx *ctx)
{
    double round = 0.0;
    for (int64_t id : ctx->active) round += static_cast<double>(ctx->sreqs[id].req.batch_histories);
    while (!ctx->pending.empty() && static_cast<int>(ctx->active.size()) < ctx->max_active) {
        ServeReq &R = ctx->sreqs[ctx->pending.front()];
        // first in, first out: a request joins the running set only while one round of
        // every running request stays within the round budget (one request always may)
        const double b = static_cast<double>(R.req.batch_histories);
        if (!ctx->active.empty() && round + b > ctx->round_histories) break;
        Phantom *P = find(ctx, R.ph);
        if (!P) {
            R.state = CTD_REQ_FAILED;
            ctx->pending.erase(ctx->pending.begin());
            continue;
        }
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const double need = P->tally.p ? 0.0 : 6.0 * 8.0 * static_cast<double>(P->nvox);
        if (static_cast<double>(free_b) < need + ctx->reserve_bytes) break;
        int rc;
        // one allocation for batches of batch_histories: n = 2B in 2 batches
        if ((rc = prepare_run(ctx, *P, 2 * R.req.batch_histories, 2))) {
            R.state = CTD_REQ_FAILED;
            P->busy_req = 0;
            ctx->pending.erase(ctx->pending.begin());
            continue;
        }
        const size_t nv = P->nvox;
        CK(cudaMemsetAsync(P->tally.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P->sum_d.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P->sum_d2.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P->edep.p, 0, nv * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
        P->have_result = false;
        R.state = CTD_REQ_RUNNING;
        R.t_start = now_s();
        round += b;
        ctx->active.push_back(R.id);
        ctx->pending.erase(ctx->pending.begin());
    }
    return CTD_OK;
}

void retire(ctd_ctx *ctx, ServeReq &R, int state)
{
    R.state = state;
    R.t_done = now_s();
    Phantom *P = find(ctx, R.ph);
    if (P) P->busy_req = 0;
    for (size_t i = 0; i < ctx->active.size(); ++i)
        if (ctx->active[i] == R.id) {
            ctx->active.erase(ctx->active.begin() + i);
            break;
        }
}

}  // namespace

extern "C" {

int ctd_submit(ctd_ctx *ctx, ctd_phantom ph, const ctd_request *req, ctd_req_id *out)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!req || !out) return fail(CTD_EINVAL, "null argument");
    if ((rc = busy(P))) return rc;
    if (req->batch_histories == 0) return fail(CTD_EINVAL, "batch_histories must be positive");
    if (req->min_batches == 1 || req->min_batches < 0) return fail(CTD_EINVAL, "min_batches must be >= 2 (0: 10)");
    if (!(req->rsd_target >= 0.0)) return fail(CTD_EINVAL, "rsd_target must be >= 0");
    if (req->rsd_target == 0.0 && req->n_histories_max == 0) return fail(CTD_EINVAL, "request could never stop");
    if ((rc = check_ready(*P))) return rc;
    ServeReq R;
    R.id = ctx->next_req++;
    R.ph = ph;
    R.req = *req;
    if (R.req.min_batches == 0) R.req.min_batches = 10;
    R.t_submit = now_s();
    P->busy_req = R.id;
    ctx->sreqs[R.id] = R;
    ctx->pending.push_back(R.id);
    *out = R.id;
    return CTD_OK;
}

int ctd_serve_step(ctd_ctx *ctx, int *n_active)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    // cancellations take effect at round boundaries
    for (size_t i = 0; i < ctx->active.size();) {
        ServeReq &R = ctx->sreqs[ctx->active[i]];
        if (R.cancel) retire(ctx, R, CTD_REQ_CANCELLED);
        else ++i;
    }
    if ((rc = admit(ctx))) return rc;
    const int n = static_cast<int>(ctx->active.size());
    if (n == 0) {
        if (n_active) *n_active = static_cast<int>(ctx->pending.size());
        return CTD_OK;
    }
    std::vector<Phantom *> ps(n);
    for (int i = 0; i < n; ++i) ps[i] = find(ctx, ctx->sreqs[ctx->active[i]].ph);
    for (int i = 1; i < n && ctx->shared_launch; ++i) {
        const ctd_physics &a = ps[0]->phys, &b = ps[i]->phys;
        if (a.e_min_kev != b.e_min_kev || a.e_max_kev != b.e_max_kev || a.n_zeta != b.n_zeta) {
            retire(ctx, ctx->sreqs[ctx->active[i]], CTD_REQ_FAILED);
            return fail(CTD_EINVAL, "served requests must share one node grid");
        }
    }
    int max_n_mat = 0;
    for (int i = 0; i < n; ++i) max_n_mat = std::max(max_n_mat, static_cast<int>(ps[i]->mats.size()));
    int rc2;
    if ((rc2 = ctx->u_work.ensure(n))) return rc2;
    std::vector<ctd::RequestDesc> descs(n);
    std::vector<uint64_t> tiles(n + 1, 0);
    std::vector<ctd::FoldDesc> folds(n);
    for (int i = 0; i < n; ++i) {
        ServeReq &R = ctx->sreqs[ctx->active[i]];
        Phantom &P = *ps[i];
        const uint64_t B = R.req.batch_histories;
        ctd::RequestDesc &q = descs[i];
        fill_request(P, R.req.seed, q);
        q.work = ctx->u_work.p + i;
        q.pref = P.pref.p + 1 * (q.nbins + 1);    // batches of exactly B histories
        q.h_base = static_cast<uint64_t>(R.batches) * B;
        q.local_begin = 0;
        q.local_end = B;
        q.tally = P.tally.p;
        tiles[i + 1] = tiles[i] + (P.nvox + ctd::kFoldTile - 1) / ctd::kFoldTile;
        ctd::FoldDesc &f = folds[i];
        f.tally = P.tally.p;
        f.rho = P.rho.p;
        f.sum_d = P.sum_d.p;
        f.sum_d2 = P.sum_d2.p;
        f.edep = P.edep.p;
        f.nvox = P.nvox;
        f.scale = ctd::kKevToJ * 1000.0 / (P.dx * P.dy * P.dz * static_cast<double>(B));
    }
    // one batch of every running request; those past min_batches also get their
    // statistics for the stopping test
    std::vector<int> checked;
    for (int i = 0; i < n; ++i) {
        ServeReq &R = ctx->sreqs[ctx->active[i]];
        R.batches += 1;
        R.histories += R.req.batch_histories;
        if (R.batches >= R.req.min_batches) checked.push_back(i);
    }
    auto stats = [&](int i, cudaStream_t s) {
        Phantom &P = *ps[i];
        const int nb = ctx->sreqs[ctx->active[i]].batches;
        int e = ctd::launch_finalize(P.sum_d.p, P.sum_d2.p, nb, P.dose.p, P.sd.p, P.nvox, s);
        if (e == CTD_OK) e = ctd::launch_rsd(P.dose.p, P.sd.p, P.rho.p, P.nvox, P.partials.p, kRsdParts, P.result.p, s);
        return e;
    };
    if (!ctx->shared_launch) {
        // each request on its own stream: transport, fold, statistics
        if ((rc = ensure_lanes(ctx, n))) return rc;
        CK(cudaMemsetAsync(ctx->u_work.p, 0, n * sizeof(unsigned long long), ctx->stream));
        if ((rc = fork_lanes(ctx, ctx->stream, n))) return rc;
        size_t c = 0;
        for (int i = 0; i < n; ++i) {
            Phantom &P = *ps[i];
            const cudaStream_t s = lane(ctx, i);
            CKS(launch_one(ctx, P, descs[i], s));
            CKS(ctd::launch_fold(P.tally.p, P.rho.p, P.sum_d.p, P.sum_d2.p, P.edep.p, P.nvox, folds[i].scale, s));
            if (c < checked.size() && checked[c] == i) {
                CKS(stats(i, s));
                ++c;
            }
        }
        if ((rc = join_lanes(ctx, ctx->stream, n))) return rc;
    } else {
        if ((rc = ctx->u_reqs.ensure(n)) || (rc = ctx->u_folds.ensure(n)) || (rc = ctx->u_tiles.ensure(n + 1)))
            return rc;
        CK(cudaMemcpyAsync(ctx->u_reqs.p, descs.data(), n * sizeof(ctd::RequestDesc), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->u_folds.p, folds.data(), n * sizeof(ctd::FoldDesc), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->u_tiles.p, tiles.data(), (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaMemsetAsync(ctx->u_work.p, 0, n * sizeof(unsigned long long), ctx->stream));
        ctd::LaunchParams L;
        std::memset(&L, 0, sizeof(L));
        fill_shared(*ps[0], L.sh);
        L.sh.max_n_mat = max_n_mat;
        L.reqs = ctx->u_reqs.p;
        L.n_req = n;
        L.chunk = ctx->chunk;
        L.flight_cap = ctx->flight_cap;
        const int mgrid = ctx->num_sms * ctx->multi_blocks_per_sm;
        CKS(ctd::launch_transport(L, mgrid, ctx->threads, ctx->threads * ctx->multi_blocks_per_sm, ctx->stream));
        CKS(ctd::launch_fold_multi(ctx->u_folds.p, ctx->u_tiles.p, n, tiles[n], ctx->stream));
        for (int i : checked) CKS(stats(i, ctx->stream));
    }
    std::vector<std::array<double, 3>> res(checked.size());
    for (size_t c = 0; c < checked.size(); ++c)
        CK(cudaMemcpyAsync(res[c].data(), ps[checked[c]]->result.p, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<int64_t> finished;
    for (size_t c = 0; c < checked.size(); ++c) {
        ServeReq &R = ctx->sreqs[ctx->active[checked[c]]];
        R.avg_rsd = res[c][0];
        R.sigma_bar = res[c][1];
        const bool hit = R.req.rsd_target > 0.0 && R.avg_rsd > 0.0 && R.avg_rsd <= R.req.rsd_target;
        const bool cap = R.req.n_histories_max && R.histories >= R.req.n_histories_max;
        if (hit || cap) finished.push_back(R.id);
    }
    std::vector<Phantom *> fp;
    std::vector<double> ft;
    for (int64_t id : finished) {
        ServeReq &R = ctx->sreqs[id];
        Phantom &P = *find(ctx, R.ph);
        CKS(ctd::launch_sum(P.edep.p, P.nvox, P.partials.p + 5 * kRsdParts, kRsdParts, P.result.p + 3, ctx->stream));
        fp.push_back(&P);
        ft.push_back(R.t_start);
    }
    if (!fp.empty() && (rc = collect_many(ctx, fp.data(), static_cast<int>(fp.size()), 0, 0.0, ft.data()))) return rc;
    for (size_t i = 0; i < finished.size(); ++i) {
        ServeReq &R = ctx->sreqs[finished[i]];
        fp[i]->stats.histories = R.histories;
        fp[i]->stats.n_batches = R.batches;
        fp[i]->have_result = true;
        retire(ctx, R, CTD_REQ_DONE);
    }
    if (n_active) *n_active = static_cast<int>(ctx->active.size() + ctx->pending.size());
    return CTD_OK;
}

int ctd_poll(ctd_ctx *ctx, ctd_req_id id, ctd_req_status *out)
{
    if (!ctx) return fail(CTD_EINVAL, "null context");
    auto it = ctx->sreqs.find(id);
    if (it == ctx->sreqs.end()) return fail(CTD_ENOTFOUND, "unknown request %lld", static_cast<long long>(id));
    if (out) {
        const ServeReq &R = it->second;
        out->state = R.state;
        out->batches = R.batches;
        out->histories = R.histories;
        out->avg_rsd = R.avg_rsd;
        out->paper_sigma_bar = R.sigma_bar;
        const double now = now_s();
        out->t_queued_s = (R.state == CTD_REQ_QUEUED ? now : (R.t_start > 0 ? R.t_start : now)) - R.t_submit;
        out->t_latency_s = (R.state >= CTD_REQ_DONE ? R.t_done : now) - R.t_submit;
    }
    return CTD_OK;
}

int ctd_wait(ctd_ctx *ctx, ctd_req_id id, double timeout_s, ctd_req_status *out)
{
    int rc;
    if (!ctx) return fail(CTD_EINVAL, "null context");
    if (ctx->sreqs.find(id) == ctx->sreqs.end())
        return fail(CTD_ENOTFOUND, "unknown request %lld", static_cast<long long>(id));
    const double t0 = now_s();
    for (;;) {
        const ServeReq &R = ctx->sreqs[id];
        if (R.state >= CTD_REQ_DONE) break;
        if (elapsed_since(t0) > timeout_s) {
            if (out) ctd_poll(ctx, id, out);
            return fail(CTD_ETIMEOUT, "request %lld not finished after %.3f s", static_cast<long long>(id), timeout_s);
        }
        const size_t before = ctx->active.size();
        if ((rc = ctd_serve_step(ctx, nullptr))) return rc;
        if (before == 0 && ctx->active.empty() && ctx->sreqs[id].state == CTD_REQ_QUEUED)
            return fail(CTD_ENOMEM, "request %lld cannot be admitted: not enough free device memory",
                        static_cast<long long>(id));
    }
    const ServeReq &R = ctx->sreqs[id];
    if (out) ctd_poll(ctx, id, out);
    if (R.state == CTD_REQ_CANCELLED) return fail(CTD_ECANCELLED, "request was cancelled");
    if (R.state == CTD_REQ_FAILED) return fail(CTD_ECUDA, "request failed");
    return CTD_OK;
}

int ctd_cancel(ctd_ctx *ctx, ctd_req_id id)
{
    if (!ctx) return fail(CTD_EINVAL, "null context");
    auto it = ctx->sreqs.find(id);
    if (it == ctx->sreqs.end()) return fail(CTD_ENOTFOUND, "unknown request %lld", static_cast<long long>(id));
    ServeReq &R = it->second;
    if (R.state == CTD_REQ_QUEUED) {
        for (size_t i = 0; i < ctx->pending.size(); ++i)
            if (ctx->pending[i] == id) {
                ctx->pending.erase(ctx->pending.begin() + i);
                break;
            }
        R.state = CTD_REQ_CANCELLED;
        R.t_done = now_s();
        Phantom *P = find(ctx, R.ph);
        if (P) P->busy_req = 0;
    } else if (R.state == CTD_REQ_RUNNING) {
        R.cancel = true;
    }
    return CTD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner
extern "C" {

int ctd_probe_memory(ctd_ctx *ctx, int kind, uint64_t n_slots, uint64_t n_ops, double *ops_per_s)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (kind < 0 || kind > 2 || n_slots < 1 || n_slots >= (1ull << 32) || n_ops < 1 || n_ops > (1ull << 40) ||
        !ops_per_s)
        return fail(CTD_EINVAL, "probe: kind 0-2, 1 <= n_slots < 2^32, 1 <= n_ops <= 2^40");
    const int block = 256, grid = ctx->num_sms * 8;
    const uint64_t per_round = static_cast<uint64_t>(grid) * block * 8;
    const uint64_t rounds64 = (n_ops + per_round - 1) / per_round;
    // operation indices are 32-bit
    if (rounds64 * per_round >= (1ull << 32)) return fail(CTD_EINVAL, "probe: n_ops too large for one launch");
    const uint32_t rounds = static_cast<uint32_t>(rounds64);
    DevBuf<double> dbuf;
    DevBuf<float> fbuf, out;
    DevBuf<uint8_t> mbuf;
    if (kind == 0) rc = dbuf.ensure(n_slots);
    else rc = fbuf.ensure(n_slots);
    if (!rc && kind == 2) rc = mbuf.ensure(n_slots);
    if (!rc && kind != 0) rc = out.ensure(static_cast<size_t>(grid) * block);
    if (rc) return rc;
    if (kind == 0) CK(cudaMemsetAsync(dbuf.p, 0, n_slots * sizeof(double), ctx->stream));
    if (kind != 0) CK(cudaMemsetAsync(fbuf.p, 0, n_slots * sizeof(float), ctx->stream));
    if (kind == 2) CK(cudaMemsetAsync(mbuf.p, 0, n_slots, ctx->stream));
    if (!event_at(ctx, 0) || !event_at(ctx, 1)) return fail(CTD_ECUDA, "cudaEventCreate failed");
    const uint32_t n32 = static_cast<uint32_t>(n_slots);
    CKS(ctd::launch_probe(kind, dbuf.p, fbuf.p, mbuf.p, out.p, n32, rounds, 0x9E3779B9u, grid, block, ctx->stream));
    double t = 0.0;
    for (int k = 0; k < 3; ++k) {
        CK(cudaEventRecord(ctx->events[0], ctx->stream));
        CKS(ctd::launch_probe(kind, dbuf.p, fbuf.p, mbuf.p, out.p, n32, rounds, 0x85EBCA6Bu * (k + 1), grid, block,
                              ctx->stream));
        CK(cudaEventRecord(ctx->events[1], ctx->stream));
        CK(cudaEventSynchronize(ctx->events[1]));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->events[0], ctx->events[1]));
        t += ms * 1e-3;
    }
    *ops_per_s = 3.0 * static_cast<double>(rounds) * static_cast<double>(per_round) / t;
    return CTD_OK;
}

int ctd_autotune(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_probe, uint64_t seed, ctd_tune_result *out)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if ((rc = busy(P))) return rc;
    if (n_probe < 1000) return fail(CTD_EINVAL, "n_probe must be at least 1000");
    const uint64_t n = 10 * n_probe;
    if ((rc = prepare_run(ctx, *P, n, 10))) return rc;
    P->have_result = false;
    ctd::RequestDesc q;
    fill_request(*P, seed, q);
    const int old_bps = ctx->blocks_per_sm, old_chunk = ctx->chunk, old_cap = ctx->flight_cap,
              old_threads = ctx->threads;
    struct Shape {
        int threads, bps, chunk, cap;
    };
    std::vector<Shape> shapes;
    shapes.push_back({old_threads, old_bps, old_chunk, old_cap});
    // blocks of 256 threads, 3 or 4 per SM, or of 128 threads, 7 or 8 per SM
    const int blocks[4][2] = {{256, 3}, {256, 4}, {128, 7}, {128, 8}};
    for (const auto &b : blocks)
        for (int chunk : {64, 256, 1024})
            for (int cap : {1, 2, 4, 8})
                if (!(b[0] == old_threads && b[1] == old_bps && chunk == old_chunk && cap == old_cap))
                    shapes.push_back({b[0], b[1], chunk, cap});
    double best = 1e300, base = 0.0;
    Shape pick = shapes[0];
    for (size_t k = 0; k < shapes.size(); ++k) {
        ctx->threads = shapes[k].threads;
        ctx->blocks_per_sm = shapes[k].bps;
        ctx->chunk = shapes[k].chunk;
        ctx->flight_cap = shapes[k].cap;
        double t_min = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
            if ((rc = transport(ctx, *P, q, 0, 0, 0, n_probe, P->tally.p, 0))) {
                ctx->threads = old_threads;
                ctx->blocks_per_sm = old_bps;
                ctx->chunk = old_chunk;
                ctx->flight_cap = old_cap;
                return rc;
            }
            CK(cudaStreamSynchronize(ctx->stream));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ctx->events[0], ctx->events[1]));
            t_min = std::min(t_min, static_cast<double>(ms) * 1e-3);
        }
        if (k == 0) base = t_min;
        if (t_min < best) {
            best = t_min;
            pick = shapes[k];
        }
    }
    CK(cudaMemsetAsync(P->tally.p, 0, P->nvox * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->threads = pick.threads;
    ctx->blocks_per_sm = pick.bps;
    ctx->chunk = pick.chunk;
    ctx->flight_cap = pick.cap;
    if (out) {
        out->threads_per_block = pick.threads;
        out->blocks_per_sm = pick.bps;
        out->chunk = pick.chunk;
        out->flight_cap = pick.cap;
        out->n_tried = static_cast<int>(shapes.size());
        out->histories_per_s = static_cast<double>(n_probe) / best;
        out->baseline_per_s = static_cast<double>(n_probe) / base;
    }
    return CTD_OK;
}

}  // extern "C"
