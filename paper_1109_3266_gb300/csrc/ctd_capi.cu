// ctd_capi.cu -- the C ABI of include/ctd.h: contexts, resident phantoms,
// source/spectrum/fluence/physics set-up, the plain form (the batch loop of
// Sec. 2.2.1) and results.  The batched and served forms are in ctd_forms.cu,
// the launch-shape search and the memory probes in ctd_tune.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "ctd_host.h"

namespace ctd {
namespace host {

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
const std::vector<float> &angular_surface(ctd_ctx *ctx, int kind, double q0, const ctd::Elements *el, int e_min, int n_e,
                                         int n_zeta)
{
    std::vector<double> key{static_cast<double>(kind), (kind == 1 || kind == 2) && q0 > 0.0 ? q0 : 0.0,
                            static_cast<double>(e_min), static_cast<double>(n_e), static_cast<double>(n_zeta)};
    if (kind == 3)
        for (int i = 0; i < el->n; ++i) {
            key.push_back(static_cast<double>(el->z[i]));
            key.push_back(el->count[i]);
        }
    auto it = ctx->surfaces.find(key);
    if (it != ctx->surfaces.end()) return it->second;
    if (ctx->surfaces.size() >= 64) ctx->surfaces.clear();
    const size_t row = static_cast<size_t>(n_e) * n_zeta;
    std::vector<double> tmp(row);
    ctd::build_surface(kind, q0, el, e_min, n_e, n_zeta, tmp.data());
    std::vector<float> f(row);
    for (size_t i = 0; i < row; ++i) f[i] = static_cast<float>(tmp[i]);
    return ctx->surfaces.emplace(key, std::move(f)).first->second;
}

// Surfaces [k][n_e][n_zeta] as cells [k][n_e - 1][n_zeta - 1][4]: the corners
// S[j][i], S[j][i+1], S[j+1][i], S[j+1][i+1] of the bilinear lookup in cell (j, i)
static std::vector<float> surface_cells(const std::vector<float> &rows, int n_e, int n_zeta)
{
    const size_t row = static_cast<size_t>(n_e) * n_zeta;
    const size_t cells = static_cast<size_t>(n_e - 1) * (n_zeta - 1);
    const size_t k_max = rows.size() / row;
    std::vector<float> out(k_max * cells * 4);
    for (size_t k = 0; k < k_max; ++k)
        for (int j = 0; j + 1 < n_e; ++j)
            for (int i = 0; i + 1 < n_zeta; ++i) {
                const float *r0 = &rows[k * row + static_cast<size_t>(j) * n_zeta + i];
                const float *r1 = r0 + n_zeta;
                float *o = &out[((k * (n_e - 1) + j) * (n_zeta - 1) + i) * 4];
                o[0] = r0[0];
                o[1] = r0[1];
                o[2] = r1[0];
                o[3] = r1[1];
            }
    return out;
}

// One material's node-table columns, from the context's cache
static const std::vector<double> &material_columns(ctd_ctx *ctx, const ctd_material &mat, const ctd::Elements &el,
                                                   int e_min, int n_e, int compton_model)
{
    std::vector<double> key{static_cast<double>(compton_model), static_cast<double>(e_min), static_cast<double>(n_e),
                            mat.z_over_a, mat.a_mol, mat.z_eff, mat.q0, mat.sq0, static_cast<double>(el.n)};
    for (int i = 0; i < el.n; ++i) {
        key.push_back(static_cast<double>(el.z[i]));
        key.push_back(el.count[i]);
    }
    auto it = ctx->columns.find(key);
    if (it != ctx->columns.end()) return it->second;
    if (ctx->columns.size() >= 256) ctx->columns.clear();
    std::vector<double> col(static_cast<size_t>(n_e) * 3);
    ctd::material_columns(mat, el, e_min, n_e, compton_model, col.data());
    return ctx->columns.emplace(std::move(key), std::move(col)).first->second;
}

int build_tables(ctd_ctx *ctx, Phantom &P)
{
    if (P.tables_ok) return CTD_OK;
    const ctd_physics &ph = P.phys;
    const int n_e = ph.e_max_kev - ph.e_min_kev + 1;
    const int nm = static_cast<int>(P.mats.size());
    std::vector<double> cum(static_cast<size_t>(nm) * n_e * 3), mmax;
    for (int m = 0; m < nm; ++m) {
        const std::vector<double> &col = material_columns(ctx, P.mats[m], P.els[m], ph.e_min_kev, n_e, ph.compton_model);
        std::copy(col.begin(), col.end(), cum.begin() + static_cast<size_t>(m) * n_e * 3);
    }
    ctd::build_majorant(cum, P.rho_max, P.present, n_e, ph.majorant_scale, mmax);
    P.h_tab.assign(static_cast<size_t>(nm) * n_e * 4, 0.0f);
    for (size_t i = 0; i < static_cast<size_t>(nm) * n_e; ++i)
        for (int c = 0; c < 3; ++c) P.h_tab[i * 4 + c] = static_cast<float>(cum[i * 3 + c]);
    // fourth column: c3 at the next node minus c3 here, the binary32 difference the
    // interpolation of the total share takes (0 at the last node)
    for (int m = 0; m < nm; ++m)
        for (int j = 0; j + 1 < n_e; ++j) {
            const size_t i = static_cast<size_t>(m) * n_e + j;
            P.h_tab[i * 4 + 3] = P.h_tab[(i + 1) * 4 + 2] - P.h_tab[i * 4 + 2];
        }
    P.h_mm.resize(n_e);
    for (int j = 0; j < n_e; ++j) P.h_mm[j] = static_cast<float>(mmax[j]);
    const size_t row = static_cast<size_t>(n_e) * ph.n_zeta;
    if (ph.compton_model == CTD_COMPTON_WH) {
        // one Waller-Hartree C surface per material
        P.h_cs.resize(row * nm);
        for (int m = 0; m < nm; ++m) {
            const std::vector<float> &c = angular_surface(ctx, 2, P.mats[m].sq0, nullptr, ph.e_min_kev, n_e, ph.n_zeta);
            std::copy(c.begin(), c.end(), P.h_cs.begin() + m * row);
        }
    } else {
        P.h_cs = angular_surface(ctx, 0, 0.0, nullptr, ph.e_min_kev, n_e, ph.n_zeta);
    }
    P.h_rs.resize(row * nm);
    for (int m = 0; m < nm; ++m) {
        const std::vector<float> &r = P.els[m].n > 0
                                          ? angular_surface(ctx, 3, 0.0, &P.els[m], ph.e_min_kev, n_e, ph.n_zeta)
                                          : angular_surface(ctx, 1, P.mats[m].q0, nullptr, ph.e_min_kev, n_e, ph.n_zeta);
        std::copy(r.begin(), r.end(), P.h_rs.begin() + m * row);
    }
    // the device holds each surface as cells of the four corners of a bilinear lookup
    const std::vector<float> cs_cells = surface_cells(P.h_cs, n_e, ph.n_zeta);
    const std::vector<float> rs_cells = surface_cells(P.h_rs, n_e, ph.n_zeta);
    int rc;
    if ((rc = P.tab.ensure(P.h_tab.size())) || (rc = P.mm.ensure(n_e)) || (rc = P.cs.ensure(cs_cells.size())) ||
        (rc = P.rs.ensure(rs_cells.size())))
        return rc;
    CK(cudaMemcpyAsync(P.tab.p, P.h_tab.data(), P.h_tab.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P.mm.p, P.h_mm.data(), n_e * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P.cs.p, cs_cells.data(), cs_cells.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P.rs.p, rs_cells.data(), rs_cells.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
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
        (rc = P.work.ensure(2)))
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
    q.vox = P.vox.p;
    q.unused = nullptr;
    q.tab = P.tab.p;
    q.mmax = P.mm.p;
    q.rsurf = P.rs.p;
    q.csurf = P.cs.p;
    q.cs_stride = P.phys.compton_model == CTD_COMPTON_WH ? (P.n_e - 1) * (P.phys.n_zeta - 1) : 0;
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
    q.fnx = static_cast<float>(P.nx);
    q.fny = static_cast<float>(P.ny);
    q.fnz = static_cast<float>(P.nz);
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

// The second stream, its events and the phantom's second tally of an overlapped plain run.
int ensure_plain_aux(ctd_ctx *ctx, Phantom &P)
{
    if (!ctx->plain_aux) CK(cudaStreamCreateWithFlags(&ctx->plain_aux, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&ctx->plain_fork, &ctx->plain_fold[0], &ctx->plain_fold[1]})
        if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return P.tally2.ensure(P.nvox);
}

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
              uint64_t le, double *tally, size_t ev_index, uint4 *trace, uint64_t trace_h0, uint64_t trace_n,
              cudaStream_t s, unsigned long long *work)
{
    if (!s) s = ctx->stream;
    if (!work) work = P.work.p;
    ctd::LaunchParams L;
    std::memset(&L, 0, sizeof(L));
    L.trace = trace;
    L.trace_h0 = trace_h0;
    L.trace_n = trace_n;
    fill_shared(P, L.sh);
    q.pref = P.pref.p + which_size * (q.nbins + 1);
    q.h_base = h_base;
    q.local_begin = lb;
    q.local_end = le;
    q.tally = tally;
    q.work = work;
    L.one = q;
    L.chunk = ctx->chunk;
    L.flight_cap = ctx->flight_cap;
    CK(cudaMemsetAsync(work, 0, sizeof(unsigned long long), s));
    cudaEvent_t e0 = event_at(ctx, 2 * ev_index), e1 = event_at(ctx, 2 * ev_index + 1);
    if (!e0 || !e1) return fail(CTD_ECUDA, "cudaEventCreate failed");
    CK(cudaEventRecord(e0, s));
    const int grid = ctx->num_sms * ctx->blocks_per_sm;
    ctd::L2Window win{};
    if (ctx->l2_persist) {
        // the tally's (or the voxel words') lines stay in L2
        win.base = ctx->l2_persist == 1 ? static_cast<void *>(tally) : static_cast<void *>(P.vox.p);
        win.bytes = std::min(P.nvox * (ctx->l2_persist == 1 ? sizeof(double) : sizeof(uint32_t)), ctx->l2_window_max);
        // a set-aside of the window's size, no more: the rest of L2 stays for the other data
        const size_t want = std::min(win.bytes, ctx->l2_persist_max);
        if (want != ctx->l2_asked) {
            ctx->l2_asked = want;
            CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
            CK(cudaDeviceGetLimit(&ctx->l2_setaside, cudaLimitPersistingL2CacheSize));
        }
        win.hit_ratio = static_cast<float>(std::min(1.0, static_cast<double>(ctx->l2_setaside) / win.bytes));
    }
    CKS(ctd::launch_transport(L, grid, ctx->threads, ctx->threads * ctx->blocks_per_sm, s,
                              ctx->l2_persist ? &win : nullptr));
    CK(cudaEventRecord(e1, s));
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
                 const double *t0_each, cudaStream_t stream)
{
    const cudaStream_t cs = stream ? stream : ctx->stream;
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
                           cs));
        CK(cudaMemcpyAsync(ctx->staged[i].res, ps[i]->result.p, sizeof(ctx->staged[i].res), cudaMemcpyDeviceToHost,
                           cs));
    }
    CK(cudaStreamSynchronize(cs));
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

}  // namespace host

void set_error(const char *msg) { host::g_error = msg; }

}  // namespace ctd

using namespace ctd::host;

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
        if (opt->serve_reserve_bytes > 0) ctx->reserve_bytes = opt->serve_reserve_bytes;
        if (opt->threads_per_block > 0) ctx->threads = opt->threads_per_block;
        if (opt->chunk > 0) ctx->chunk = opt->chunk;
        if (opt->flight_cap > 0) ctx->flight_cap = opt->flight_cap;
        ctx->shared_launch = opt->shared_launch != 0;
        ctx->l2_persist = opt->l2_persist > 0 ? opt->l2_persist : 0;
        ctx->plain_overlap = opt->plain_overlap > 0;
        if (opt->batch_lanes < 0 || opt->batch_lanes > kMaxLanes) return fail(CTD_EINVAL, "batch_lanes must be 0..64");
        if (opt->batch_lanes > 0) ctx->batch_lanes = opt->batch_lanes;
        if (ctx->l2_persist > 2) return fail(CTD_EINVAL, "l2_persist must be -1, 0, 1 or 2");
    }
    if (ctx->threads % 32 != 0 || ctx->threads > 256) return fail(CTD_EINVAL, "threads_per_block must be a multiple of 32 and at most 256");
    if (ctx->blocks_per_sm > 64 || ctx->multi_blocks_per_sm > 64) return fail(CTD_EINVAL, "blocks_per_sm at most 64");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (ctx->device < 0 || ctx->device >= ndev) return fail(CTD_EINVAL, "device %d out of range (%d devices)", ctx->device, ndev);
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (ctx->l2_persist) {
        // the largest persisting set-aside the device grants, for this context's lifetime
        int max_persist = 0, max_window = 0;
        CK(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device));
        CK(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device));
        CK(cudaDeviceGetLimit(&ctx->l2_prev_limit, cudaLimitPersistingL2CacheSize));
        ctx->l2_persist_max = static_cast<size_t>(std::max(max_persist, 0));
        ctx->l2_window_max = static_cast<size_t>(std::max(max_window, 0));
        if (!ctx->l2_persist_max || !ctx->l2_window_max) ctx->l2_persist = 0;
    }
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
    for (auto l : ctx->lanes) cudaStreamSynchronize(l);
    for (auto l : ctx->serve_hi) cudaStreamSynchronize(l);
    ctx->phantoms.clear();
    if (ctx->l2_persist) {
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, ctx->l2_prev_limit);
    }
    if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
    for (auto e : ctx->events) cudaEventDestroy(e);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (auto l : ctx->lanes) cudaStreamDestroy(l);
    for (auto e : ctx->lane_done) cudaEventDestroy(e);
    if (ctx->fork_event) cudaEventDestroy(ctx->fork_event);
    for (auto e : ctx->serve_ev) cudaEventDestroy(e);
    for (auto e : ctx->serve_ev_pre) cudaEventDestroy(e);
    if (ctx->plain_aux) {
        cudaStreamSynchronize(ctx->plain_aux);
        cudaStreamDestroy(ctx->plain_aux);
    }
    for (cudaEvent_t e : {ctx->plain_fork, ctx->plain_fold[0], ctx->plain_fold[1]})
        if (e) cudaEventDestroy(e);
    for (auto l : ctx->serve_hi) cudaStreamDestroy(l);
    if (ctx->serve_res) cudaFreeHost(ctx->serve_res);
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
    // voxel indices are 32-bit on the device
    if (nvox >= (static_cast<size_t>(1) << 32)) return fail(CTD_EINVAL, "phantom too large (2^32 voxels or more)");
    std::unique_ptr<Phantom> P(new Phantom());
    P->use_cache(&ctx->buffers);
    P->nx = nx; P->ny = ny; P->nz = nz;
    P->dx = dx; P->dy = dy; P->dz = dz;
    P->nvox = nvox;
    P->mats.assign(mats, mats + n_mat);
    P->els.assign(static_cast<size_t>(n_mat), ctd::Elements{});
    P->rho_max.assign(n_mat, 0.0);
    P->present.assign(n_mat, 0);
    P->phys.e_min_kev = 1;
    P->phys.e_max_kev = 150;
    P->phys.n_zeta = 1024;
    P->phys.majorant_scale = 1.0;
    P->phys.mode = CTD_MODE_FULL;
    P->phys.max_real = 0;
    P->phys.compton_model = CTD_COMPTON_KN;
    if ((rc = P->mat.ensure(nvox)) || (rc = P->rho.ensure(nvox)) || (rc = P->vox.ensure(nvox)) ||
        (rc = P->rinv.ensure(nvox)))
        return rc;
    CK(cudaMemcpyAsync(P->mat.p, mat, nvox, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P->rho.p, density, nvox * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    // range checks, materials present and their largest densities, on the device
    DevBuf<ctd::PhantomScan> scan;
    if ((rc = scan.ensure(1))) return rc;
    CKS(ctd::launch_scan_phantom(P->mat.p, P->rho.p, nvox, n_mat, P->vox.p, P->rinv.p, scan.p, ctx->stream));
    ctd::PhantomScan sc{};
    CK(cudaMemcpyAsync(&sc, scan.p, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (sc.first_bad_mat != ~0ull && sc.first_bad_mat <= sc.first_bad_rho)
        return fail(CTD_EINVAL, "voxel %llu has material %d >= n_mat", sc.first_bad_mat,
                    static_cast<int>(mat[sc.first_bad_mat]));
    if (sc.first_bad_rho != ~0ull)
        return fail(CTD_EINVAL, "voxel %llu has density %g: densities must be 0 or in [2^-18, 2^13) g/cm^3",
                    sc.first_bad_rho, static_cast<double>(density[sc.first_bad_rho]));
    for (int m = 0; m < n_mat; ++m) {
        P->present[m] = static_cast<int>(sc.present_mask >> m & 1u);
        float r;
        std::memcpy(&r, &sc.max_bits[m], sizeof(r));
        P->rho_max[m] = P->present[m] ? static_cast<double>(r) : 0.0;
    }
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

int ctd_set_material_elements(ctd_ctx *ctx, ctd_phantom ph, int material, int n_el, const int *z,
                              const double *count)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if ((rc = busy(P))) return rc;
    if (material < 0 || material >= static_cast<int>(P->mats.size())) return fail(CTD_EINVAL, "material out of range");
    if (n_el < 0 || n_el > CTD_MAX_ELEMENTS) return fail(CTD_EINVAL, "n_el must be 0..%d", CTD_MAX_ELEMENTS);
    if (n_el > 0 && (!z || !count)) return fail(CTD_EINVAL, "null element arrays");
    ctd::Elements el;
    el.n = n_el;
    for (int i = 0; i < n_el; ++i) {
        if (z[i] < 1 || z[i] > 100) return fail(CTD_EINVAL, "atomic number %d out of 1..100", z[i]);
        if (!(count[i] > 0.0) || !std::isfinite(count[i])) return fail(CTD_EINVAL, "atom counts must be finite and > 0");
        el.z[i] = z[i];
        el.count[i] = count[i];
    }
    P->els[material] = el;
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

int ctd_spectrum_kramers(int kvp, double mm_al, int e_min, double *e_lo, double *e_hi, double *w, int *nbins)
{
    g_error.clear();
    if (e_min < 1 || kvp <= e_min || kvp > 100000 || !(mm_al >= 0.0) || !std::isfinite(mm_al) || !nbins)
        return fail(CTD_EINVAL, "need 1 <= e_min < kvp <= 100000 and mm_al >= 0");
    *nbins = kvp - e_min;
    for (int j = 0; j < *nbins; ++j) {
        const double lo = static_cast<double>(e_min + j), mid = lo + 0.5;
        const double mu_al = 26300.0 / (mid * mid * mid) + 0.15;
        if (e_lo) e_lo[j] = lo;
        if (e_hi) e_hi[j] = lo + 1.0;
        if (w) w[j] = (static_cast<double>(kvp) - mid) / mid * std::exp(-mu_al * 2.699 * (mm_al / 10.0));
    }
    return CTD_OK;
}

// elements of ctd_material_columns / ctd_angular_surface, checked as in ctd_set_material_elements
static int host_elements(int n_el, const int *z, const double *count, ctd::Elements &el)
{
    if (n_el < 0 || n_el > CTD_MAX_ELEMENTS) return fail(CTD_EINVAL, "n_el must be 0..%d", CTD_MAX_ELEMENTS);
    if (n_el > 0 && (!z || !count)) return fail(CTD_EINVAL, "null element arrays");
    el.n = n_el;
    for (int i = 0; i < n_el; ++i) {
        if (z[i] < 1 || z[i] > 100) return fail(CTD_EINVAL, "atomic number %d out of 1..100", z[i]);
        if (!(count[i] > 0.0) || !std::isfinite(count[i])) return fail(CTD_EINVAL, "atom counts must be finite and > 0");
        el.z[i] = z[i];
        el.count[i] = count[i];
    }
    return CTD_OK;
}

static int host_grid(const ctd_material *mat, int e_min_kev, int e_max_kev, const double *out)
{
    if (!mat || !out) return fail(CTD_EINVAL, "null pointer argument");
    if (!(mat->z_over_a > 0 && mat->a_mol > 0 && mat->z_eff > 0) || !std::isfinite(mat->q0) || !std::isfinite(mat->sq0))
        return fail(CTD_EINVAL, "material has non-positive or non-finite parameters");
    if (e_min_kev < 1 || e_max_kev <= e_min_kev || e_max_kev > 100000)
        return fail(CTD_EINVAL, "node grid must satisfy 1 <= e_min < e_max <= 100000");
    return CTD_OK;
}

int ctd_material_columns(const ctd_material *mat, int n_el, const int *z, const double *count, int e_min_kev,
                         int e_max_kev, int compton_model, double *out)
{
    g_error.clear();
    int rc;
    ctd::Elements el;
    if ((rc = host_grid(mat, e_min_kev, e_max_kev, out)) || (rc = host_elements(n_el, z, count, el))) return rc;
    if (compton_model != CTD_COMPTON_KN && compton_model != CTD_COMPTON_WH) return fail(CTD_EINVAL, "unknown Compton model");
    ctd::material_columns(*mat, el, e_min_kev, e_max_kev - e_min_kev + 1, compton_model, out);
    return CTD_OK;
}

int ctd_angular_surface(int kind, const ctd_material *mat, int n_el, const int *z, const double *count,
                        int e_min_kev, int e_max_kev, int n_zeta, double *out)
{
    g_error.clear();
    int rc;
    ctd::Elements el;
    if ((rc = host_grid(mat, e_min_kev, e_max_kev, out)) || (rc = host_elements(n_el, z, count, el))) return rc;
    if (n_zeta < 2 || n_zeta > (1 << 20)) return fail(CTD_EINVAL, "n_zeta must be 2..2^20");
    const int n_e = e_max_kev - e_min_kev + 1;
    switch (kind) {
    case 0: ctd::build_surface(0, 0.0, nullptr, e_min_kev, n_e, n_zeta, out); break;
    case 1:
        if (el.n > 0) ctd::build_surface(3, 0.0, &el, e_min_kev, n_e, n_zeta, out);
        else ctd::build_surface(1, mat->q0, nullptr, e_min_kev, n_e, n_zeta, out);
        break;
    case 2: ctd::build_surface(2, mat->sq0, nullptr, e_min_kev, n_e, n_zeta, out); break;
    default: return fail(CTD_EINVAL, "kind is 0 (Klein-Nishina C), 1 (R) or 2 (Waller-Hartree C)");
    }
    return CTD_OK;
}

int ctd_allocate_histories(uint64_t n, int nbins, const double *w, uint64_t *out)
{
    g_error.clear();
    if (!w || !out || nbins < 1) return fail(CTD_EINVAL, "need weights, output and nbins >= 1");
    const std::vector<double> wv(w, w + nbins);
    std::vector<uint64_t> o;
    if (!ctd::allocate(n, wv, o)) return fail(CTD_EINVAL, "weights must be finite, >= 0, not all zero, with a finite sum");
    std::copy(o.begin(), o.end(), out);
    return CTD_OK;
}

int ctd_alias_table(int n, const double *f, uint32_t *thr, int32_t *alias)
{
    g_error.clear();
    if (!f || !thr || !alias || n < 1) return fail(CTD_EINVAL, "need intensities, outputs and n >= 1");
    if (!ctd::alias_build(n, f, thr, alias)) return fail(CTD_EINVAL, "intensities must be finite, >= 0 and not all zero");
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
    const bool two = ctx->plain_overlap;
    if (two && (rc = ensure_plain_aux(ctx, *P))) return rc;
    CK(cudaMemsetAsync(P->tally.p, 0, nv * sizeof(double), ctx->stream));
    if (two) CK(cudaMemsetAsync(P->tally2.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->sum_d.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->sum_d2.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->edep.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
    ctd::RequestDesc T;
    fill_request(*P, seed, T);
    const uint64_t n_lo = n_histories / n_batches, rem = n_histories % n_batches;
    const double vol = P->dx * P->dy * P->dz;
    if (two) {
        CK(cudaEventRecord(ctx->plain_fork, ctx->stream));
        CK(cudaStreamWaitEvent(ctx->plain_aux, ctx->plain_fork, 0));
    }
    // With two streams, odd batches run on the second one with the second tally: a
    // batch's launch waits only for the fold two batches back (same stream, same
    // tally), so it starts while the previous batch drains; each fold waits for the
    // previous batch's fold, so Sigma d and Sigma d^2 add up in batch order.
    uint64_t h = 0;
    for (int b = 0; b < n_batches; ++b) {
        const uint64_t nb = static_cast<uint64_t>(b) < rem ? n_lo + 1 : n_lo;
        const int which = static_cast<uint64_t>(b) < rem ? 0 : 1;
        const int k = two ? b & 1 : 0;
        const cudaStream_t s = k ? ctx->plain_aux : ctx->stream;
        double *tally = k ? P->tally2.p : P->tally.p;
        if ((rc = transport(ctx, *P, T, which, h, 0, nb, tally, b, nullptr, 0, 0, s, P->work.p + k))) return rc;
        if (two && b > 0) CK(cudaStreamWaitEvent(s, ctx->plain_fold[k ^ 1], 0));
        // d = E / (m n_b) with m = rho V / 1000 kg
        const double scale = ctd::kKevToJ * 1000.0 / (vol * static_cast<double>(nb));
        CKS(ctd::launch_fold(tally, P->rinv.p, P->sum_d.p, P->sum_d2.p, P->edep.p, nv, scale, s));
        if (two) CK(cudaEventRecord(ctx->plain_fold[k], s));
        h += nb;
    }
    // the context's stream continues after the last fold (which followed every other)
    if (two && ((n_batches - 1) & 1)) CK(cudaStreamWaitEvent(ctx->stream, ctx->plain_fold[1], 0));
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

extern "C" {

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

int ctd_shard_begin(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (n_batches < 2 || static_cast<uint64_t>(n_batches) > n_histories)
        return fail(CTD_EINVAL, "need 2 <= n_batches <= n_histories");
    if ((rc = busy(P))) return rc;
    if ((rc = prepare_run(ctx, *P, n_histories, n_batches))) return rc;
    const size_t nv = P->nvox;
    CK(cudaMemsetAsync(P->sum_d.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->sum_d2.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->edep.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
    P->have_result = false;
    P->shard_n = n_histories;
    P->shard_nb = n_batches;
    P->shard_seed = seed;
    P->shard_t0 = now_s();
    return CTD_OK;
}

// batch b of the sharded run: its size, which allocation it uses, its first history
static void shard_batch_of(const Phantom &P, int b, uint64_t &size, int &which, uint64_t &h0)
{
    const uint64_t n_lo = P.shard_n / P.shard_nb, rem = P.shard_n % P.shard_nb;
    const uint64_t ub = static_cast<uint64_t>(b);
    size = ub < rem ? n_lo + 1 : n_lo;
    which = ub < rem ? 0 : 1;
    h0 = ub * n_lo + (ub < rem ? ub : rem);
}

int ctd_shard_batch(ctd_ctx *ctx, ctd_phantom ph, int batch, uint64_t local_begin, uint64_t local_end,
                    double *tally_dev)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (P->shard_nb == 0) return fail(CTD_EINVAL, "no sharded run begun on phantom %d", ph);
    if (batch < 0 || batch >= P->shard_nb) return fail(CTD_EINVAL, "batch %d outside [0, %d)", batch, P->shard_nb);
    if (!tally_dev) return fail(CTD_EINVAL, "null tally buffer");
    uint64_t size, h0;
    int which;
    shard_batch_of(*P, batch, size, which, h0);
    if (local_begin > local_end || local_end > size)
        return fail(CTD_EINVAL, "history range outside batch %d of %llu histories", batch,
                    static_cast<unsigned long long>(size));
    if (local_begin == local_end) return CTD_OK;
    ctd::RequestDesc T;
    fill_request(*P, P->shard_seed, T);
    return transport(ctx, *P, T, which, h0, local_begin, local_end, tally_dev, static_cast<size_t>(batch));
}

int ctd_shard_fold(ctd_ctx *ctx, ctd_phantom ph, int batch, double *tally_dev)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (P->shard_nb == 0) return fail(CTD_EINVAL, "no sharded run begun on phantom %d", ph);
    if (batch < 0 || batch >= P->shard_nb) return fail(CTD_EINVAL, "batch %d outside [0, %d)", batch, P->shard_nb);
    if (!tally_dev) return fail(CTD_EINVAL, "null tally buffer");
    uint64_t size, h0;
    int which;
    shard_batch_of(*P, batch, size, which, h0);
    // d = E / (m n_b) with m = rho V / 1000 kg
    const double scale = ctd::kKevToJ * 1000.0 / (P->dx * P->dy * P->dz * static_cast<double>(size));
    CKS(ctd::launch_fold(tally_dev, P->rinv.p, P->sum_d.p, P->sum_d2.p, P->edep.p, P->nvox, scale, ctx->stream));
    return CTD_OK;
}

int ctd_shard_counts(ctd_ctx *ctx, ctd_phantom ph, uint64_t *counts, double *energies)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!counts || !energies) return fail(CTD_EINVAL, "null output");
    ctd::DeviceCounts c;
    CK(cudaMemcpyAsync(&c, P->counts.p, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 10; ++i) counts[i] = c.n[i];
    energies[0] = ctd::fixed_kev(c.e_fix[0], c.e_fix[1]);
    energies[1] = ctd::fixed_kev(c.e_fix[2], c.e_fix[3]);
    return CTD_OK;
}

int ctd_shard_finish(ctd_ctx *ctx, ctd_phantom ph, const uint64_t *counts, const double *energies)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (P->shard_nb == 0) return fail(CTD_EINVAL, "no sharded run begun on phantom %d", ph);
    if (!counts || !energies) return fail(CTD_EINVAL, "null totals");
    CKS(finish_stats(*P, P->shard_nb, ctx->stream));
    if ((rc = collect(ctx, *P, 0, P->shard_t0))) return rc;
    ctd_run_stats &s = P->stats;
    s.pe = counts[ctd::kCntPe];
    s.compton = counts[ctd::kCntCompton];
    s.rayleigh = counts[ctd::kCntRayleigh];
    s.fictitious = counts[ctd::kCntFict];
    s.escaped = counts[ctd::kCntEscaped];
    s.missed = counts[ctd::kCntMissed];
    s.cutoff = counts[ctd::kCntCutoff];
    s.terminated = counts[ctd::kCntTerminated];
    s.aborted = counts[ctd::kCntAborted];
    s.steps = counts[ctd::kCntSteps];
    s.e_emitted_kev = energies[0];
    s.e_escaped_kev = energies[1];
    s.histories = P->shard_n;
    s.n_batches = P->shard_nb;
    P->have_result = true;
    P->shard_nb = 0;
    return CTD_OK;
}

int ctd_trace_range(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches,
                    uint64_t h_begin, uint64_t h_end, ctd_track *out)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    Phantom *P = find(ctx, ph);
    if (!P) return fail(CTD_ENOTFOUND, "unknown phantom %d", ph);
    if (!out && h_end > h_begin) return fail(CTD_EINVAL, "null output pointer");
    if (n_batches < 1 || static_cast<uint64_t>(n_batches) > n_histories)
        return fail(CTD_EINVAL, "need 1 <= n_batches <= n_histories");
    if (h_begin > h_end || h_end > n_histories) return fail(CTD_EINVAL, "history range outside [0, n_histories]");
    const uint64_t n = h_end - h_begin;
    if (n > kMaxTrace) return fail(CTD_EINVAL, "at most %llu histories per trace", static_cast<unsigned long long>(kMaxTrace));
    if ((rc = busy(P))) return rc;
    const double t0 = now_s();
    if ((rc = prepare_run(ctx, *P, n_histories, n_batches))) return rc;
    DevBuf<uint4> rec;
    if ((rc = rec.ensure(n))) return rc;
    const size_t nv = P->nvox;
    CK(cudaMemsetAsync(rec.p, 0, (n ? n : 1) * sizeof(uint4), ctx->stream));
    CK(cudaMemsetAsync(P->edep.p, 0, nv * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
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
            if ((rc = transport(ctx, *P, T, static_cast<uint64_t>(b) < rem ? 0 : 1, h, lo - h, hi - h, P->edep.p,
                                launches, rec.p, h_begin, n)))
                return rc;
            ++launches;
        }
        h += nb;
    }
    CK(cudaMemsetAsync(P->result.p, 0, 3 * sizeof(double), ctx->stream));
    CKS(ctd::launch_sum(P->edep.p, nv, P->partials.p + 5 * kRsdParts, kRsdParts, P->result.p + 3, ctx->stream));
    if (n) CK(cudaMemcpyAsync(out, rec.p, n * sizeof(ctd_track), cudaMemcpyDeviceToHost, ctx->stream));
    if ((rc = collect(ctx, *P, launches, t0))) return rc;
    P->stats.histories = n;
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
    const size_t cell_floats = static_cast<size_t>(P->n_e - 1) * (P->phys.n_zeta - 1) * 4;
    const float *surf = kind == 1 ? P->rs.p + material * cell_floats
                                  : P->cs.p + (P->phys.compton_model == CTD_COMPTON_WH ? material * cell_floats : 0);
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
    if (fn < 0 || fn > 2) return fail(CTD_EINVAL, "fn is 0 (log), 1 (sincos of 2 pi x) or 2 (uniform of a word)");
    if (n == 0) return CTD_OK;
    if (!x || !out) return fail(CTD_EINVAL, "null buffer");
    DevBuf<float> bx, bo;
    const size_t no = fn == 1 ? 2 * n : n;
    if ((rc = bx.ensure(n)) || (rc = bo.ensure(no))) return rc;
    CK(cudaMemcpyAsync(bx.p, x, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CKS(ctd::launch_eval_math(fn, bx.p, bo.p, n, ctx->stream));
    CK(cudaMemcpyAsync(out, bo.p, no * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CTD_OK;
}

}  // extern "C"
