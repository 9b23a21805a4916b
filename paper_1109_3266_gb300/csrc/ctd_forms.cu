// ctd_forms.cu -- the batched form (ctd_run_batch: many requests as one CUDA
// graph of request chains or shared launches) and the served form
// (continuous batching: submit, one round per ctd_serve_step, poll, wait,
// cancel) of the C ABI in include/ctd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <chrono>
#include <functional>
#include <thread>

#include "ctd_host.h"

using namespace ctd::host;

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
            f.rinv = P.rinv.p;
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
    const int shape[9] = {n_batches, ctx->shared_launch, ctx->num_sms, ctx->blocks_per_sm, ctx->multi_blocks_per_sm,
                          ctx->threads, ctx->chunk, ctx->flight_cap, ctx->batch_lanes};
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
        const int n_lanes = std::min(n_req, ctx->batch_lanes);
        if ((rc = ensure_lanes(ctx, n_lanes))) return rc;
        if (!event_at(ctx, 0) || !event_at(ctx, 1)) return fail(CTD_ECUDA, "cudaEventCreate failed");
        // chains are issued largest first, so that the last to finish are short ones
        // (longest processing time first: the smaller requests fill the tail)
        std::vector<int> order(n_req);
        for (int r = 0; r < n_req; ++r) order[r] = r;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return n_histories[a] > n_histories[b]; });
        put(order.data(), order.size() * sizeof(int));
        body = [&, order, n_lanes](cudaStream_t cs) {
            if (cudaMemsetAsync(ctx->u_work.p, 0, static_cast<size_t>(n_batches) * n_req * sizeof(unsigned long long),
                                cs) != cudaSuccess ||
                cudaEventRecordWithFlags(ctx->events[0], cs, cudaEventRecordExternal) != cudaSuccess)
                return static_cast<int>(CTD_ECUDA);
            int e = fork_lanes(ctx, cs, n_lanes);
            for (int k = 0; k < n_req && e == CTD_OK; ++k) {
                const int r = order[k];
                Phantom &P = *ps[r];
                // the k-th largest request on lane k (mod the lanes)
                const cudaStream_t ls = ctx->lanes[k % n_lanes];
                for (int b = 0; b < n_batches && e == CTD_OK; ++b) {
                    const size_t d = static_cast<size_t>(b) * n_req + r;
                    e = launch_one(ctx, P, descs[d], ls);
                    if (e == CTD_OK)
                        e = ctd::launch_fold(P.tally.p, P.rinv.p, P.sum_d.p, P.sum_d2.p, P.edep.p, P.nvox, folds[d].scale,
                                             ls);
                }
                if (e == CTD_OK) e = finish_stats(P, n_batches, ls);
            }
            if (e == CTD_OK) e = join_lanes(ctx, cs, n_lanes);
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
        for (int r = 0; r < n_req; ++r) L.any_fluence |= ps[r]->fl_nu > 0;
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

}  // extern "C"

// ---------------------------------------------------------------- served form
namespace {

double elapsed_since(double t) { return now_s() - t; }

constexpr int kServeSlices = 8;   // slices of a batch of a served request not first in line

// Lanes, their events and pinned result slots for served request chains, made
// once per context.
int ensure_serve_lanes(ctd_ctx *ctx)
{
    int rc;
    if ((rc = ensure_lanes(ctx, kMaxLanes))) return rc;
    if (ctx->lane_owner.empty()) ctx->lane_owner.assign(kMaxLanes, 0);
    if (ctx->serve_hi.empty()) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        for (int i = 0; i < kMaxLanes; ++i) {
            cudaStream_t st;
            CK(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest));
            ctx->serve_hi.push_back(st);
        }
    }
    while (ctx->serve_ev.size() < static_cast<size_t>(kMaxLanes)) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->serve_ev.push_back(e);
    }
    while (ctx->serve_ev_pre.size() < static_cast<size_t>(kMaxLanes)) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->serve_ev_pre.push_back(e);
    }
    if (!ctx->serve_res) {
        if (cudaMallocHost(reinterpret_cast<void **>(&ctx->serve_res), kMaxLanes * 4 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            ctx->serve_res = nullptr;
            return fail(CTD_ENOMEM, "cudaMallocHost failed");
        }
    }
    return ctx->serve_work.ensure(kMaxLanes);
}

int free_lane(ctd_ctx *ctx)
{
    for (int i = 0; i < static_cast<int>(ctx->lane_owner.size()); ++i)
        if (ctx->lane_owner[i] == 0) return i;
    return -1;
}

// A request's tallies, statistics and counters cleared on stream s.
int clear_run(Phantom &P, cudaStream_t s)
{
    const size_t nv = P.nvox;
    CK(cudaMemsetAsync(P.tally.p, 0, nv * sizeof(double), s));
    CK(cudaMemsetAsync(P.sum_d.p, 0, nv * sizeof(double), s));
    CK(cudaMemsetAsync(P.sum_d2.p, 0, nv * sizeof(double), s));
    CK(cudaMemsetAsync(P.edep.p, 0, nv * sizeof(double), s));
    CK(cudaMemsetAsync(P.counts.p, 0, sizeof(ctd::DeviceCounts), s));
    return CTD_OK;
}

// Admit queued requests in order while memory and slots allow.  Request chains
// (chains = true) also need a free lane; a request's buffers are cleared on the
// stream it will run on.
int admit(ctd_ctx *ctx, bool chains)
{
    double round = 0.0;
    for (int64_t id : ctx->active) round += static_cast<double>(ctx->sreqs[id].req.batch_histories);
    while (!ctx->pending.empty() && static_cast<int>(ctx->active.size()) < ctx->max_active) {
        ServeReq &R = ctx->sreqs[ctx->pending.front()];
        // first in, first out: a request joins the running set only while one batch of
        // every running request stays within the round budget (one request always may)
        const double b = static_cast<double>(R.req.batch_histories);
        if (!ctx->active.empty() && round + b > ctx->round_histories) break;
        const int lane_i = chains ? free_lane(ctx) : -1;
        if (chains && lane_i < 0) break;
        Phantom *P = find(ctx, R.ph);
        if (!P) {
            R.state = CTD_REQ_FAILED;
            ctx->pending.erase(ctx->pending.begin());
            continue;
        }
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        free_b += ctx->buffers.cached;   // released buffers the context holds for reuse
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
        // request chains clear the buffers on the stream of their first launch
        if (!chains && (rc = clear_run(*P, ctx->stream))) return rc;
        P->have_result = false;
        R.state = CTD_REQ_RUNNING;
        R.t_start = now_s();
        if (chains) {
            R.lane = lane_i;
            ctx->lane_owner[lane_i] = R.id;
        }
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
    R.in_flight = false;
    Phantom *P = find(ctx, R.ph);
    if (P) P->busy_req = 0;
    if (R.lane >= 0) {
        ctx->lane_owner[R.lane] = 0;
        R.lane = -1;
    }
    for (size_t i = 0; i < ctx->active.size(); ++i)
        if (ctx->active[i] == R.id) {
            ctx->active.erase(ctx->active.begin() + i);
            break;
        }
}

// Histories of one launch that fill the GPU: kFillPerLane per resident lane.
constexpr double kFillPerLane = 64.0;

double fill_histories(const ctd_ctx *ctx)
{
    return kFillPerLane * static_cast<double>(ctx->num_sms) * ctx->blocks_per_sm * ctx->threads;
}

// The next work of a running request on its own lane: transport, the fold of each
// batch it completes and, from min_batches on, the statistics of the stop test with
// their copy to the lane's pinned slot; the lane's event marks its end.
// The first request in line sends, on its lane's high-priority stream, the rest of
// a batch it began in slices and every batch before its first stop test at once
// (nothing is decided between them), one launch each; a second event marks the end
// of all of them but the last.  Any other request sends one slice (1/kServeSlices of
// a batch of consecutive histories) of a batch that fills the GPU, or one whole
// smaller batch, on the lane's own stream: its persistent blocks give the SMs back
// after a slice, so the first request's blocks, dispatched first, wait at most one
// slice for them.  Work starts only after the request's previous work has finished
// (the host saw its event), so switching streams keeps the order.
int launch_work(ctd_ctx *ctx, ServeReq &R, Phantom &P, bool first_in_line)
{
    const cudaStream_t s = first_in_line ? ctx->serve_hi[R.lane] : ctx->lanes[R.lane];
    int rc;
    if (R.batches == 0 && R.slice == 0 && (rc = clear_run(P, s))) return rc;
    const uint64_t B = R.req.batch_histories;
    const uint64_t S = kServeSlices;
    const uint64_t lo = B * static_cast<uint64_t>(R.slice) / S;   // first history of the first launch
    uint64_t hi = B;
    int n = 1;                                                     // batches the launches complete
    int slice_after = 0;
    if (first_in_line) {
        if (R.batches + 1 < R.req.min_batches) n = R.req.min_batches - R.batches;
    } else if (static_cast<double>(B) >= fill_histories(ctx)) {
        hi = B * static_cast<uint64_t>(R.slice + 1) / S;
        n = R.slice + 1 == kServeSlices ? 1 : 0;
        slice_after = n ? 0 : R.slice + 1;
    }
    ctd::RequestDesc q;
    fill_request(P, R.req.seed, q);
    q.work = ctx->serve_work.p + R.lane;
    q.pref = P.pref.p + 1 * (q.nbins + 1);    // batches of exactly B histories
    q.tally = P.tally.p;
    const double scale = ctd::kKevToJ * 1000.0 / (P.dx * P.dy * P.dz * static_cast<double>(B));
    double hist = 0.0;
    for (int j = 0; j < std::max(n, 1); ++j) {
        q.h_base = static_cast<uint64_t>(R.batches + j) * B;
        q.local_begin = j == 0 ? lo : 0;
        q.local_end = j == 0 ? hi : B;
        if (q.local_begin < q.local_end) {
            CK(cudaMemsetAsync(q.work, 0, sizeof(unsigned long long), s));
            CKS(launch_one(ctx, P, q, s));
            hist += static_cast<double>(q.local_end - q.local_begin);
        }
        if (j < n) CKS(ctd::launch_fold(P.tally.p, P.rinv.p, P.sum_d.p, P.sum_d2.p, P.edep.p, P.nvox, scale, s));
        if (j == n - 2) CK(cudaEventRecord(ctx->serve_ev_pre[R.lane], s));
    }
    const int done = R.batches + n;
    R.checked = n > 0 && done >= R.req.min_batches;
    if (R.checked) {
        CKS(ctd::launch_finalize(P.sum_d.p, P.sum_d2.p, done, P.dose.p, P.sd.p, P.nvox, s));
        CKS(ctd::launch_rsd(P.dose.p, P.sd.p, P.rho.p, P.nvox, P.partials.p, kRsdParts, P.result.p, s));
        CK(cudaMemcpyAsync(ctx->serve_res + 4 * R.lane, P.result.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(ctx->serve_ev[R.lane], s));
    R.group = n;
    R.slice_after = slice_after;
    R.flight_histories = first_in_line ? static_cast<double>(B) : hist;
    R.split = n > 1;
    R.in_flight = true;
    return CTD_OK;
}

// Histories a running request is estimated to still need, counting its batches
// on the GPU as done: the batches up to min_batches and, once the avg RSD is known,
// n ((rsd / target)^2 - 1) for the avg RSD falling as 1 / sqrt(n), at least one
// batch, at most what its history cap leaves.
double remaining(const ServeReq &R)
{
    const double B = static_cast<double>(R.req.batch_histories);
    const double ran = static_cast<double>(R.histories) + R.group * B;
    const double cap = static_cast<double>(R.req.n_histories_max);
    double need = std::max(0, R.req.min_batches - R.batches - R.group) * B;
    if (R.req.rsd_target == 0.0) {
        need = std::max(need, cap - ran);   // runs to its cap
    } else if (R.batches >= R.req.min_batches && R.avg_rsd > 0.0) {
        const double n = static_cast<double>(R.histories);
        const double r = R.avg_rsd / R.req.rsd_target;
        need = std::max(need, n * r * r - ran);
    }
    if (R.req.n_histories_max) need = std::min(need, std::max(0.0, cap - ran));
    return std::max(need, B);
}

// Whether the first request in line leaves room for the others: not while it has
// batches on the GPU of which none can be its last; during a batch that may be its
// last they fill the SMs it leaves idle and the gap until the host sees it end.
bool first_leaves_room(ctd_ctx *ctx, const ServeReq &F)
{
    if (!F.in_flight) return true;
    if (!F.checked) return false;
    return !F.split || cudaEventQuery(ctx->serve_ev_pre[F.lane]) != cudaErrorNotReady;
}

// A request that reached its target or its history cap: total deposit, results
// read back on its lane, then retired.
int finish_request(ctd_ctx *ctx, ServeReq &R, Phantom &P)
{
    const cudaStream_t s = ctx->lanes[R.lane];
    CKS(ctd::launch_sum(P.edep.p, P.nvox, P.partials.p + 5 * kRsdParts, kRsdParts, P.result.p + 3, s));
    Phantom *ps[1] = {&P};
    const double t0[1] = {R.t_start};
    int rc;
    if ((rc = collect_many(ctx, ps, 1, 0, 0.0, t0, s))) return rc;
    P.stats.histories = R.histories;
    P.stats.n_batches = R.batches;
    P.have_result = true;
    retire(ctx, R, CTD_REQ_DONE);
    return CTD_OK;
}

bool reached_stop(const ServeReq &R)
{
    const bool hit = R.req.rsd_target > 0.0 && R.avg_rsd > 0.0 && R.avg_rsd <= R.req.rsd_target;
    const bool cap = R.req.n_histories_max && R.histories >= R.req.n_histories_max;
    return hit || cap;
}

// Request chains (shared_launch = 0): every running request advances on its own
// lane independently of the others.  One call takes in the batches that have
// finished, retires cancelled and finished requests, admits queued ones and
// launches the next batch of every request with nothing on the GPU; it does not
// wait for the GPU, except for the batch in flight of a cancelled request.
// *progress: whether anything was taken in, retired, admitted or launched.
int serve_chains(ctd_ctx *ctx, bool *progress)
{
    int rc;
    if ((rc = ensure_serve_lanes(ctx))) return rc;
    bool moved = false;
    const std::vector<int64_t> act = ctx->active;
    for (int64_t id : act) {
        ServeReq &R = ctx->sreqs[id];
        if (!R.in_flight) continue;
        const cudaError_t q = R.cancel ? cudaEventSynchronize(ctx->serve_ev[R.lane])
                                       : cudaEventQuery(ctx->serve_ev[R.lane]);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            retire(ctx, R, CTD_REQ_FAILED);
            return fail(CTD_ECUDA, "served request %lld: %s", static_cast<long long>(id), cudaGetErrorString(q));
        }
        moved = true;
        // the batches are done: only now do they count
        R.in_flight = false;
        R.batches += R.group;
        R.histories += static_cast<uint64_t>(R.group) * R.req.batch_histories;
        R.slice = R.slice_after;
        R.group = 0;
        R.split = false;
        if (R.checked) {
            R.avg_rsd = ctx->serve_res[4 * R.lane];
            R.sigma_bar = ctx->serve_res[4 * R.lane + 1];
        }
        if (!R.cancel && R.checked && reached_stop(R)) {
            Phantom *P = find(ctx, R.ph);
            if (!P) {
                retire(ctx, R, CTD_REQ_FAILED);
                continue;
            }
            if ((rc = finish_request(ctx, R, *P))) {
                retire(ctx, R, CTD_REQ_FAILED);
                return rc;
            }
        }
    }
    // cancellations take effect once nothing of the request is on the GPU
    for (size_t i = 0; i < ctx->active.size();) {
        ServeReq &R = ctx->sreqs[ctx->active[i]];
        if (R.cancel && !R.in_flight) {
            retire(ctx, R, CTD_REQ_CANCELLED);
            moved = true;
        } else {
            ++i;
        }
    }
    const size_t before = ctx->active.size();
    if ((rc = admit(ctx, true))) return rc;
    moved = moved || ctx->active.size() != before;
    // In order of the estimated histories still needed (the earliest admitted among
    // equals): the first in line goes out first, so that its blocks are queued ahead of
    // the others'.  When its batches fill the GPU, only the second in line runs beside
    // it, and only while the first leaves room; when they do not, the others run while
    // the histories on the GPU stay below two launches that fill it.
    std::vector<std::pair<double, int64_t>> by_need;
    for (int64_t id : ctx->active) by_need.emplace_back(remaining(ctx->sreqs[id]), id);
    std::stable_sort(by_need.begin(), by_need.end(),
                     [](const std::pair<double, int64_t> &a, const std::pair<double, int64_t> &b) {
                         return a.first < b.first;
                     });
    auto launch = [&](ServeReq &R, bool first) {
        Phantom *P = find(ctx, R.ph);
        int code = P ? launch_work(ctx, R, *P, first) : CTD_OK;
        if (!P || code) retire(ctx, R, CTD_REQ_FAILED);
        else moved = true;
        return code;
    };
    if (!by_need.empty()) {
        const int64_t first = by_need.front().second;
        ServeReq &F = ctx->sreqs[first];
        if (!F.in_flight && (rc = launch(F, true))) return rc;
        const bool fills = static_cast<double>(F.req.batch_histories) >= fill_histories(ctx);
        if (fills) {
            if (by_need.size() > 1 && first_leaves_room(ctx, F)) {
                ServeReq &R = ctx->sreqs[by_need[1].second];
                if (!R.in_flight && (rc = launch(R, false))) return rc;
            }
        } else {
            const double budget = 2.0 * fill_histories(ctx);
            double on_gpu = 0.0;
            for (const auto &e : by_need)
                if (ctx->sreqs[e.second].in_flight) on_gpu += ctx->sreqs[e.second].flight_histories;
            for (size_t k = 1; k < by_need.size() && on_gpu < budget; ++k) {
                ServeReq &R = ctx->sreqs[by_need[k].second];
                if (R.in_flight) continue;
                if ((rc = launch(R, false))) return rc;
                on_gpu += R.flight_histories;
            }
        }
    }
    *progress = moved;
    return CTD_OK;
}

// Shared launches (shared_launch = 1): one round, one batch of every running
// request in one multi-request launch, waited for.
int serve_round(ctd_ctx *ctx)
{
    int rc;
    for (size_t i = 0; i < ctx->active.size();) {
        ServeReq &R = ctx->sreqs[ctx->active[i]];
        if (R.cancel) retire(ctx, R, CTD_REQ_CANCELLED);
        else ++i;
    }
    if ((rc = admit(ctx, false))) return rc;
    const int n = static_cast<int>(ctx->active.size());
    if (n == 0) return CTD_OK;
    std::vector<Phantom *> ps(n);
    for (int i = 0; i < n; ++i) ps[i] = find(ctx, ctx->sreqs[ctx->active[i]].ph);
    for (int i = 1; i < n; ++i) {
        const ctd_physics &a = ps[0]->phys, &b = ps[i]->phys;
        if (a.e_min_kev != b.e_min_kev || a.e_max_kev != b.e_max_kev || a.n_zeta != b.n_zeta) {
            retire(ctx, ctx->sreqs[ctx->active[i]], CTD_REQ_FAILED);
            return fail(CTD_EINVAL, "served requests must share one node grid");
        }
    }
    int max_n_mat = 0;
    for (int i = 0; i < n; ++i) max_n_mat = std::max(max_n_mat, static_cast<int>(ps[i]->mats.size()));
    if ((rc = ctx->u_work.ensure(n))) return rc;
    std::vector<ctd::RequestDesc> descs(n);
    std::vector<uint64_t> tiles(n + 1, 0);
    std::vector<ctd::FoldDesc> folds(n);
    std::vector<int> checked;
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
        f.rinv = P.rinv.p;
        f.sum_d = P.sum_d.p;
        f.sum_d2 = P.sum_d2.p;
        f.edep = P.edep.p;
        f.nvox = P.nvox;
        f.scale = ctd::kKevToJ * 1000.0 / (P.dx * P.dy * P.dz * static_cast<double>(B));
        // those past min_batches after this round also get their statistics
        if (R.batches + 1 >= R.req.min_batches) checked.push_back(i);
    }
    // a round whose launches fail counts for no request: their batches stay as they were
    auto failed = [&](int code) {
        for (int64_t id : std::vector<int64_t>(ctx->active)) retire(ctx, ctx->sreqs[id], CTD_REQ_FAILED);
        return code;
    };
    if ((rc = ctx->u_reqs.ensure(n)) || (rc = ctx->u_folds.ensure(n)) || (rc = ctx->u_tiles.ensure(n + 1)))
        return failed(rc);
    if (cudaMemcpyAsync(ctx->u_reqs.p, descs.data(), n * sizeof(ctd::RequestDesc), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ctx->u_folds.p, folds.data(), n * sizeof(ctd::FoldDesc), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ctx->u_tiles.p, tiles.data(), (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->u_work.p, 0, n * sizeof(unsigned long long), ctx->stream) != cudaSuccess)
        return failed(fail(CTD_ECUDA, "served round: copying the request table failed"));
    ctd::LaunchParams L;
    std::memset(&L, 0, sizeof(L));
    fill_shared(*ps[0], L.sh);
    L.sh.max_n_mat = max_n_mat;
    L.reqs = ctx->u_reqs.p;
    L.n_req = n;
    for (int i = 0; i < n; ++i) L.any_fluence |= ps[i]->fl_nu > 0;
    L.chunk = ctx->chunk;
    L.flight_cap = ctx->flight_cap;
    const int mgrid = ctx->num_sms * ctx->multi_blocks_per_sm;
    if ((rc = ctd::launch_transport(L, mgrid, ctx->threads, ctx->threads * ctx->multi_blocks_per_sm, ctx->stream)) ||
        (rc = ctd::launch_fold_multi(ctx->u_folds.p, ctx->u_tiles.p, n, tiles[n], ctx->stream)))
        return failed(rc);
    for (int i : checked) {
        Phantom &P = *ps[i];
        const int nb = ctx->sreqs[ctx->active[i]].batches + 1;
        if ((rc = ctd::launch_finalize(P.sum_d.p, P.sum_d2.p, nb, P.dose.p, P.sd.p, P.nvox, ctx->stream)) ||
            (rc = ctd::launch_rsd(P.dose.p, P.sd.p, P.rho.p, P.nvox, P.partials.p, kRsdParts, P.result.p,
                                  ctx->stream)))
            return failed(rc);
    }
    std::vector<std::array<double, 3>> res(checked.size());
    for (size_t c = 0; c < checked.size(); ++c)
        if (cudaMemcpyAsync(res[c].data(), ps[checked[c]]->result.p, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess)
            return failed(fail(CTD_ECUDA, "served round: reading the statistics failed"));
    const cudaError_t se = cudaStreamSynchronize(ctx->stream);
    if (se != cudaSuccess) return failed(fail(CTD_ECUDA, "served round: %s", cudaGetErrorString(se)));
    // the round is done: now its batch counts for every running request
    for (int i = 0; i < n; ++i) {
        ServeReq &R = ctx->sreqs[ctx->active[i]];
        R.batches += 1;
        R.histories += R.req.batch_histories;
    }
    std::vector<int64_t> finished;
    for (size_t c = 0; c < checked.size(); ++c) {
        ServeReq &R = ctx->sreqs[ctx->active[checked[c]]];
        R.avg_rsd = res[c][0];
        R.sigma_bar = res[c][1];
        if (reached_stop(R)) finished.push_back(R.id);
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
    return CTD_OK;
}

int serve_pump(ctd_ctx *ctx, bool *progress)
{
    *progress = true;
    return ctx->shared_launch ? serve_round(ctx) : serve_chains(ctx, progress);
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
    bool progress;
    rc = serve_pump(ctx, &progress);
    if (n_active) *n_active = static_cast<int>(ctx->active.size() + ctx->pending.size());
    return rc;
}

int ctd_serve_wait(ctd_ctx *ctx, double timeout_s, int *n_active)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (!(timeout_s >= 0.0)) return fail(CTD_EINVAL, "timeout_s must be >= 0");
    const double t0 = now_s();
    for (;;) {
        bool progress = false;
        if ((rc = serve_pump(ctx, &progress))) break;
        if (progress || (ctx->active.empty() && ctx->pending.empty()) || elapsed_since(t0) >= timeout_s) break;
        // every running request's work is on the GPU: look again shortly instead of spinning
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (n_active) *n_active = static_cast<int>(ctx->active.size() + ctx->pending.size());
    return rc;
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
        bool progress = false;
        if ((rc = use_device(ctx)) || (rc = serve_pump(ctx, &progress))) return rc;
        if (before == 0 && ctx->active.empty() && ctx->sreqs[id].state == CTD_REQ_QUEUED)
            return fail(CTD_ENOMEM, "request %lld cannot be admitted: not enough free device memory",
                        static_cast<long long>(id));
        // every batch is on the GPU: look again shortly instead of spinning
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
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
