// ctd_forms.cu -- the batched form (ctd_run_batch: many requests as one CUDA
// graph of request chains or shared launches) and the served form
// (continuous batching: submit, one round per ctd_serve_step, poll, wait,
// cancel) of the C ABI in include/ctd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <functional>

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
