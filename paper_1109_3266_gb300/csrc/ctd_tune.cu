// ctd_tune.cu -- the launch-shape searches for the single-request transport
// kernel (ctd_autotune) and for the batched form (ctd_autotune_batch), and the
// memory-ceiling probes (ctd_probe_memory) of the C ABI in include/ctd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ctd_host.h"

using namespace ctd::host;

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
    // best of two timed probes of histories [0, n) of batch 0 in shape s
    auto time_shape = [&](const Shape &s, uint64_t n, double &t_min) -> int {
        ctx->threads = s.threads;
        ctx->blocks_per_sm = s.bps;
        ctx->chunk = s.chunk;
        ctx->flight_cap = s.cap;
        t_min = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaMemsetAsync(P->counts.p, 0, sizeof(ctd::DeviceCounts), ctx->stream));
            int e;
            if ((e = transport(ctx, *P, q, 0, 0, 0, n, P->tally.p, 0))) return e;
            CK(cudaStreamSynchronize(ctx->stream));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ctx->events[0], ctx->events[1]));
            t_min = std::min(t_min, static_cast<double>(ms) * 1e-3);
        }
        return CTD_OK;
    };
    auto restore = [&]() {
        ctx->threads = old_threads;
        ctx->blocks_per_sm = old_bps;
        ctx->chunk = old_chunk;
        ctx->flight_cap = old_cap;
    };
    // first pass: every shape on n_probe histories
    std::vector<std::pair<double, size_t>> t1;
    for (size_t k = 0; k < shapes.size(); ++k) {
        double t;
        if ((rc = time_shape(shapes[k], n_probe, t))) {
            restore();
            return rc;
        }
        t1.push_back({t, k});
    }
    // second pass: the four fastest and the current shape on 5 n_probe histories (short
    // probes overrate shapes whose blocks drain a launch's tail sooner)
    std::sort(t1.begin(), t1.end());
    std::vector<size_t> finalists{0};
    for (size_t r = 0; r < t1.size() && finalists.size() < 5; ++r)
        if (t1[r].second != 0) finalists.push_back(t1[r].second);
    const uint64_t n2 = 5 * n_probe;
    if ((rc = prepare_run(ctx, *P, 10 * n2, 10))) {
        restore();
        return rc;
    }
    fill_request(*P, seed, q);
    double best = 1e300, base = 0.0;
    Shape pick = shapes[0];
    for (size_t k : finalists) {
        double t;
        if ((rc = time_shape(shapes[k], n2, t))) {
            restore();
            return rc;
        }
        if (k == 0) base = t;
        if (t < best) {
            best = t;
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
        out->histories_per_s = static_cast<double>(n2) / best;
        out->baseline_per_s = static_cast<double>(n2) / base;
        out->shared_launch = ctx->shared_launch;
        out->multi_blocks_per_sm = ctx->multi_blocks_per_sm;
    }
    return CTD_OK;
}

int ctd_autotune_batch(ctd_ctx *ctx, int n_req, const ctd_phantom *phantoms, const uint64_t *n_histories,
                       const uint64_t *seeds, int n_batches, double probe_fraction, ctd_tune_result *out)
{
    int rc;
    if ((rc = use_device(ctx))) return rc;
    if (n_req <= 0 || !phantoms || !n_histories || !seeds) return fail(CTD_EINVAL, "bad request arrays");
    if (n_batches < 2) return fail(CTD_EINVAL, "need n_batches >= 2");
    if (!(probe_fraction > 0.0 && probe_fraction <= 1.0)) return fail(CTD_EINVAL, "probe_fraction in (0, 1]");
    // the probe: every request with a fraction of its histories (at least one per batch)
    std::vector<uint64_t> nh(n_req);
    uint64_t total = 0;
    for (int r = 0; r < n_req; ++r) {
        const double x = static_cast<double>(n_histories[r]) * probe_fraction;
        nh[r] = std::max<uint64_t>(static_cast<uint64_t>(n_batches), static_cast<uint64_t>(x));
        total += nh[r];
    }
    struct Shape {
        int shared, threads, bps, mbps, chunk, cap, lanes;
    };
    const Shape old{ctx->shared_launch, ctx->threads, ctx->blocks_per_sm, ctx->multi_blocks_per_sm, ctx->chunk,
                    ctx->flight_cap, ctx->batch_lanes};
    std::vector<Shape> shapes{old};
    // request chains: block shape and residency of each request's launches; shared
    // launches: blocks per SM of the multi-request kernel; both: claim size (how many
    // histories a warp takes into its photon queue at a time) and flight cap (how many
    // Woodcock flights a lane runs before its warp regroups at the queue)
    const int chains[3][2] = {{256, 4}, {256, 3}, {128, 8}};
    for (const auto &b : chains)
        for (int chunk : {256, 1024})
            for (int cap : {2, 4})
                shapes.push_back({0, b[0], b[1], old.mbps, chunk, cap, old.lanes});
    // request chains sharing fewer streams: fewer requests' phantoms and tallies in L2 at once
    for (int lanes : {2, 4, 8, 16})
        shapes.push_back({0, 256, 4, old.mbps, 256, 4, lanes});
    for (int mbps : {2, 3, 4})
        for (int chunk : {256, 1024})
            for (int cap : {2, 4})
                shapes.push_back({1, 256, old.bps, mbps, chunk, cap, old.lanes});
    auto apply = [&](const Shape &s) {
        ctx->shared_launch = s.shared;
        ctx->threads = s.threads;
        ctx->blocks_per_sm = s.bps;
        ctx->multi_blocks_per_sm = s.mbps;
        ctx->chunk = s.chunk;
        ctx->flight_cap = s.cap;
        ctx->batch_lanes = s.lanes;
    };
    // best of two timed batched calls (the first call of a shape records its graph)
    auto time_shape = [&](const Shape &s, double &t_min) -> int {
        apply(s);
        t_min = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            const double t0 = now_s();
            int e;
            if ((e = ctd_run_batch(ctx, n_req, phantoms, nh.data(), seeds, n_batches))) return e;
            if (rep > 0) t_min = std::min(t_min, now_s() - t0);
        }
        return CTD_OK;
    };
    std::vector<std::pair<double, size_t>> t1;
    for (size_t k = 0; k < shapes.size(); ++k) {
        // one node grid per shared launch: shapes the requests cannot share are skipped
        if (shapes[k].shared && k > 0) {
            bool same = true;
            const Phantom *P0 = find(ctx, phantoms[0]);
            for (int r = 1; r < n_req && same && P0; ++r) {
                const Phantom *P = find(ctx, phantoms[r]);
                same = P && P->phys.e_min_kev == P0->phys.e_min_kev && P->phys.e_max_kev == P0->phys.e_max_kev &&
                       P->phys.n_zeta == P0->phys.n_zeta;
            }
            if (!same) continue;
        }
        double t;
        if ((rc = time_shape(shapes[k], t))) {
            apply(old);
            return rc;
        }
        t1.push_back({t, k});
    }
    // second pass: the three fastest and the context's own shape on probes five times
    // longer (short probes overrate shapes that drain a launch's tail sooner)
    std::sort(t1.begin(), t1.end());
    std::vector<size_t> finalists{0};
    for (size_t r = 0; r < t1.size() && finalists.size() < 4; ++r)
        if (t1[r].second != 0) finalists.push_back(t1[r].second);
    const double f2 = std::min(1.0, 5.0 * probe_fraction);
    total = 0;
    for (int r = 0; r < n_req; ++r) {
        const double x = static_cast<double>(n_histories[r]) * f2;
        nh[r] = std::max<uint64_t>(static_cast<uint64_t>(n_batches), static_cast<uint64_t>(x));
        total += nh[r];
    }
    double best = 1e300, base = 0.0;
    Shape pick = old;
    for (size_t k : finalists) {
        double t;
        if ((rc = time_shape(shapes[k], t))) {
            apply(old);
            return rc;
        }
        if (k == 0) base = t;
        if (t < best) {
            best = t;
            pick = shapes[k];
        }
    }
    apply(pick);
    if (out) {
        out->threads_per_block = pick.threads;
        out->blocks_per_sm = pick.bps;
        out->chunk = pick.chunk;
        out->flight_cap = pick.cap;
        out->n_tried = static_cast<int>(t1.size());
        out->histories_per_s = static_cast<double>(total) / best;
        out->baseline_per_s = static_cast<double>(total) / base;
        out->shared_launch = pick.shared;
        out->multi_blocks_per_sm = pick.mbps;
        out->batch_lanes = pick.lanes;
    }
    return CTD_OK;
}

}  // extern "C"
