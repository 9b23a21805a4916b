// ctd_host.h -- host-side state behind the C ABI of include/ctd.h, shared by
// ctd_capi.cu (contexts, phantoms, set-up, the plain form, results),
// ctd_forms.cu (the batched and served forms) and ctd_tune.cu (launch-shape
// search, memory probes).
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ctd_internal.h"

namespace ctd {
namespace host {

// the calling thread's message for ctd_last_error(); fail() sets it and returns code
extern thread_local std::string g_error;
int fail(int code, const char *fmt, ...);

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return ::ctd::host::fail(CTD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

#define CKS(call)                                                                                         \
    do {                                                                                                  \
        int s_ = (call);                                                                                  \
        if (s_ != CTD_OK) {                                                                               \
            if (::ctd::host::g_error.empty()) ::ctd::host::fail(s_, "%s failed: %s", #call, cudaGetErrorString(cudaGetLastError())); \
            return s_;                                                                                    \
        }                                                                                                 \
    } while (0)

// Device buffers a context has released and may hand out again: the byte size of
// each, up to `cap` bytes in all.  A phantom's buffers return here when it is
// destroyed (after its context's stream is idle), so a phantom of the same size
// created next takes them without cudaMalloc, and no cudaFree synchronises the
// device meanwhile.  The context frees what is left when it is destroyed.
struct BufferCache {
    std::multimap<size_t, void *> blocks;
    size_t cached = 0;
    size_t cap = size_t(4) << 30;
    void *take(size_t bytes)
    {
        auto it = blocks.find(bytes);
        if (it == blocks.end()) return nullptr;
        void *p = it->second;
        blocks.erase(it);
        cached -= bytes;
        return p;
    }
    bool give(void *p, size_t bytes)
    {
        if (cached + bytes > cap) return false;
        blocks.emplace(bytes, p);
        cached += bytes;
        return true;
    }
    ~BufferCache()
    {
        for (auto &b : blocks) cudaFree(b.second);
    }
};

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    BufferCache *cache = nullptr;   // where released buffers go (nullptr: cudaFree)
    ~DevBuf() { release(); }
    void release()
    {
        if (p && !(cache && cache->give(p, n * sizeof(T)))) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    int ensure(size_t count)
    {
        if (count <= n && p) return CTD_OK;
        release();
        if (count == 0) count = 1;
        if (cache && (p = static_cast<T *>(cache->take(count * sizeof(T))))) {
            n = count;
            return CTD_OK;
        }
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
    std::vector<ctd::Elements> els;   // per material: independent-atom Rayleigh form factor (n = 0: none)
    std::vector<double> rho_max;
    std::vector<int> present;
    ctd_physics phys{};
    ctd_source src{};
    bool has_src = false;
    std::vector<double> e_lo, e_hi, w;
    bool has_spec = false;

    DevBuf<uint8_t> mat;
    DevBuf<float> rho;
    DevBuf<uint32_t> vox;      // material and density packed (what the transport reads)
    DevBuf<double> rinv;       // 1 / density per voxel, 0 where it is 0 (what the fold reads)
    // tables
    bool tables_ok = false;
    int n_e = 0;
    std::vector<float> h_tab, h_mm, h_cs, h_rs;
    DevBuf<float> tab, mm, cs, rs;
    // per-run state
    DevBuf<double> tally, sum_d, sum_d2, edep, dose, sd, partials, result;
    DevBuf<double> tally2;     // the second stream's batch tally of an overlapped plain run
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
    // a sharded run in progress (ctd_shard_*): its history count, batches and seed
    uint64_t shard_n = 0, shard_seed = 0;
    int shard_nb = 0;
    double shard_t0 = 0.0;
    // every device buffer of the phantom takes from and returns to cache c
    void use_cache(BufferCache *c)
    {
        for (DevBuf<float> *b : {&rho, &tab, &mm, &cs, &rs, &bins, &proj}) b->cache = c;
        for (DevBuf<double> *b : {&tally, &tally2, &sum_d, &sum_d2, &edep, &dose, &sd, &partials, &result})
            b->cache = c;
        mat.cache = c;
        vox.cache = c;
        rinv.cache = c;
        counts.cache = c;
        work.cache = c;
        pref.cache = c;
        fl_thr.cache = c;
        fl_alias.cache = c;
    }
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
    // request chains (shared_launch = 0): the stream slot the request runs on; the
    // slices of its current batch done (`slice`); what it has on the GPU: the
    // batches those launches complete (`group`, the last followed by the stop
    // test's statistics when `checked`), the slice count after them, their
    // histories, and whether the lane's second event marks the end of all of them
    // but the last (`split`)
    int lane = -1;
    int slice = 0, group = 0, slice_after = 0;
    double flight_histories = 0.0;
    bool in_flight = false, checked = false, split = false;
};

constexpr int kRsdParts = 1024;   // partial sums of the statistics reductions
constexpr int kMaxLanes = 64;     // streams for request chains
constexpr uint64_t kMaxTrace = 1ull << 26;   // histories of one trace call (16 B of device memory each)

}  // namespace host
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
    // released device buffers (declared before the phantoms: it outlives them)
    ctd::host::BufferCache buffers;
    std::map<int, std::unique_ptr<ctd::host::Phantom>> phantoms;
    int next_id = 1;
    std::vector<cudaEvent_t> events;
    // multi-request launches: request and fold descriptors, claim counters
    ctd::host::DevBuf<ctd::RequestDesc> u_reqs;
    ctd::host::DevBuf<uint64_t> u_tiles;
    ctd::host::DevBuf<ctd::FoldDesc> u_folds;
    ctd::host::DevBuf<unsigned long long> u_work;
    // served form: all requests by id, the admission queue and the running set
    std::map<int64_t, ctd::host::ServeReq> sreqs;
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
    int batch_lanes = 64;          // batched form: streams the request chains share
    // plain-form launches: an L2 access-policy window over the tally (1) or the
    // packed voxel words (2), with a persisting set-aside of its size (granted bytes; at
    // most the device's maximum), no larger than the device's window; the context's
    // persisting-L2 limit before, put back on destroy
    int l2_persist = 0;
    // overlapped plain runs: the second stream, the event that starts it, and one event
    // per stream marking its last fold (folds run in batch order)
    bool plain_overlap = false;
    cudaStream_t plain_aux = nullptr;
    cudaEvent_t plain_fork = nullptr, plain_fold[2] = {nullptr, nullptr};
    size_t l2_asked = 0, l2_setaside = 0, l2_persist_max = 0, l2_window_max = 0, l2_prev_limit = 0;
    ctd::host::Staged *staged = nullptr;      // pinned read-back of counts and results
    size_t staged_n = 0;
    // angular surfaces by (kind, q0, e_min, n_e, n_zeta[, the elements' (Z, count) pairs]):
    // they do not depend on the phantom
    std::map<std::vector<double>, std::vector<float>> surfaces;
    // node-table columns of a material by (Compton model, e_min, n_e, its parameters and
    // elements): the Waller-Hartree and independent-atom totals are numeric integrals
    std::map<std::vector<double>, std::vector<double>> columns;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fork_event = nullptr;
    // served request chains: the request holding each lane (0: free), an event per lane
    // marking the end of its batch in flight, and pinned slots [lane][4] the batch's
    // avg RSD, sigma_bar and D_max come back to
    std::vector<int64_t> lane_owner;
    std::vector<cudaStream_t> serve_hi;   // per lane, a stream of the device's greatest priority
    std::vector<cudaEvent_t> serve_ev;
    std::vector<cudaEvent_t> serve_ev_pre;   // per lane: every batch in flight but the last done
    double *serve_res = nullptr;
    ctd::host::DevBuf<unsigned long long> serve_work;   // claim counter per lane
};

namespace ctd {
namespace host {

int use_device(ctd_ctx *ctx);
Phantom *find(ctd_ctx *ctx, ctd_phantom id);
// CTD_EBUSY while a served request holds the phantom
int busy(Phantom *P);
// Klein-Nishina C (kind 0), Rayleigh R (kind 1, form-factor width q0) or
// Waller-Hartree C (kind 2, scattering-function width q0) surface in binary32,
// built once per context and node grid
const std::vector<float> &angular_surface(ctd_ctx *ctx, int kind, double q0, const ctd::Elements *el, int e_min, int n_e,
                                         int n_zeta);
// attenuation tables, majorant and surfaces of the phantom's physics, uploaded
int build_tables(ctd_ctx *ctx, Phantom &P);
// bin starts of the stratified allocation for batches of n / nb (and one more)
int upload_allocation(ctd_ctx *ctx, Phantom &P, uint64_t n, int nb);
int ensure_run_buffers(Phantom &P);
int check_ready(Phantom &P);
int prepare_run(ctd_ctx *ctx, Phantom &P, uint64_t n, int nb);
// the per-request part of a transport launch; the shared part
void fill_request(Phantom &P, uint64_t seed, ctd::RequestDesc &q);
void fill_shared(Phantom &P, ctd::SharedTables &sh);
cudaEvent_t event_at(ctd_ctx *ctx, size_t i);
// streams for independent request chains: chain r runs on lane(ctx, r)
int ensure_lanes(ctd_ctx *ctx, int n);
int fork_lanes(ctd_ctx *ctx, cudaStream_t origin, int n);
int join_lanes(ctd_ctx *ctx, cudaStream_t origin, int n);
// one single-request launch of q on stream s at the context's launch shape
int launch_one(ctd_ctx *ctx, Phantom &P, const ctd::RequestDesc &q, cudaStream_t s);
// mean, standard error, avg RSD and deposited energy of nb finished batches
int finish_stats(Phantom &P, int nb, cudaStream_t s);
// one transport launch over local histories [lb, le) of a batch starting at h_base,
// bracketed by timing events 2 ev_index and 2 ev_index + 1
// (trace: per-history records of histories trace_h0 .. trace_h0 + trace_n - 1, or nullptr)
// on stream s (null: the context's) with claim counter work (null: the phantom's first)
int transport(ctd_ctx *ctx, Phantom &P, ctd::RequestDesc &q, int which_size, uint64_t h_base, uint64_t lb,
              uint64_t le, double *tally, size_t ev_index, uint4 *trace = nullptr, uint64_t trace_h0 = 0,
              uint64_t trace_n = 0, cudaStream_t s = nullptr, unsigned long long *work = nullptr);
double now_s();
int transport_time(ctd_ctx *ctx, size_t n_launch, double &t);
// counts and results of several phantoms read back through pinned staging
int collect_many(ctd_ctx *ctx, Phantom *const *ps, int n, size_t n_launch, double t0_wall,
                 const double *t0_each = nullptr, cudaStream_t stream = nullptr);
int collect(ctd_ctx *ctx, Phantom &P, size_t n_launch, double t0_wall);

}  // namespace host
}  // namespace ctd
