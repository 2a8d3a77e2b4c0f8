// serve.cu -- continuous-batching localization server (lift + LO-RANSAC PnP).
//
// Clients submit queries (host matches, views into a device-resident map
// store, camera, options) and poll for results.  One scheduler thread owns
// the GPU and loops over steps:
//   1. admission: queued queries enter free slots in arrival order while the
//      sum of resident footprints stays within the device budget (first-fit
//      allocator over one device pool);
//   2. newly admitted queries: matches uploaded from the pinned host ring,
//      lifted into their slot, descriptors written;
//   3. one merged launch sequence advances every resident query by its next
//      RANSAC rounds (sample + P3P, score, replay/LO/termination, final
//      refinement when done) -- queries of different sizes and at different
//      rounds share the launches;
//   4. finished queries hand their result to the ticket table and free their
//      slot and memory.
// Steps are pipelined two deep on the server's stream: the scheduler
// enqueues step k+1 (uploads, lifts, launches, the read-back of the query
// states) before it waits for step k's event and retires step k's finished
// queries, so the GPU runs step k+1 while the host retires, admits and
// marshals.  A query that finished in step k is still part of step k+1,
// whose kernels skip it (its state is done).  The host blocks of a step
// (descriptors, round plan, states, results) are double-buffered pinned
// memory, and each step remembers the ticket of the query in each slot, so
// that a slot refilled meanwhile is not retired with the old query's state.
// A query that arrives while others are on the GPU joins at the next step.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "ransac_internal.h"

namespace imloc {

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing frees.
class FreeList {
   public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        in_use_ = 0;
    }
    size_t alloc(size_t bytes) {
        bytes = align_up(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                const size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                in_use_ += bytes;
                return off;
            }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes, 256);
        in_use_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t in_use() const { return in_use_; }

   private:
    std::map<size_t, size_t> free_;
    size_t in_use_ = 0;
};

struct ServeQuery {
    uint64_t ticket = 0;
    std::vector<imloc_view> views;
    std::vector<imloc_segment> segs;
    int64_t n = 0;
    imloc_camera cam{};
    imloc_ransac_opts opts{};
    size_t ring_off = 0, ring_size = 0, ring_waste = 0;
    const float* dmatch[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // device-submitted matches (caller's)
    bool on_device = false;
    double t_submit = 0.0;
    size_t footprint = 0;
    // resident
    int slot = -1;
    size_t pool_off = 0;
    int64_t H = 0, B = 0, R = 0, r_next = 0;
};

// Device footprint of one resident query and the offsets inside it.
struct Layout {
    size_t match[5], cx, cy, cX, cY, cZ, cw, csrc, ccount, fixidx, subset, slots, compact, round_best, round_hyps, total;
};

static Layout layout_of(int64_t n, int32_t m_cap, int64_t step_samples, int64_t rounds, bool with_matches = true) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + std::max<size_t>(bytes, 1), 256);
        return at;
    };
    for (int k = 0; k < 5; ++k) L.match[k] = with_matches ? take(sizeof(float) * n) : 0;
    L.cx = take(sizeof(float) * n);
    L.cy = take(sizeof(float) * n);
    L.cX = take(sizeof(float) * n);
    L.cY = take(sizeof(float) * n);
    L.cZ = take(sizeof(float) * n);
    L.cw = take(sizeof(float) * n);
    L.csrc = take(sizeof(int32_t) * n);
    L.ccount = take(sizeof(int32_t));
    L.fixidx = take(sizeof(int32_t) * static_cast<size_t>(n));
    L.subset = take(sizeof(ScorePair) * static_cast<size_t>((m_cap + 1) / 2));
    L.slots = take(sizeof(PoseF) * 4 * static_cast<size_t>(step_samples));
    L.compact = take(sizeof(int32_t) * 4 * static_cast<size_t>(step_samples));
    L.round_best = take(sizeof(uint64_t) * static_cast<size_t>(rounds));
    L.round_hyps = take(sizeof(int32_t) * static_cast<size_t>(rounds));
    L.total = o;
    return L;
}

}  // namespace imloc

using imloc::ServeQuery;

struct imloc_server {
    imloc_ctx* ictx = nullptr;
    imloc_serve_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    // device pool for resident queries (admission by bytes)
    char* pool = nullptr;
    imloc::FreeList pool_alloc;
    // per-slot control (device + pinned host mirrors)
    imloc::QueryDesc* d_qd = nullptr;
    imloc::QueryState* d_qs = nullptr;
    imloc::WaveQ* d_wq = nullptr;
    int64_t* d_prefix = nullptr;
    int32_t* d_nhyp = nullptr;
    int32_t* d_tiles = nullptr;
    uint32_t* d_counter = nullptr;
    int32_t* d_init = nullptr;
    imloc_result* d_res = nullptr;
    // host side: the descriptors of every slot, and per step parity the pinned
    // copies the step's transfers read or write, its completion event and its
    // slot occupants
    std::vector<imloc::QueryDesc> qd_master;
    imloc::QueryDesc* h_qd[2] = {nullptr, nullptr};
    imloc::WaveQ* h_wq[2] = {nullptr, nullptr};
    int64_t* h_prefix[2] = {nullptr, nullptr};
    int32_t* h_init[2] = {nullptr, nullptr};
    imloc::QueryState* h_qs[2] = {nullptr, nullptr};
    imloc_result* h_res[2] = {nullptr, nullptr};
    cudaEvent_t step_done[2] = {nullptr, nullptr};
    std::vector<uint64_t> occ[2];  // ticket of each slot's query during the step (0: empty); tickets are
                                   // never reused, unlike the addresses of freed queries
    std::vector<ServeQuery*> step_admitted[2];
    // pinned FIFO ring holding submitted matches until their upload
    char* ring = nullptr;
    size_t ring_bytes = 0, ring_head = 0, ring_tail = 0, ring_used = 0;
    // queues
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeQuery*> pending;
    std::vector<ServeQuery*> slots;
    std::unordered_map<uint64_t, std::pair<imloc_result, double>> done;
    std::unordered_map<uint64_t, int> live;  // 1 queued, 2 resident
    uint64_t next_ticket = 1;
    bool stop = false;
    int worker_error = IMLOC_OK;
    std::thread worker;
    imloc_serve_stats stats{};
};

namespace imloc {

// FIFO ring: used bytes live in [head, tail) (wrapping); an entry that does
// not fit before the end starts again at 0 and owns the unused end
static bool ring_alloc(imloc_server* S, size_t bytes, ServeQuery* q) {
    bytes = align_up(std::max<size_t>(bytes, 1), 256);
    if (S->ring_used == 0) S->ring_head = S->ring_tail = 0;
    q->ring_waste = 0;
    if (S->ring_used == 0 || S->ring_tail > S->ring_head) {
        // free space: [tail, end) and [0, head)
        if (S->ring_tail + bytes <= S->ring_bytes) {
            q->ring_off = S->ring_tail;
        } else if (bytes <= S->ring_head) {
            q->ring_waste = S->ring_bytes - S->ring_tail;
            q->ring_off = 0;
        } else {
            return false;
        }
    } else {
        // free space: [tail, head)
        if (S->ring_tail + bytes > S->ring_head) return false;
        q->ring_off = S->ring_tail;
    }
    q->ring_size = bytes;
    S->ring_tail = q->ring_off + bytes;
    S->ring_used += bytes + q->ring_waste;
    return true;
}

// entries are released in submission order
static void ring_release(imloc_server* S, ServeQuery* q) {
    S->ring_head = q->ring_off + q->ring_size;
    S->ring_used -= q->ring_size + q->ring_waste;
    if (S->ring_used == 0) S->ring_head = S->ring_tail = 0;
}

static void fill_desc(imloc_server* S, ServeQuery* q, const Layout& L) {
    char* base = S->pool + q->pool_off;
    QueryDesc& d = S->qd_master[q->slot];
    memset(&d, 0, sizeof(d));
    d.x = reinterpret_cast<float*>(base + L.cx);
    d.y = reinterpret_cast<float*>(base + L.cy);
    d.X = reinterpret_cast<float*>(base + L.cX);
    d.Y = reinterpret_cast<float*>(base + L.cY);
    d.Z = reinterpret_cast<float*>(base + L.cZ);
    d.w = reinterpret_cast<float*>(base + L.cw);
    d.d_count = reinterpret_cast<int32_t*>(base + L.ccount);
    d.n_host = q->n;
    d.result = S->d_res + q->slot;
    d.fx = q->cam.fx; d.fy = q->cam.fy; d.cx = q->cam.cx; d.cy = q->cam.cy;
    {
        const double ifx = 1.0 / static_cast<double>(q->cam.fx), ify = 1.0 / static_cast<double>(q->cam.fy);
        d.ifx_hi = static_cast<float>(ifx);
        d.ifx_lo = static_cast<float>(ifx - static_cast<double>(d.ifx_hi));
        d.ify_hi = static_cast<float>(ify);
        d.ify_lo = static_cast<float>(ify - static_cast<double>(d.ify_hi));
    }
    const imloc_ransac_opts& o = q->opts;
    d.tau2 = static_cast<float>(o.tau_px * o.tau_px);
    const double cs = o.cauchy_scale > 0.0 ? o.cauchy_scale : o.tau_px;
    d.cauchy2 = static_cast<float>(cs * cs);
    d.m_cap = o.max_score_corr;
    d.batch = static_cast<int32_t>(q->B);
    d.hyps = static_cast<int32_t>(q->H);
    d.rounds = static_cast<int32_t>(q->R);
    d.lo_iters = o.lo_iters;
    d.final_iters = o.final_iters;
    d.polish = o.p3p_fp64_polish;
    d.enumerate_all = 0;
    d.lo_fp64 = o.lo_fp64_accumulate;
    d.lo_solve64 = o.lo_fp64_solve;
    d.p_miss = o.p_miss;
    d.seed = o.seed;
    d.query_id = o.query_id;
    d.n_cap = static_cast<int32_t>(q->n);
    d.subset = reinterpret_cast<ScorePair*>(base + L.subset);
    d.slots = reinterpret_cast<PoseF*>(base + L.slots);
    d.compact = reinterpret_cast<int32_t*>(base + L.compact);
    d.round_best = reinterpret_cast<uint64_t*>(base + L.round_best);
    d.round_hyps = reinterpret_cast<int32_t*>(base + L.round_hyps);
    d.fixidx = reinterpret_cast<int32_t*>(base + L.fixidx);
}

static int64_t step_samples(const imloc_serve_config& c, int64_t B) { return B * std::max(1, c.rounds_per_step); }

static void fail_all(imloc_server* S, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->worker_error = status;
    for (auto& kv : S->live) {
        imloc_result r;
        memset(&r, 0, sizeof(r));
        r.status = status;
        S->done[kv.first] = {r, 0.0};
    }
    S->live.clear();
}

// Enqueue one scheduler step with host buffers of parity p: newly admitted
// queries (upload, lift, descriptors), then every resident query's next
// rounds in one merged launch sequence, then the read-back of the query
// states and results; records the step's event.  Does not wait for the GPU.
static int enqueue_step(imloc_server* S, const std::vector<ServeQuery*>& admitted, int p) {
    cudaStream_t st = S->stream;
    const int ns = S->cfg.max_slots;
    // one call on the lift context per step: its staging buffer and workspace
    // hold the tables of every newly admitted query
    if (!admitted.empty()) {
        int rc = begin_call(S->ictx, st);
        if (rc != IMLOC_OK) return rc;
    }
    for (ServeQuery* q : admitted) {
        const int64_t m_cap = q->opts.max_score_corr;
        const Layout L = layout_of(q->n, static_cast<int32_t>(m_cap), step_samples(S->cfg, q->B), q->R, !q->on_device);
        char* base = S->pool + q->pool_off;
        const float* dm[5];
        for (int k = 0; k < 5; ++k) {
            if (q->on_device) {
                dm[k] = q->dmatch[k];  // the lift reads the caller's device arrays
                continue;
            }
            float* dst = reinterpret_cast<float*>(base + L.match[k]);
            IMLOC_CUDA_TRY(cudaMemcpyAsync(dst, S->ring + q->ring_off + k * sizeof(float) * q->n,
                                           sizeof(float) * q->n, cudaMemcpyHostToDevice, st));
            dm[k] = dst;
        }
        imloc_matches m{dm[0], dm[1], dm[2], dm[3], dm[4], q->n, q->segs.data(), static_cast<int32_t>(q->segs.size())};
        imloc_corr c{reinterpret_cast<float*>(base + L.cx), reinterpret_cast<float*>(base + L.cy),
                     reinterpret_cast<float*>(base + L.cX), reinterpret_cast<float*>(base + L.cY),
                     reinterpret_cast<float*>(base + L.cZ), reinterpret_cast<float*>(base + L.cw),
                     reinterpret_cast<int32_t*>(base + L.csrc), reinterpret_cast<int32_t*>(base + L.ccount), q->n};
        const int64_t qb[2] = {0, q->n};
        int rc = lift_impl(S->ictx, 1, qb, q->views.data(), static_cast<int32_t>(q->views.size()), &m, &c, nullptr, st);
        if (rc != IMLOC_OK) return rc;
        fill_desc(S, q, L);
    }
    if (!admitted.empty()) {
        int rc = end_call(S->ictx, st);
        if (rc != IMLOC_OK) return rc;
    }
    int n_init = 0;
    for (ServeQuery* q : admitted) S->h_init[p][n_init++] = q->slot;
    // rounds of this step per resident query
    int64_t total = 0;
    for (int s = 0; s < ns; ++s) {
        ServeQuery* q = S->slots[s];
        S->occ[p][s] = q ? q->ticket : 0;
        WaveQ& w = S->h_wq[p][s];
        memset(&w, 0, sizeof(w));
        S->h_prefix[p][s] = total;
        if (!q) continue;
        const int64_t r0 = q->r_next;
        const int64_t r1 = std::min<int64_t>(q->R, r0 + (r0 == 0 ? 1 : std::max(1, S->cfg.rounds_per_step)));
        const int64_t sb = std::min(r0 * q->B, q->H), se = std::min(r1 * q->B, q->H);
        w.s_begin = sb;
        w.n_samples = static_cast<int32_t>(se - sb);
        w.r0 = static_cast<int32_t>(r0);
        w.r1 = static_cast<int32_t>(r1);
        total += se - sb;
        q->r_next = r1;
    }
    S->h_prefix[p][ns] = total;
    if (!admitted.empty()) {
        memcpy(S->h_qd[p], S->qd_master.data(), sizeof(QueryDesc) * ns);
        IMLOC_CUDA_TRY(cudaMemcpyAsync(S->d_qd, S->h_qd[p], sizeof(QueryDesc) * ns, cudaMemcpyHostToDevice, st));
        IMLOC_CUDA_TRY(cudaMemcpyAsync(S->d_init, S->h_init[p], sizeof(int32_t) * n_init, cudaMemcpyHostToDevice, st));
    }
    IMLOC_CUDA_TRY(cudaMemcpyAsync(S->d_wq, S->h_wq[p], sizeof(WaveQ) * ns, cudaMemcpyHostToDevice, st));
    IMLOC_CUDA_TRY(cudaMemcpyAsync(S->d_prefix, S->h_prefix[p], sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, st));
    IMLOC_CUDA_TRY(cudaMemsetAsync(S->d_nhyp, 0, sizeof(int32_t) * ns, st));
    StepBuffers b;
    b.d_qd = S->d_qd;
    b.d_qs = S->d_qs;
    b.d_wq = S->d_wq;
    b.d_prefix = S->d_prefix;
    b.d_nhyp = S->d_nhyp;
    b.d_tiles = S->d_tiles;
    b.d_counter = S->d_counter;
    b.d_nhyp_all = nullptr;
    b.nhyp_all_len = 0;
    b.d_init = S->d_init;
    b.any_fp64 = false;
    b.fuse = true;  // one launch less per step, replays overlap the other queries' scoring
    for (int s = 0; s < ns; ++s)
        if (S->slots[s] && S->slots[s]->opts.lo_fp64_accumulate) b.any_fp64 = true;
    int rc = run_step(S->ictx, b, ns, n_init, total, false, st);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaMemcpyAsync(S->h_qs[p], S->d_qs, sizeof(QueryState) * ns, cudaMemcpyDeviceToHost, st));
    IMLOC_CUDA_TRY(cudaMemcpyAsync(S->h_res[p], S->d_res, sizeof(imloc_result) * ns, cudaMemcpyDeviceToHost, st));
    IMLOC_CUDA_TRY(cudaEventRecord(S->step_done[p], st));
    S->step_admitted[p] = admitted;
    return IMLOC_OK;
}

// Wait for the step of parity p and retire its finished queries (only those
// still in the slot they held during that step).
static int retire_step(imloc_server* S, int p) {
    IMLOC_CUDA_TRY(cudaEventSynchronize(S->step_done[p]));
    const int ns = S->cfg.max_slots;
    const double t = now_ms();
    std::lock_guard<std::mutex> lk(S->mu);
    for (ServeQuery* q : S->step_admitted[p])
        if (!q->on_device) ring_release(S, q);
    S->step_admitted[p].clear();
    for (int s = 0; s < ns; ++s) {
        const uint64_t ticket = S->occ[p][s];
        S->occ[p][s] = 0;
        ServeQuery* q = S->slots[s];
        if (!ticket || !q || q->ticket != ticket || !S->h_qs[p][s].finished) continue;
        S->done[q->ticket] = {S->h_res[p][s], t - q->t_submit};
        S->live.erase(q->ticket);
        S->pool_alloc.release(q->pool_off, q->footprint);
        S->slots[s] = nullptr;
        S->stats.completed++;
        S->stats.resident--;
        delete q;
    }
    S->stats.steps++;
    S->stats.device_bytes_in_use = S->pool_alloc.in_use();
    return IMLOC_OK;
}

static void worker_main(imloc_server* S) {
    cudaSetDevice(S->device);
    int p = 0;               // parity of the next step to enqueue
    bool in_flight = false;  // a step of parity p ^ 1 is enqueued and not yet retired
    for (;;) {
        std::vector<ServeQuery*> admitted;
        bool any_resident;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            // admission: arrival order, free slot and device budget
            while (!S->pending.empty()) {
                ServeQuery* q = S->pending.front();
                int slot = -1;
                for (int s = 0; s < S->cfg.max_slots; ++s)
                    if (!S->slots[s]) { slot = s; break; }
                if (slot < 0) break;
                const size_t off = S->pool_alloc.alloc(q->footprint);
                if (off == SIZE_MAX) break;
                S->pending.pop_front();
                q->slot = slot;
                q->pool_off = off;
                S->slots[slot] = q;
                S->live[q->ticket] = 2;
                S->stats.admitted++;
                S->stats.pending--;
                S->stats.resident++;
                admitted.push_back(q);
            }
            any_resident = S->stats.resident > 0;
            if (!any_resident && !in_flight) {
                S->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        // the next step goes onto the stream before the previous one is retired
        bool enqueued = false;
        if (any_resident) {
            const int rc = enqueue_step(S, admitted, p);
            if (rc != IMLOC_OK) {
                fail_all(S, rc);
                break;
            }
            enqueued = true;
        }
        if (in_flight) {
            const int rc = retire_step(S, p ^ 1);
            if (rc != IMLOC_OK) {
                fail_all(S, rc);
                break;
            }
        }
        in_flight = enqueued;
        if (enqueued) p ^= 1;
    }
    // the last enqueued step completes before the server's memory goes away
    if (in_flight) cudaEventSynchronize(S->step_done[p ^ 1]);
}

}  // namespace imloc

extern "C" {

void imloc_serve_default_config(imloc_serve_config* c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->max_slots = 64;
    c->max_queue = 4096;
    c->device_budget_bytes = size_t(1) << 30;
    c->host_staging_bytes = size_t(256) << 20;
    c->rounds_per_step = 2;
}

int imloc_serve_create(imloc_ctx* ctx, const imloc_serve_config* cfg, imloc_server** out) {
    if (!ctx || !cfg || !out) return IMLOC_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_slots <= 0 || cfg->max_slots > 4096 || cfg->max_queue <= 0 || cfg->device_budget_bytes == 0 ||
        cfg->host_staging_bytes == 0 || cfg->rounds_per_step <= 0)
        return IMLOC_ERR_INVALID_ARG;
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    imloc_server* S = new imloc_server();
    S->cfg = *cfg;
    S->device = ctx->device;
    int rc = imloc_create(&S->ictx, ctx->device, size_t(64) << 20);
    const int ns = cfg->max_slots;
    bool ok = rc == IMLOC_OK;
    ok = ok && cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMalloc(&S->pool, cfg->device_budget_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_qd, sizeof(imloc::QueryDesc) * ns) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_qs, sizeof(imloc::QueryState) * ns) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_wq, sizeof(imloc::WaveQ) * ns) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_prefix, sizeof(int64_t) * (ns + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_nhyp, sizeof(int32_t) * ns) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_tiles, sizeof(int32_t) * (3 * ns + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_counter, sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_init, sizeof(int32_t) * ns) == cudaSuccess;
    ok = ok && cudaMalloc(&S->d_res, sizeof(imloc_result) * ns) == cudaSuccess;
    for (int k = 0; k < 2; ++k) {
        ok = ok && cudaMallocHost(&S->h_qd[k], sizeof(imloc::QueryDesc) * ns) == cudaSuccess;
        ok = ok && cudaMallocHost(&S->h_wq[k], sizeof(imloc::WaveQ) * ns) == cudaSuccess;
        ok = ok && cudaMallocHost(&S->h_prefix[k], sizeof(int64_t) * (ns + 1)) == cudaSuccess;
        ok = ok && cudaMallocHost(&S->h_init[k], sizeof(int32_t) * ns) == cudaSuccess;
        ok = ok && cudaMallocHost(&S->h_qs[k], sizeof(imloc::QueryState) * ns) == cudaSuccess;
        ok = ok && cudaMallocHost(&S->h_res[k], sizeof(imloc_result) * ns) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&S->step_done[k], cudaEventDisableTiming) == cudaSuccess;
        S->occ[k].assign(ns, 0);
    }
    ok = ok && cudaMallocHost(&S->ring, cfg->host_staging_bytes) == cudaSuccess;
    if (!ok) {
        imloc_serve_destroy(S);
        return rc != IMLOC_OK ? rc : IMLOC_ERR_OOM;
    }
    S->ring_bytes = cfg->host_staging_bytes;
    S->pool_alloc.reset(cfg->device_budget_bytes);
    S->slots.assign(ns, nullptr);
    S->qd_master.assign(ns, imloc::QueryDesc());
    memset(S->qd_master.data(), 0, sizeof(imloc::QueryDesc) * ns);
    // every slot starts finished: the kernels skip it until a query is set up there
    for (int s = 0; s < ns; ++s) {
        memset(&S->h_qs[0][s], 0, sizeof(imloc::QueryState));
        S->h_qs[0][s].done = 1;
        S->h_qs[0][s].finished = 1;
    }
    if (cudaMemcpy(S->d_qs, S->h_qs[0], sizeof(imloc::QueryState) * ns, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(S->d_qd, S->qd_master.data(), sizeof(imloc::QueryDesc) * ns, cudaMemcpyHostToDevice) != cudaSuccess) {
        imloc_serve_destroy(S);
        return IMLOC_ERR_CUDA;
    }
    S->worker = std::thread(imloc::worker_main, S);
    *out = S;
    return IMLOC_OK;
}

}  // extern "C"

namespace imloc {

static int serve_submit_impl(imloc_server* S, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                             const imloc_camera* qcam, const imloc_ransac_opts* opts, uint64_t* ticket, bool on_device) {
    if (!S || !views || n_views <= 0 || !m || !qcam || !opts || !ticket) return IMLOC_ERR_INVALID_ARG;
    if (m->n < 0 || m->n >= (int64_t(1) << 31) || (m->n > 0 && (!m->q_u || !m->q_v || !m->db_u || !m->db_v || !m->conf)))
        return IMLOC_ERR_INVALID_ARG;
    if (m->n > 0 && (!m->segments || m->n_segments <= 0 || m->segments[0].begin != 0)) return IMLOC_ERR_INVALID_ARG;
    if (!(opts->tau_px > 0.0) || opts->max_score_corr < 3 || opts->batch <= 0 || opts->max_iters <= 0 ||
        opts->enumerate_all)
        return IMLOC_ERR_INVALID_ARG;
    for (int s = 0; s < m->n_segments; ++s) {
        const imloc_segment& sg = m->segments[s];
        if (sg.view < 0 || sg.view >= n_views || (sg.direction != 0 && sg.direction != 1) || sg.begin > m->n ||
            (s > 0 && sg.begin < m->segments[s - 1].begin))
            return IMLOC_ERR_INVALID_ARG;
    }
    ServeQuery* q = new ServeQuery();
    q->views.assign(views, views + n_views);
    q->segs.assign(m->segments, m->segments + m->n_segments);
    q->n = m->n;
    q->cam = *qcam;
    q->opts = *opts;
    q->H = opts->max_iters;
    q->B = opts->batch;
    q->R = (q->H + q->B - 1) / q->B;
    q->on_device = on_device;
    q->footprint = layout_of(q->n, opts->max_score_corr, step_samples(S->cfg, q->B), q->R, !on_device).total;
    const float* src[5] = {m->q_u, m->q_v, m->db_u, m->db_v, m->conf};
    if (on_device)
        for (int k = 0; k < 5; ++k) q->dmatch[k] = src[k];
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->worker_error != IMLOC_OK || S->stop) {
        delete q;
        return S->worker_error != IMLOC_OK ? S->worker_error : IMLOC_ERR_INVALID_ARG;
    }
    // never admissible, queue full, or no room in the staging ring: refused
    if (q->footprint > S->cfg.device_budget_bytes || static_cast<int>(S->pending.size()) >= S->cfg.max_queue ||
        (!on_device && !ring_alloc(S, sizeof(float) * 5 * static_cast<size_t>(q->n), q))) {
        S->stats.rejected++;
        delete q;
        return IMLOC_ERR_REJECTED;
    }
    if (!on_device)
        for (int k = 0; k < 5; ++k)
            if (q->n) memcpy(S->ring + q->ring_off + k * sizeof(float) * q->n, src[k], sizeof(float) * q->n);
    q->ticket = S->next_ticket++;
    q->t_submit = now_ms();
    S->pending.push_back(q);
    S->live[q->ticket] = 1;
    S->stats.submitted++;
    S->stats.pending++;
    *ticket = q->ticket;
    S->cv.notify_one();
    return IMLOC_OK;
}

}  // namespace imloc

extern "C" {

int imloc_serve_submit(imloc_server* S, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                       const imloc_camera* qcam, const imloc_ransac_opts* opts, uint64_t* ticket) {
    return imloc::serve_submit_impl(S, views, n_views, m, qcam, opts, ticket, false);
}

int imloc_serve_submit_device(imloc_server* S, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                              const imloc_camera* qcam, const imloc_ransac_opts* opts, uint64_t* ticket) {
    return imloc::serve_submit_impl(S, views, n_views, m, qcam, opts, ticket, true);
}

int imloc_serve_poll(imloc_server* S, uint64_t ticket, imloc_result* out, double* latency_ms) {
    if (!S || !out) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it != S->done.end()) {
        *out = it->second.first;
        if (latency_ms) *latency_ms = it->second.second;
        S->done.erase(it);
        return IMLOC_OK;
    }
    if (S->live.count(ticket)) return IMLOC_PENDING;
    return IMLOC_ERR_NOT_FOUND;
}

int imloc_serve_read_stats(imloc_server* S, imloc_serve_stats* out) {
    if (!S || !out) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return S->worker_error;
}

int imloc_serve_destroy(imloc_server* S) {
    if (!S) return IMLOC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (ServeQuery* q : S->pending) delete q;
    for (ServeQuery* q : S->slots) delete q;
    cudaFree(S->pool);
    cudaFree(S->d_qd); cudaFree(S->d_qs); cudaFree(S->d_wq); cudaFree(S->d_prefix); cudaFree(S->d_nhyp);
    cudaFree(S->d_tiles); cudaFree(S->d_counter); cudaFree(S->d_init); cudaFree(S->d_res);
    for (int k = 0; k < 2; ++k) {
        cudaFreeHost(S->h_qd[k]); cudaFreeHost(S->h_wq[k]); cudaFreeHost(S->h_prefix[k]); cudaFreeHost(S->h_init[k]);
        cudaFreeHost(S->h_qs[k]); cudaFreeHost(S->h_res[k]);
        if (S->step_done[k]) cudaEventDestroy(S->step_done[k]);
    }
    cudaFreeHost(S->ring);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->ictx) imloc_destroy(S->ictx);
    delete S;
    return IMLOC_OK;
}

}  // extern "C"
