// Serving loop: continuous batching of motif queries over one resident graph.
//
// A scheduler thread owns `streams` slots.  Whenever a slot is free and
// requests are waiting, it forms a batch under the server lock and launches it
// without the lock (submit and poll never wait behind CUDA calls): a count
// launch for every request of the batch, then, for the enumerate requests, a
// chunk-offset scan per request and one multi-query fill launch.  Completion
// is detected with CUDA events; results stay on the device until released.
// Requests arriving while batches run are admitted as slots and memory free
// up (continuous batching).
//
// Batches are formed by expected cost.  The graph keeps, per motif shape,
// delta bucket and flavour (count / enumerate), a running estimate of the
// device time one request takes, learnt from the launches its servers have
// timed (so a new server of the same graph starts with what earlier ones
// learnt).  The
// oldest waiting request that fits the memory budget always leads the next
// batch.  A request expected to take long (or never seen) runs alone; short
// ones are grouped with later short requests until the batch's expected time
// reaches a budget, so a short request never waits for a long one inside a
// batch.  Inside a batch the longest request comes first: the persistent
// kernel claims root chunks in query order, so the critical path starts
// first and the short requests fill its tail.  Short batches go to a
// high-priority stream, so when launches queue for the SMs theirs are placed
// first.  Each launch's persistent grid can be limited to a share of the GPU,
// leaving room for launches on other slots to run beside it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tm_internal.cuh"

namespace tmg {

namespace {

using clk = std::chrono::steady_clock;

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Req {
    uint64_t ticket = 0;
    tm_query* q = nullptr;
    Plan plan{};
    int enumerate = 0;
    uint64_t cap = 0;
    uint64_t need = 0;          // admitted device bytes
    uint64_t key = 0;           // cost-model key: shape, delta bucket, flavour
    double est_ms = -1.0;       // expected device time when batched (< 0: unknown)
    int occ = 0;                // launch shape (resident grid, warps per block) of the request alone
    ReqState state = QUEUED;
    clk::time_point t_submit, t_done;
    int32_t* match = nullptr;   // device rows (enumerate)
    unsigned long long* chunk = nullptr;  // device chunk counts / offsets
    void* scan_tmp = nullptr;
    uint64_t nch = 0;
    uint64_t total = 0, n_written = 0;
    tm_status status = TM_OK;
};

struct Slot {
    cudaStream_t st_hi = nullptr, st_lo = nullptr;   // high / low priority
    cudaStream_t st = nullptr;                       // the one the current batch runs on
    cudaEvent_t start = nullptr, done = nullptr;
    Scratch count_s, fill_s;    // staging + scratch of the two launches
    std::vector<Req*> batch;
    bool busy = false;
};

}  // namespace

}  // namespace tmg

using namespace tmg;

struct tm_server {
    tm_graph* g = nullptr;
    tm_serve_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_ticket = 1;
    uint64_t mem_used = 0;
    bool stop = false;
    std::vector<Slot> slots;
    std::thread th;
    cudaStream_t free_st = nullptr;
};

namespace tmg {

namespace {

uint64_t req_bytes(const tm_graph* g, const Plan& p, int enumerate, uint64_t cap) {
    if (!enumerate) return 0;
    uint64_t nch = ((uint64_t)g->v.m + p.tune.chunk_roots - 1) / (uint64_t)p.tune.chunk_roots;
    return cap * (uint64_t)p.k * 4 + chunk_buf_bytes(nch) + scan_temp_bytes(nch + 1);
}

uint64_t cost_key(const Plan& p, int enumerate) {
    int bucket = 0;
    for (int64_t d = p.delta; d > 0; d >>= 1) ++bucket;
    return (p.shape_hash * 1099511628211ULL) ^ ((uint64_t)bucket << 1) ^ (uint64_t)(enumerate != 0);
}

double estimate(const tm_server* s, const Req* r) {
    std::lock_guard<std::mutex> lk(s->g->cost_mu);
    auto it = s->g->serve_cost_ms.find(r->key);
    return it == s->g->serve_cost_ms.end() ? -1.0 : it->second;
}

// The persistent grid of one launch: the full resident grid, or the configured share of it.
int launch_grid(const tm_server* s, const LaunchCfg& c) {
    const int pct = s->cfg.grid_pct;
    if (pct <= 0 || pct >= 100) return c.grid;
    return std::max(s->g->num_sms, c.grid * pct / 100);
}

tm_status launch_batch(tm_server* s, Slot& sl) {
    tm_graph* g = s->g;
    const int nq = (int)sl.batch.size();
    const uint64_t m = (uint64_t)g->v.m;
    TM_CUDA(cudaEventRecord(sl.start, sl.st));
    tm_status r = scratch_reserve(&sl.count_s, g->device, nq, (uint64_t)nq, 0, 1u << 18);
    if (r != TM_OK) return r;
    r = scratch_reserve(&sl.fill_s, g->device, nq, (uint64_t)nq, 0, 0);
    if (r != TM_OK) return r;
    // enumerate buffers (stream-ordered allocations: no device-wide sync)
    for (Req* q : sl.batch) {
        if (!q->enumerate) continue;
        q->nch = (m + q->plan.tune.chunk_roots - 1) / (uint64_t)q->plan.tune.chunk_roots;
        TM_CUDA(dev_malloc_async((void**)&q->match, std::max<uint64_t>(q->cap * q->plan.k * 4, 16), sl.st));
        TM_CUDA(dev_malloc_async((void**)&q->chunk, chunk_buf_bytes(q->nch), sl.st));
        TM_CUDA(dev_malloc_async(&q->scan_tmp, scan_temp_bytes(q->nch + 1), sl.st));
        TM_CUDA(cudaMemsetAsync(q->chunk, 0, (q->nch + 2) * 8, sl.st));   // counts + list length
    }
    // count launch over every request of the batch
    Scratch& cs = sl.count_s;
    Ctrl* c = cs.ctrl_stage();
    memset(c, 0, sizeof(Ctrl));
    uint64_t base = 0;
    int warp_smem = 16, warps = 1;
    unsigned feat = 0, ffeat = 0;
    for (int j = 0; j < nq; ++j) {
        Req* q = sl.batch[j];
        QueryDev* qd = cs.qdev_stage() + j;
        memset(qd, 0, sizeof(QueryDev));
        qd->plan = q->plan;
        qd->root_begin = 0;
        qd->root_end = m;
        qd->n_chunks = (m + q->plan.tune.chunk_roots - 1) / (uint64_t)q->plan.tune.chunk_roots;
        qd->chunk_base = base;
        base += qd->n_chunks;
        qd->total = cs.counters + j;
        qd->chunk_cnt = q->enumerate ? q->chunk : nullptr;
        warp_smem = std::max(warp_smem, q->plan.warp_smem);
        warps = std::max(warps, q->plan.tune.warps_per_block);
        feat |= plan_features(q->plan);
        if (q->enumerate) ffeat |= plan_features(q->plan);
    }
    c->total_chunks = base;
    TM_CUDA(cudaMemcpyAsync(cs.head, cs.stage, cs.head_bytes(nq), cudaMemcpyHostToDevice, sl.st));
    TM_CUDA(cudaMemsetAsync(cs.counters, 0, (size_t)nq * 8, sl.st));
    TM_CUDA(cudaMemsetAsync(cs.ready, 0, cs.task_cap, sl.st));
    LaunchCfg lc = search_launch_cfg(g, MODE_COUNT, warp_smem, warps);
    r = launch_search(g, MODE_COUNT, cs.qdev(), nq, warp_smem, warps, feat, &cs, sl.st, launch_grid(s, lc));
    if (r != TM_OK) return r;
    // fill launch over the enumerate requests
    int ne = 0;
    Scratch& fs = sl.fill_s;
    Ctrl* fc = fs.ctrl_stage();
    memset(fc, 0, sizeof(Ctrl));
    uint64_t fbase = 0;
    int fsmem = 16;
    for (Req* q : sl.batch) {
        if (!q->enumerate) continue;
        r = exclusive_scan_u64(q->chunk, q->chunk, q->nch + 1, q->scan_tmp, sl.st);
        if (r != TM_OK) return r;
        r = list_chunks(q->chunk, q->nch, q->cap, g->num_sms, sl.st);
        if (r != TM_OK) return r;
        QueryDev* qd = fs.qdev_stage() + ne;
        memset(qd, 0, sizeof(QueryDev));
        qd->plan = q->plan;
        qd->root_begin = 0;
        qd->root_end = m;
        qd->n_chunks = q->nch;
        qd->chunk_base = fbase;
        fbase += q->nch;
        qd->total = fs.counters + ne;
        qd->chunk_off = q->chunk;
        qd->match_out = q->match;
        qd->cap = q->cap;
        fsmem = std::max(fsmem, q->plan.warp_smem_fill);
        ++ne;
    }
    if (ne > 0) {
        fc->total_chunks = fbase;
        TM_CUDA(cudaMemcpyAsync(fs.head, fs.stage, fs.head_bytes(ne), cudaMemcpyHostToDevice, sl.st));
        LaunchCfg lf = search_launch_cfg(g, MODE_FILL, fsmem, warps);
        r = launch_search(g, MODE_FILL, fs.qdev(), ne, fsmem, warps, ffeat, &fs, sl.st, launch_grid(s, lf));
        if (r != TM_OK) return r;
    }
    TM_CUDA(cudaMemcpyAsync(cs.counters_host, cs.counters, (size_t)nq * 8, cudaMemcpyDeviceToHost, sl.st));
    TM_CUDA(cudaMemcpyAsync(cs.stage, cs.head, sizeof(Ctrl), cudaMemcpyDeviceToHost, sl.st));
    for (Req* q : sl.batch) {
        if (!q->enumerate) continue;
        TM_CUDA(cudaFreeAsync(q->chunk, sl.st));
        TM_CUDA(cudaFreeAsync(q->scan_tmp, sl.st));
        q->chunk = nullptr;
        q->scan_tmp = nullptr;
    }
    TM_CUDA(cudaEventRecord(sl.done, sl.st));
    return TM_OK;
}

// Learn per-request device times from a finished batch: its measured time is
// shared among its requests in proportion to their estimates (unknown ones
// count as the batch's mean), and each estimate moves a third of the way.
void learn(tm_server* s, Slot& sl) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sl.start, sl.done) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    double known = 0.0;
    int n_known = 0;
    for (Req* q : sl.batch)
        if (q->est_ms > 0) { known += q->est_ms; ++n_known; }
    const double unknown_w = n_known ? known / n_known : 1.0;
    double wsum = 0.0;
    for (Req* q : sl.batch) wsum += q->est_ms > 0 ? q->est_ms : unknown_w;
    std::lock_guard<std::mutex> lk(s->g->cost_mu);
    auto& cost = s->g->serve_cost_ms;
    for (Req* q : sl.batch) {
        const double share = ms * (q->est_ms > 0 ? q->est_ms : unknown_w) / wsum;
        auto it = cost.find(q->key);
        if (it == cost.end()) cost[q->key] = share;
        else it->second += (share - it->second) / 3.0;
    }
}

void finish_batch(tm_server* s, Slot& sl, tm_status launch_status) {
    // caller holds s->mu
    bool timeout = launch_status == TM_OK && sl.count_s.ctrl_stage()->err != 0;
    if (launch_status == TM_OK && !timeout) learn(s, sl);
    auto now = clk::now();
    for (size_t j = 0; j < sl.batch.size(); ++j) {
        Req* q = sl.batch[j];
        q->t_done = now;
        if (launch_status != TM_OK) {
            q->status = launch_status;
        } else if (timeout) {
            q->status = TM_E_TIMEOUT;
        } else {
            q->total = sl.count_s.counters_host[j];
            q->n_written = q->enumerate ? std::min(q->total, q->cap) : 0;
            q->status = (q->enumerate && q->total > q->cap) ? TM_E_TRUNCATED : TM_OK;
        }
        if (q->status != TM_OK && q->status != TM_E_TRUNCATED) {
            // a failed request keeps no device memory (frees are ordered after its launches)
            if (q->match) cudaFreeAsync(q->match, sl.st);
            if (q->chunk) cudaFreeAsync(q->chunk, sl.st);
            if (q->scan_tmp) cudaFreeAsync(q->scan_tmp, sl.st);
            cudaGetLastError();
            q->match = nullptr;
            q->chunk = nullptr;
            q->scan_tmp = nullptr;
            q->n_written = 0;
        }
        // chunk scratch was freed on the stream; the match buffer stays until release
        uint64_t keep = q->match ? q->cap * (uint64_t)q->plan.k * 4 : 0;
        s->mem_used -= (q->need - keep);
        q->need = keep;
        q->state = DONE;
    }
    sl.batch.clear();
    sl.busy = false;
}

// Form the next batch for a free slot (caller holds s->mu): the oldest request
// that fits the memory budget leads; with the cost-aware policy, short
// requests behind it join while the batch's expected time stays within
// batch_ms, and a long or never-seen leader runs alone.  Returns false when
// nothing can be admitted.
bool pick_batch(tm_server* s, Slot& sl) {
    const int max_batch = s->cfg.max_batch;
    const bool by_cost = s->cfg.policy == 0;
    const double long_ms = s->cfg.long_ms, budget = s->cfg.batch_ms;
    auto fits = [&](const Req* q) { return s->mem_used + q->need <= s->cfg.mem_budget_bytes; };
    auto lead = s->pending.begin();
    while (lead != s->pending.end() && !fits(*lead)) ++lead;
    if (lead == s->pending.end()) return false;
    Req* head = *lead;
    head->est_ms = estimate(s, head);
    std::vector<std::deque<Req*>::iterator> take{lead};
    s->mem_used += head->need;
    const bool head_short = head->est_ms >= 0 && head->est_ms < long_ms;
    if (!by_cost || head_short) {
        double total = head->est_ms;
        for (auto it = std::next(lead); it != s->pending.end() && (int)take.size() < max_batch; ++it) {
            Req* q = *it;
            if (!fits(q)) continue;
            if (by_cost) {
                // same occupancy as the leader: one launch shares one frame size
                if (q->occ != head->occ) continue;
                q->est_ms = estimate(s, q);
                if (q->est_ms < 0 || q->est_ms >= long_ms || total + q->est_ms > budget) continue;
                total += q->est_ms;
            }
            s->mem_used += q->need;
            take.push_back(it);
        }
    }
    for (auto it : take) {
        (*it)->state = RUNNING;
        sl.batch.push_back(*it);
    }
    // one pass drops the taken requests (an erase inside a deque would invalidate
    // the other iterators kept in `take`)
    s->pending.erase(std::remove_if(s->pending.begin(), s->pending.end(),
                                    [](const Req* r) { return r->state == RUNNING; }),
                     s->pending.end());
    if (by_cost)   // the critical path first: the kernel claims chunks in query order
        std::stable_sort(sl.batch.begin(), sl.batch.end(),
                         [](const Req* a, const Req* b) { return a->est_ms > b->est_ms; });
    sl.st = (by_cost && head_short) ? sl.st_hi : sl.st_lo;
    return true;
}

void scheduler(tm_server* s) {
    cudaSetDevice(s->g->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // completions
        bool any_busy = false;
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaSuccess) {
                finish_batch(s, sl, TM_OK);
                s->cv_done.notify_all();
            } else if (e != cudaErrorNotReady) {
                cudaGetLastError();
                finish_batch(s, sl, TM_E_CUDA);
                s->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        if (s->stop && s->pending.empty() && !any_busy) break;
        // admission into a free slot; the launch itself runs without the lock
        Slot* free_slot = nullptr;
        for (Slot& sl : s->slots)
            if (!sl.busy) { free_slot = &sl; break; }
        if (free_slot && !s->pending.empty() && pick_batch(s, *free_slot)) {
            free_slot->busy = true;
            lk.unlock();
            tm_status r = launch_batch(s, *free_slot);
            lk.lock();
            if (r != TM_OK) {
                finish_batch(s, *free_slot, r);
                s->cv_done.notify_all();
            }
            continue;
        }
        if (any_busy) {
            // batches in flight: poll their events at microsecond granularity
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            s->cv_work.wait_for(lk, std::chrono::microseconds(2000));
        }
    }
}

void destroy_slots(tm_server* s) {
    for (Slot& sl : s->slots) {
        scratch_free(&sl.count_s);
        scratch_free(&sl.fill_s);
        if (sl.start) cudaEventDestroy(sl.start);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st_hi) cudaStreamDestroy(sl.st_hi);
        if (sl.st_lo) cudaStreamDestroy(sl.st_lo);
    }
    if (s->free_st) cudaStreamDestroy(s->free_st);
    cudaGetLastError();
}

}  // namespace

}  // namespace tmg

extern "C" tm_status tm_serve_start(tm_graph* g, const tm_serve_cfg* cfg, tm_server** out) {
    if (!g || !out) { set_error("null argument"); return TM_E_INVALID; }
    if (cfg && (cfg->grid_pct < 0 || cfg->grid_pct > 100 || cfg->policy < 0 || cfg->policy > 1 ||
                cfg->long_ms < 0 || cfg->batch_ms < 0)) {
        set_error("serving configuration out of range");
        return TM_E_INVALID;
    }
    TM_ENTER(g->device);
    tm_server* s = new tm_server();
    s->g = g;
    if (cfg) s->cfg = *cfg;
    if (s->cfg.mem_budget_bytes == 0) s->cfg.mem_budget_bytes = 4ull << 30;
    if (s->cfg.streams <= 0) s->cfg.streams = 2;
    if (s->cfg.streams > 32) s->cfg.streams = 32;
    if (s->cfg.max_batch <= 0) s->cfg.max_batch = 16;
    if (s->cfg.grid_pct == 0) s->cfg.grid_pct = 100;
    if (s->cfg.long_ms == 0) s->cfg.long_ms = 1.0;
    if (s->cfg.batch_ms == 0) s->cfg.batch_ms = 2.0;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    s->slots.resize(s->cfg.streams);
    bool ok = cudaStreamCreateWithFlags(&s->free_st, cudaStreamNonBlocking) == cudaSuccess;
    for (Slot& sl : s->slots) {
        ok = ok && cudaStreamCreateWithPriority(&sl.st_hi, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
             cudaStreamCreateWithPriority(&sl.st_lo, cudaStreamNonBlocking, prio_lo) == cudaSuccess &&
             cudaEventCreate(&sl.start) == cudaSuccess && cudaEventCreate(&sl.done) == cudaSuccess;
        sl.st = sl.st_lo;
    }
    if (!ok) {
        cudaGetLastError();
        set_error("stream/event creation failed");
        destroy_slots(s);
        delete s;
        return TM_E_CUDA;
    }
    // keep freed match buffers in the device's stream-ordered pool instead of
    // returning them to the driver at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, g->device) == cudaSuccess) {
        uint64_t keep = s->cfg.mem_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    s->th = std::thread(scheduler, s);
    *out = s;
    return TM_OK;
}

extern "C" tm_status tm_serve_submit(tm_server* s, tm_query* q, int enumerate, uint64_t cap, uint64_t* ticket) {
    if (!s || !q || !ticket) { set_error("null argument"); return TM_E_INVALID; }
    if (enumerate && cap < 1) { set_error("enumerate request needs cap >= 1"); return TM_E_INVALID; }
    if (query_graph(q) != s->g) { set_error("query compiled for another graph"); return TM_E_INVALID; }
    std::unique_ptr<Req> r(new Req());
    // snapshot the plan (with the graph's tuning for this shape) at submit time
    query_plan(q, &r->plan);
    r->q = q;
    r->enumerate = enumerate ? 1 : 0;
    r->cap = enumerate ? cap : 0;
    r->need = req_bytes(s->g, r->plan, r->enumerate, r->cap);
    r->key = cost_key(r->plan, r->enumerate);
    TM_ENTER(s->g->device);   // the launch shape may query the device's occupancy once
    const LaunchCfg lc = search_launch_cfg(s->g, MODE_COUNT, r->plan.warp_smem, r->plan.tune.warps_per_block);
    r->occ = lc.grid * 32 + lc.warps_per_block;
    if (r->need > s->cfg.mem_budget_bytes) {
        set_error("request needs more device memory than the serving budget");
        return TM_E_ADMISSION;
    }
    r->t_submit = clk::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) { set_error("server stopping"); return TM_E_INVALID; }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->pending.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
    s->cv_work.notify_one();
    return TM_OK;
}

static void fill_result(const Req* r, tm_result* out) {
    out->status = r->status;
    out->total = r->total;
    out->n_written = r->n_written;
    out->matches_dev = r->match;
    out->k = r->plan.k;
    out->submit_to_done_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
}

extern "C" tm_status tm_serve_poll(tm_server* s, uint64_t ticket, tm_result* out) {
    if (!s || !out) { set_error("null argument"); return TM_E_INVALID; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket"); return TM_E_INVALID; }
    if (it->second->state != DONE) return TM_E_BUSY;
    fill_result(it->second.get(), out);
    return TM_OK;
}

extern "C" tm_status tm_serve_wait(tm_server* s, uint64_t ticket, int64_t timeout_ms, tm_result* out) {
    if (!s || !out) { set_error("null argument"); return TM_E_INVALID; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket"); return TM_E_INVALID; }
    Req* r = it->second.get();
    bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max<int64_t>(0, timeout_ms)),
                                  [&] { return r->state == DONE; });
    if (!ok) { set_error("request still running at timeout"); return TM_E_TIMEOUT; }
    fill_result(r, out);
    return TM_OK;
}

extern "C" tm_status tm_result_release(tm_server* s, uint64_t ticket) {
    if (!s) { set_error("null argument"); return TM_E_INVALID; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("unknown ticket"); return TM_E_INVALID; }
    Req* r = it->second.get();
    if (r->state != DONE) { set_error("request not finished"); return TM_E_BUSY; }
    if (r->match) {
        cudaSetDevice(s->g->device);
        cudaFreeAsync(r->match, s->free_st);
        r->match = nullptr;
    }
    s->mem_used -= r->need;
    s->reqs.erase(it);
    return TM_OK;
}

extern "C" tm_status tm_serve_stop(tm_server* s) {
    if (!s) return TM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->g->device);
    for (auto& kv : s->reqs)
        if (kv.second->match) cudaFreeAsync(kv.second->match, s->free_st);
    cudaStreamSynchronize(s->free_st);
    for (Slot& sl : s->slots) {
        if (sl.st_hi) cudaStreamSynchronize(sl.st_hi);
        if (sl.st_lo) cudaStreamSynchronize(sl.st_lo);
    }
    destroy_slots(s);
    delete s;
    return TM_OK;
}
