// C ABI: query compilation (the per-level plan), count, enumerate, batched
// count (CUDA-graph replay), work counters, autotuning, status strings.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "tm_internal.cuh"

namespace tmg {

static thread_local std::string g_last_error;
static thread_local uint64_t g_last_donated = 0, g_last_reserved = 0;
static std::atomic<uint64_t> g_launches{0};

void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

void note_search_stats(const Ctrl& c) {
    g_last_donated = c.donated;
    g_last_reserved = c.q_reserve;
}

// Allocations left before an injected failure (-1: none armed).
static std::atomic<int64_t> g_alloc_fault{-1};

static bool alloc_fault_due() {
    int64_t v = g_alloc_fault.load();
    while (v >= 0) {
        if (g_alloc_fault.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
    if (alloc_fault_due()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    if (alloc_fault_due()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, st);
}

cudaError_t host_alloc_pinned(void** p, size_t bytes) {
    if (alloc_fault_due()) return cudaErrorMemoryAllocation;
    return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

tm_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TM_E_OOM : TM_E_CUDA;
}

// ---------------------------------------------------------------- the plan

uint64_t plan_shape_hash(const tm_motif* m) {
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&](uint64_t x) { h = (h ^ x) * 1099511628211ULL; };
    mix((uint64_t)m->k);
    mix((uint64_t)m->n_nodes);
    for (int i = 0; i < m->k; ++i) {
        mix(m->esrc[i]);
        mix(m->edst[i]);
        mix((uint64_t)(m->elabel[i] >= 0));
        if (i + 1 < m->k) mix((uint64_t)(m->gap[i] != INT64_MAX));
    }
    for (int j = 0; j < m->n_nodes; ++j) mix((uint64_t)(m->nlabel[j] >= 0));
    mix((uint64_t)m->n_anti);
    for (int a = 0; a < m->n_anti; ++a) {
        mix(m->anti_src[a]);
        mix(m->anti_dst[a]);
        mix(m->anti_edge[a]);
    }
    return h;
}

// Per-level plan of a motif (paper Section 5.1.2): motif nodes get slots in
// the order they are first bound; level i reads the candidate list of an
// already-mapped endpoint (out-list of x_i, in-list of y_i, the shorter of the
// two when both are mapped, or the whole edge list when neither is), and only
// the slots bound so far are compared against a new node.
tm_status build_plan(const tm_graph* g, const tm_motif* m, Plan* out) {
    if (!m) { set_error("null motif"); return TM_E_INVALID; }
    const int k = m->k, nn = m->n_nodes;
    if (k < 1 || k > TM_MAX_EDGES) { set_error("k must be in [1, 8]"); return TM_E_INVALID; }
    if (nn < 2 || nn > TM_MAX_NODES) { set_error("n_nodes must be in [2, 8]"); return TM_E_INVALID; }
    if (m->delta < 0) { set_error("delta must be >= 0"); return TM_E_INVALID; }
    bool used[TM_MAX_NODES] = {false};
    for (int i = 0; i < k; ++i) {
        if (m->esrc[i] >= nn || m->edst[i] >= nn) { set_error("motif node id >= n_nodes"); return TM_E_INVALID; }
        if (m->esrc[i] == m->edst[i]) { set_error("motif self-loop"); return TM_E_INVALID; }
        used[m->esrc[i]] = used[m->edst[i]] = true;
        if (m->elabel[i] < -1 || m->elabel[i] > 255) { set_error("edge label out of range"); return TM_E_INVALID; }
        if (m->elabel[i] >= 0 && g && !g->v.elabel && g->v.m > 0) { set_error("edge label constraint on a graph without edge labels"); return TM_E_INVALID; }
        if (i + 1 < k && m->gap[i] < 0) { set_error("gap must be >= 0"); return TM_E_INVALID; }
    }
    if (m->n_anti < 0 || m->n_anti > TM_MAX_ANTI) { set_error("n_anti must be in [0, 4]"); return TM_E_INVALID; }
    for (int a = 0; a < m->n_anti; ++a) {
        if (m->anti_src[a] >= nn || m->anti_dst[a] >= nn || !used[m->anti_src[a]] || !used[m->anti_dst[a]] ||
            m->anti_src[a] == m->anti_dst[a]) {
            set_error("anti-edge endpoints must be two distinct nodes of the motif's edges");
            return TM_E_INVALID;
        }
        if (m->anti_edge[a] >= k || m->anti_delta[a] < 0) { set_error("anti-edge attached edge or delta out of range"); return TM_E_INVALID; }
    }
    for (int j = 0; j < nn; ++j) {
        if (!used[j]) { set_error("motif node not used by any edge"); return TM_E_INVALID; }
        if (m->nlabel[j] < -1 || m->nlabel[j] > 255) { set_error("node label out of range"); return TM_E_INVALID; }
        if (m->nlabel[j] >= 0 && g && !g->v.nlabel && g->v.n > 0) { set_error("node label constraint on a graph without node labels"); return TM_E_INVALID; }
    }
    Plan p;
    memset(&p, 0, sizeof p);
    p.k = k;
    p.n_nodes = nn;
    p.delta = m->delta;
    p.elabel0 = m->elabel[0];
    p.nl_x0 = m->nlabel[m->esrc[0]];
    p.nl_y0 = m->nlabel[m->edst[0]];
    int slot[TM_MAX_NODES], bound_at[TM_MAX_NODES];
    for (int j = 0; j < TM_MAX_NODES; ++j) slot[j] = bound_at[j] = -1;
    slot[m->esrc[0]] = 0;
    slot[m->edst[0]] = 1;
    bound_at[m->esrc[0]] = bound_at[m->edst[0]] = 0;
    for (int i = 1; i < k; ++i)
        for (int nd : {(int)m->esrc[i], (int)m->edst[i]})
            if (bound_at[nd] < 0) bound_at[nd] = i;
    // anti-edges: checked at the first level where both nodes and the attached edge are bound
    p.n_anti = m->n_anti;
    int anti_level[TM_MAX_ANTI];
    for (int a = 0; a < m->n_anti; ++a) {
        anti_level[a] = std::max((int)m->anti_edge[a], std::max(bound_at[m->anti_src[a]], bound_at[m->anti_dst[a]]));
        p.anti[a].edge = (int8_t)m->anti_edge[a];
        p.anti[a].delta = m->anti_delta[a];
        p.anti[a].same_pair = m->esrc[m->anti_edge[a]] == m->anti_src[a] && m->edst[m->anti_edge[a]] == m->anti_dst[a];
        if (anti_level[a] == 0) p.anti_mask0 |= (uint8_t)(1u << a);
    }
    int nb = 2;
    int off_c = 0, off_f = 0;
    for (int i = 1; i < k; ++i) {
        LevelPlan& lp = p.lv[i];
        const int x = m->esrc[i], y = m->edst[i];
        lp.nb = (int8_t)nb;
        lp.elabel = m->elabel[i];
        lp.gap = m->gap[i - 1];
        lp.nl0 = lp.nl1 = -1;
        lp.a = lp.b = -1;
        lp.nx_a = lp.nx_b = NX_NONE;
        // lists of an endpoint of edge i-1 start right after that edge's time:
        // their window start is read from the graph's successor index
        const int px = slot[m->esrc[i - 1]], py = slot[m->edst[i - 1]];
        auto succ = [&](int s, bool in_list) -> int8_t {
            if (s == px) return in_list ? NX_IN_SRC : NX_OUT_SRC;
            if (s == py) return in_list ? NX_IN_DST : NX_OUT_DST;
            return NX_NONE;
        };
        if (slot[x] >= 0 && slot[y] >= 0) {
            lp.kind = CLOSE; lp.a = (int8_t)slot[x]; lp.b = (int8_t)slot[y];
            lp.nx_a = succ(lp.a, false);
            lp.nx_b = succ(lp.b, true);
        } else if (slot[x] >= 0) {
            lp.kind = EXT_OUT; lp.a = (int8_t)slot[x]; slot[y] = nb++; lp.nl0 = m->nlabel[y];
            lp.nx_a = succ(lp.a, false);
        } else if (slot[y] >= 0) {
            lp.kind = EXT_IN; lp.a = (int8_t)slot[y]; slot[x] = nb++; lp.nl0 = m->nlabel[x];
            lp.nx_a = succ(lp.a, true);
        } else {
            lp.kind = FREE; slot[x] = nb++; slot[y] = nb++; lp.nl0 = m->nlabel[x]; lp.nl1 = m->nlabel[y];
        }
        for (int a = 0; a < m->n_anti; ++a)
            if (anti_level[a] == i) lp.anti_mask |= (uint8_t)(1u << a);
        lp.frame_off = off_c;
        lp.frame_off_fill = off_f;
        lp.anti_row_off = frame_bytes(lp.nb, i, false);
        lp.anti_row_off_fill = frame_bytes(lp.nb, i, true);
        off_c += frame_bytes(lp.nb, i, false, m->n_anti);
        off_f += frame_bytes(lp.nb, i, true, m->n_anti);
    }
    for (int a = 0; a < m->n_anti; ++a) {
        p.anti[a].xs = (int8_t)slot[m->anti_src[a]];
        p.anti[a].ys = (int8_t)slot[m->anti_dst[a]];
    }
    // Look-ahead: a later motif edge j whose two nodes are both bound by
    // edge i < j - 1 needs some graph edge between their images after t_i
    // and within the root's delta; checking that when edge i binds prunes
    // partial matches that cannot complete (the next edge is checked by its
    // own window anyway).  Only for pairs no earlier motif edge joins: a
    // chord between nodes that have not interacted yet rarely has an edge
    // in the window, while a pair that recurs (ping-pongs) mostly does, and
    // there the check costs more than it prunes.
    for (int j = 2; j < k; ++j) {
        const int x = m->esrc[j], y = m->edst[j];
        const int bl = std::max(bound_at[x], bound_at[y]);
        if (j < bl + 2) continue;
        bool recurs = false;
        for (int l = 0; l < j; ++l) recurs |= m->esrc[l] == x && m->edst[l] == y;
        if (recurs) continue;
        LevelPlan& L = p.lv[bl];
        bool dup = false;
        for (int l = 0; l < L.n_look; ++l) dup |= L.look_u[l] == slot[x] && L.look_v[l] == slot[y];
        if (dup || L.n_look >= TM_MAX_LOOK) continue;
        L.look_u[L.n_look] = (int8_t)slot[x];
        L.look_v[L.n_look] = (int8_t)slot[y];
        L.n_look++;
    }
    p.warp_smem = std::max(16, (off_c + 15) & ~15);
    p.warp_smem_fill = std::max(16, (off_f + 15) & ~15);
    p.tune.warps_per_block = 4;
    p.tune.chunk_roots = 64;
    // stars of 5+ edges on a hub grow subtrees of C(window, k-1) matches:
    // smaller root chunks spread the hubs' roots over more warps (the tuner
    // picked 32 for every such shape on the power-law workload)
    bool out_star = true, in_star = true;
    for (int i = 1; i < k; ++i) {
        out_star &= m->esrc[i] == m->esrc[0];
        in_star &= m->edst[i] == m->edst[0];
    }
    if (k >= 5 && (out_star || in_star)) p.tune.chunk_roots = 32;
    p.tune.split_depth = k >= 3 ? 2 : (k == 2 ? 1 : 0);
    p.tune.split_min = 512;
    if (m->n_anti > 0) p.tune.split_depth = 0;   // donated tasks carry no anti-edge times
    p.shape_hash = plan_shape_hash(m);
    *out = p;
    return TM_OK;
}

// ------------------------------------------------------------- scratch

static tm_status dev_alloc(void** p, size_t bytes) {
    if (dev_malloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed for search scratch");
        return TM_E_OOM;
    }
    return TM_OK;
}

tm_status scratch_reserve(Scratch* s, int device, int nq, uint64_t counters_len, uint64_t chunks, uint64_t task_cap) {
    s->device = device;
    if (nq > s->qcap) {
        if (s->head) cudaFree(s->head);
        if (s->stage) cudaFreeHost(s->stage);
        s->head = nullptr; s->stage = nullptr; s->qcap = 0;
        size_t bytes = s->head_bytes(nq);
        tm_status st = dev_alloc((void**)&s->head, bytes);
        if (st != TM_OK) return st;
        if (host_alloc_pinned((void**)&s->stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaHostAlloc failed");
            return TM_E_OOM;
        }
        memset(s->stage, 0, bytes);
        s->qcap = nq;
    }
    if (counters_len > s->counters_len) {
        if (s->counters) cudaFree(s->counters);
        if (s->counters_host) cudaFreeHost(s->counters_host);
        s->counters = nullptr; s->counters_host = nullptr; s->counters_len = 0;
        tm_status st = dev_alloc((void**)&s->counters, counters_len * 8);
        if (st != TM_OK) return st;
        if (host_alloc_pinned((void**)&s->counters_host, counters_len * 8) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaHostAlloc failed");
            return TM_E_OOM;
        }
        s->counters_len = counters_len;
    }
    if (task_cap > s->task_cap) {
        if (s->tasks) cudaFree(s->tasks);
        if (s->ready) cudaFree(s->ready);
        s->tasks = nullptr; s->ready = nullptr; s->task_cap = 0;
        tm_status st = dev_alloc((void**)&s->tasks, task_cap * sizeof(Task));
        if (st != TM_OK) return st;
        st = dev_alloc((void**)&s->ready, task_cap);
        if (st != TM_OK) return st;
        s->task_cap = task_cap;
    }
    if (chunks > s->chunk_cap) {
        if (s->chunk_cnt) cudaFree(s->chunk_cnt);
        if (s->scan_tmp) cudaFree(s->scan_tmp);
        s->chunk_cnt = nullptr; s->scan_tmp = nullptr; s->chunk_cap = 0;
        tm_status st = dev_alloc((void**)&s->chunk_cnt, chunk_buf_bytes(chunks));
        if (st != TM_OK) return st;
        s->scan_tmp_bytes = scan_temp_bytes(chunks + 1);
        st = dev_alloc(&s->scan_tmp, s->scan_tmp_bytes);
        if (st != TM_OK) return st;
        s->chunk_cap = chunks;
    }
    return TM_OK;
}

void scratch_free(Scratch* s) {
    if (s->head) cudaFree(s->head);
    if (s->stage) cudaFreeHost(s->stage);
    if (s->tasks) cudaFree(s->tasks);
    if (s->ready) cudaFree(s->ready);
    if (s->counters) cudaFree(s->counters);
    if (s->counters_host) cudaFreeHost(s->counters_host);
    if (s->chunk_cnt) cudaFree(s->chunk_cnt);
    if (s->scan_tmp) cudaFree(s->scan_tmp);
    *s = Scratch();
}

constexpr uint64_t DEFAULT_TASK_CAP = 1u << 18;   // 16 MiB of 64-byte tasks

uint64_t n_chunks(uint64_t roots, int chunk_roots) { return (roots + (uint64_t)chunk_roots - 1) / (uint64_t)chunk_roots; }

}  // namespace tmg

using namespace tmg;

struct tm_query {
    tm_graph* g = nullptr;
    int device = 0;          // the graph's device (kept here: freeing needs no graph access)
    tm_motif motif{};
    Plan plan{};
    bool explicit_tuning = false;
    Scratch scratch;
    // optional device timing of the search launches: [0,1] count pass, [2,3] fill pass
    bool profile = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool fill_timed = false;
    int inject = 0;      // test hook: fault to stage into the next count launch
};

namespace tmg {

// Apply the graph's cached tuning for this query's shape, unless set explicitly.
static void apply_cached_tuning(tm_graph* g, tm_query* q) {
    if (q->explicit_tuning) return;
    TuneKey key{q->plan.shape_hash, 0};
    int64_t d = q->plan.delta;
    while (d > 0) { key.dbucket++; d >>= 1; }
    std::lock_guard<std::mutex> lk(g->tune_mu);
    auto it = g->tuned.find(key);
    if (it != g->tuned.end()) q->plan.tune = it->second;
}

const tm_graph* query_graph(const tm_query* q) { return q->g; }
const tm_motif* query_motif(const tm_query* q) { return &q->motif; }

void query_plan(tm_query* q, Plan* out) {
    apply_cached_tuning(q->g, q);
    *out = q->plan;
}

// Stage and run one single-query count (optionally with per-root, per-chunk
// or work outputs).  Leaves results in scratch counters; does not sync.
static tm_status run_count(tm_graph* g, tm_query* q, uint64_t rb, uint64_t re, cudaStream_t st,
                           unsigned long long* per_root, bool chunk_counts, bool work, int grid_override = 0) {
    Scratch& s = q->scratch;
    const int cr = q->plan.tune.chunk_roots;
    uint64_t nch = n_chunks(re - rb, cr);
    tm_status r = scratch_reserve(&s, g->device, 1, 1 + (2 + 2 * TM_MAX_EDGES + 1), chunk_counts ? nch : 0,
                                  DEFAULT_TASK_CAP);
    if (r != TM_OK) return r;
    Ctrl* c = s.ctrl_stage();
    memset(c, 0, sizeof(Ctrl));
    c->total_chunks = nch;
    if (q->inject == 1) {
        // one reserved task slot that no warp will ever publish: a warp that
        // pops it waits out its bounded wait and reports TM_E_TIMEOUT
        c->q_reserve = 1;
        q->inject = 0;
    }
    QueryDev* qd = s.qdev_stage();
    memset(qd, 0, sizeof(QueryDev));
    qd->plan = q->plan;
    qd->root_begin = rb;
    qd->root_end = re;
    qd->n_chunks = nch;
    qd->chunk_base = 0;
    qd->total = s.counters;
    qd->per_root = per_root;
    qd->chunk_cnt = chunk_counts ? s.chunk_cnt : nullptr;
    qd->work = work ? s.counters + 1 : nullptr;
    TM_CUDA(cudaMemcpyAsync(s.head, s.stage, s.head_bytes(1), cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemsetAsync(s.counters, 0, s.counters_len * 8, st));
    TM_CUDA(cudaMemsetAsync(s.ready, 0, s.task_cap, st));
    if (per_root && re > rb) TM_CUDA(cudaMemsetAsync(per_root, 0, (re - rb) * 8, st));
    if (chunk_counts) TM_CUDA(cudaMemsetAsync(s.chunk_cnt, 0, (nch + 2) * 8, st));   // counts + list length
    if (q->profile) TM_CUDA(cudaEventRecord(q->ev[0], st));
    r = launch_search(g, MODE_COUNT, s.qdev(), 1, q->plan.warp_smem, q->plan.tune.warps_per_block,
                      plan_features(q->plan), &s, st,
                      grid_override, work);
    if (r != TM_OK) return r;
    if (q->profile) TM_CUDA(cudaEventRecord(q->ev[1], st));
    q->fill_timed = false;
    return TM_OK;
}

static tm_status read_back(Scratch& s, cudaStream_t st, uint64_t n_counters) {
    TM_CUDA(cudaMemcpyAsync(s.counters_host, s.counters, n_counters * 8, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaMemcpyAsync(s.stage, s.head, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    note_search_stats(*s.ctrl_stage());
    if (s.ctrl_stage()->err) {
        set_error("a bounded device wait timed out");
        return TM_E_TIMEOUT;
    }
    return TM_OK;
}

}  // namespace tmg

// ------------------------------------------------------------------- ABI

extern "C" tm_status tm_query_compile(const tm_graph* g, const tm_motif* m, tm_query** out) {
    if (!g || !m || !out) { set_error("null argument"); return TM_E_INVALID; }
    Plan p;
    tm_status s = build_plan(g, m, &p);
    if (s != TM_OK) return s;
    tm_query* q = new tm_query();
    q->g = const_cast<tm_graph*>(g);
    q->device = g->device;
    q->motif = *m;
    q->plan = p;
    *out = q;
    return TM_OK;
}

extern "C" tm_status tm_query_free(tm_query* q) {
    if (!q) return TM_OK;
    cudaSetDevice(q->device);
    scratch_free(&q->scratch);
    for (auto& e : q->ev)
        if (e) cudaEventDestroy(e);
    delete q;
    return TM_OK;
}

extern "C" tm_status tm_query_set_tuning(tm_query* q, const tm_tuning* t) {
    if (!q || !t) { set_error("null argument"); return TM_E_INVALID; }
    if (t->warps_per_block < 1 || t->warps_per_block > 16 || t->chunk_roots < 32 || (t->chunk_roots % 32) != 0 ||
        t->split_min < 0 || t->split_depth < -1 || t->split_depth > TM_MAX_EDGES - 1) {
        set_error("tuning out of range");
        return TM_E_INVALID;
    }
    q->plan.tune = *t;
    if (q->plan.n_anti > 0) q->plan.tune.split_depth = 0;   // donated tasks carry no anti-edge times
    q->explicit_tuning = true;
    return TM_OK;
}

extern "C" tm_status tm_query_profile(tm_query* q, int enable) {
    if (!q) { set_error("null query"); return TM_E_INVALID; }
    TM_ENTER(q->device);
    if (enable && !q->ev[0])
        for (auto& e : q->ev) TM_CUDA(cudaEventCreate(&e));
    q->profile = enable != 0;
    return TM_OK;
}

extern "C" tm_status tm_query_last_ms(const tm_query* q, double* search_ms, double* fill_ms) {
    if (!q || !q->profile) { set_error("profiling not enabled on this query"); return TM_E_INVALID; }
    float a = 0.f, b = 0.f;
    TM_CUDA(cudaEventElapsedTime(&a, q->ev[0], q->ev[1]));
    if (q->fill_timed) TM_CUDA(cudaEventElapsedTime(&b, q->ev[2], q->ev[3]));
    if (search_ms) *search_ms = a;
    if (fill_ms) *fill_ms = q->fill_timed ? b : 0.0;
    return TM_OK;
}

extern "C" tm_status tm_query_inject_fault(tm_query* q, int kind) {
    if (!q || kind < 0 || kind > 1) { set_error("bad fault kind"); return TM_E_INVALID; }
    q->inject = kind;
    return TM_OK;
}

extern "C" tm_status tm_query_get_tuning(const tm_query* q, tm_tuning* t) {
    if (!q || !t) { set_error("null argument"); return TM_E_INVALID; }
    *t = q->plan.tune;
    return TM_OK;
}

extern "C" tm_status tm_count_roots(tm_graph* g, tm_query* q, int64_t rb, int64_t re, void* stream, uint64_t* total,
                                    uint64_t* per_root_dev) {
    if (!g || !q || !total || q->g != g) { set_error("null or mismatched argument"); return TM_E_INVALID; }
    if (rb < 0 || re < rb || re > g->v.m) { set_error("root range out of [0, n_edges]"); return TM_E_INVALID; }
    TM_ENTER(g->device);
    apply_cached_tuning(g, q);
    cudaStream_t st = (cudaStream_t)stream;
    if (re == rb) {
        *total = 0;
        return TM_OK;
    }
    tm_status s = run_count(g, q, (uint64_t)rb, (uint64_t)re, st, (unsigned long long*)per_root_dev, false, false);
    if (s != TM_OK) return s;
    s = read_back(q->scratch, st, 1);
    if (s != TM_OK) return s;
    *total = q->scratch.counters_host[0];
    return TM_OK;
}

extern "C" tm_status tm_count(tm_graph* g, tm_query* q, void* stream, uint64_t* total, uint64_t* per_root_dev) {
    if (!g) { set_error("null graph"); return TM_E_INVALID; }
    return tm_count_roots(g, q, 0, g->v.m, stream, total, per_root_dev);
}

extern "C" tm_status tm_query_work(tm_graph* g, tm_query* q, void* stream, tm_work* out) {
    if (!g || !q || !out || q->g != g) { set_error("null or mismatched argument"); return TM_E_INVALID; }
    TM_ENTER(g->device);
    apply_cached_tuning(g, q);
    cudaStream_t st = (cudaStream_t)stream;
    memset(out, 0, sizeof *out);
    if (g->v.m == 0) return TM_OK;
    tm_status s = run_count(g, q, 0, (uint64_t)g->v.m, st, nullptr, false, true);
    if (s != TM_OK) return s;
    s = read_back(q->scratch, st, 1 + sizeof(tm_work) / 8);
    if (s != TM_OK) return s;
    memcpy(out, q->scratch.counters_host + 1, sizeof(tm_work));
    return TM_OK;
}

extern "C" tm_status tm_enumerate(tm_graph* g, tm_query* q, void* stream, int32_t* match_dev, uint64_t cap,
                                  uint64_t* n_written, uint64_t* total) {
    if (!g || !q || !n_written || !total || q->g != g || (cap > 0 && !match_dev)) {
        set_error("null or mismatched argument");
        return TM_E_INVALID;
    }
    TM_ENTER(g->device);
    apply_cached_tuning(g, q);
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t m = (uint64_t)g->v.m;
    if (m == 0) {
        *n_written = 0;
        *total = 0;
        return TM_OK;
    }
    // pass 1: per-chunk match counts
    tm_status s = run_count(g, q, 0, m, st, nullptr, true, false);
    if (s != TM_OK) return s;
    Scratch& sc = q->scratch;
    const uint64_t nch = n_chunks(m, q->plan.tune.chunk_roots);
    // pass 2: chunk offsets, and the chunks the fill pass must search
    s = exclusive_scan_u64(sc.chunk_cnt, sc.chunk_cnt, nch + 1, sc.scan_tmp, st);
    if (s != TM_OK) return s;
    if (cap > 0) {
        s = list_chunks(sc.chunk_cnt, nch, cap, g->num_sms, st);
        if (s != TM_OK) return s;
    }
    s = read_back(sc, st, 1);
    if (s != TM_OK) return s;
    const uint64_t tot = sc.counters_host[0];
    const uint64_t nw = std::min(tot, cap);
    if (nw > 0) {
        // pass 3: fill rows in lexicographic order from each chunk's offset
        Ctrl* c = sc.ctrl_stage();
        memset(c, 0, sizeof(Ctrl));
        c->total_chunks = nch;
        QueryDev* qd = sc.qdev_stage();
        qd->per_root = nullptr;
        qd->chunk_cnt = nullptr;
        qd->chunk_off = sc.chunk_cnt;
        qd->match_out = match_dev;
        qd->cap = cap;
        qd->work = nullptr;
        qd->total = sc.counters + 1;
        TM_CUDA(cudaMemcpyAsync(sc.head, sc.stage, sc.head_bytes(1), cudaMemcpyHostToDevice, st));
        if (q->profile) TM_CUDA(cudaEventRecord(q->ev[2], st));
        s = launch_search(g, MODE_FILL, sc.qdev(), 1, q->plan.warp_smem_fill, q->plan.tune.warps_per_block,
                         plan_features(q->plan), &sc, st);
        if (s != TM_OK) return s;
        if (q->profile) { TM_CUDA(cudaEventRecord(q->ev[3], st)); q->fill_timed = true; }
        TM_CUDA(cudaStreamSynchronize(st));
    }
    *total = tot;
    *n_written = nw;
    return tot > cap ? TM_E_TRUNCATED : TM_OK;
}

// ------------------------------------------------------------- batching

namespace tmg {

std::vector<LaunchGroup> occupancy_groups(const tm_graph* g, Mode mode, const Plan* const* plans, int nq,
                                          int* order) {
    std::vector<int> grid(nq), wpb(nq);
    for (int j = 0; j < nq; ++j) {
        const Plan& p = *plans[j];
        LaunchCfg c = search_launch_cfg(g, mode, mode == MODE_FILL ? p.warp_smem_fill : p.warp_smem,
                                        p.tune.warps_per_block);
        grid[j] = c.grid;
        wpb[j] = c.warps_per_block;
        order[j] = j;
    }
    // highest occupancy first; within a group the likely most expensive queries
    // (more motif edges, then longer delta) first: a persistent launch claims
    // root chunks in query order, so the cheap queries fill the tails of the
    // expensive ones instead of the other way round
    std::stable_sort(order, order + nq, [&](int a, int b) {
        if (grid[a] != grid[b]) return grid[a] > grid[b];
        if (wpb[a] != wpb[b]) return wpb[a] > wpb[b];
        if (plans[a]->k != plans[b]->k) return plans[a]->k > plans[b]->k;
        return plans[a]->delta > plans[b]->delta;
    });
    std::vector<LaunchGroup> out;
    for (int i = 0; i < nq; ++i) {
        const int j = order[i];
        const Plan& p = *plans[j];
        if (out.empty() || grid[order[out.back().first]] != grid[j] || wpb[order[out.back().first]] != wpb[j])
            out.push_back(LaunchGroup{i, 0, 16, wpb[j], 0u});
        LaunchGroup& lg = out.back();
        lg.count++;
        lg.warp_smem = std::max(lg.warp_smem, mode == MODE_FILL ? p.warp_smem_fill : p.warp_smem);
        lg.feat |= plan_features(p);
    }
    return out;
}

// One captured CUDA graph per batch geometry (its occupancy groups): stage ->
// one persistent launch per group, back to back -> read back.  Device and
// pinned staging: a control block per group, then the launch records in group
// order.
struct BatchExec {
    int nq = 0;
    Mode mode = MODE_COUNT;                    // the pass its launches run
    std::vector<LaunchGroup> groups;
    cudaEvent_t ev[2] = {nullptr, nullptr};    // optional timing of its launches
    char* head = nullptr;                      // device: Ctrl[groups] + QueryDev[nq]
    char* stage = nullptr;                     // pinned mirror
    unsigned long long* counters = nullptr;    // device totals, by the caller's query index
    unsigned long long* counters_host = nullptr;
    Task* tasks = nullptr;
    uint8_t* ready = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::mutex mu;                             // one call at a time uses these buffers
    size_t ctrl_bytes() const { return groups.size() * sizeof(Ctrl); }
    size_t head_bytes() const { return ctrl_bytes() + (size_t)nq * sizeof(QueryDev); }
    QueryDev* qdev_stage() const { return (QueryDev*)(stage + ctrl_bytes()); }
    QueryDev* qdev_dev() const { return (QueryDev*)(head + ctrl_bytes()); }
    bool same_shape(int n, const std::vector<LaunchGroup>& gs, Mode md = MODE_COUNT) const {
        if (n != nq || gs.size() != groups.size() || md != mode) return false;
        for (size_t i = 0; i < gs.size(); ++i)
            if (gs[i].count != groups[i].count || gs[i].warp_smem != groups[i].warp_smem ||
                gs[i].warps != groups[i].warps || gs[i].feat != groups[i].feat)
                return false;
        return true;
    }
    tm_status alloc() {
        if (head) return TM_OK;
        tm_status s = dev_alloc((void**)&head, head_bytes());
        if (s == TM_OK) s = dev_alloc((void**)&counters, (size_t)nq * 8);
        if (s == TM_OK) s = dev_alloc((void**)&tasks, DEFAULT_TASK_CAP * sizeof(Task));
        if (s == TM_OK) s = dev_alloc((void**)&ready, DEFAULT_TASK_CAP);
        if (s == TM_OK && (host_alloc_pinned((void**)&stage, head_bytes()) != cudaSuccess ||
                           host_alloc_pinned((void**)&counters_host, (size_t)nq * 8) != cudaSuccess)) {
            cudaGetLastError();
            set_error("cudaHostAlloc failed");
            s = TM_E_OOM;
        }
        if (s != TM_OK) release();
        return s;
    }
    void release() {
        for (auto& e : ev)
            if (e) { cudaEventDestroy(e); e = nullptr; }
        if (exec) cudaGraphExecDestroy(exec);
        if (head) cudaFree(head);
        if (counters) cudaFree(counters);
        if (tasks) cudaFree(tasks);
        if (ready) cudaFree(ready);
        if (stage) cudaFreeHost(stage);
        if (counters_host) cudaFreeHost(counters_host);
        exec = nullptr; head = stage = nullptr; counters = counters_host = nullptr; tasks = nullptr; ready = nullptr;
    }
    ~BatchExec() { release(); }
    Scratch view(size_t gi) const {   // what one group's launch reads: its Ctrl and the task queue
        Scratch v;
        v.head = head + gi * sizeof(Ctrl);
        v.tasks = tasks;
        v.ready = ready;
        v.task_cap = DEFAULT_TASK_CAP;
        return v;
    }
};

static std::mutex g_batch_mu;
static std::map<const tm_graph*, std::vector<std::unique_ptr<BatchExec>>> g_batches;

// The cached executable (buffers, groups, captured graph if any) for one batch shape.
static BatchExec* cached_exec(const tm_graph* g, int nq, const std::vector<LaunchGroup>& groups, Mode mode) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto& vec = g_batches[g];
    for (auto& p : vec)
        if (p->same_shape(nq, groups, mode)) return p.get();
    vec.emplace_back(new BatchExec());
    BatchExec* b = vec.back().get();
    b->nq = nq;
    b->groups = groups;
    b->mode = mode;
    return b;
}

static tm_status capture_batch(tm_graph* g, BatchExec* b) {
    cudaStream_t cs;
    TM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(e, "begin capture"); }
    cudaMemcpyAsync(b->head, b->stage, b->head_bytes(), cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(b->counters, 0, (size_t)b->nq * 8, cs);
    tm_status ls = TM_OK;
    for (size_t gi = 0; gi < b->groups.size() && ls == TM_OK; ++gi) {
        const LaunchGroup& lg = b->groups[gi];
        Scratch v = b->view(gi);
        cudaMemsetAsync(b->ready, 0, DEFAULT_TASK_CAP, cs);
        ls = launch_search(g, MODE_COUNT, b->qdev_dev() + lg.first, lg.count, lg.warp_smem, lg.warps, lg.feat, &v,
                           cs);
    }
    cudaMemcpyAsync(b->counters_host, b->counters, (size_t)b->nq * 8, cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(b->stage, b->head, b->ctrl_bytes(), cudaMemcpyDeviceToHost, cs);
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (ls != TM_OK) { if (graph) cudaGraphDestroy(graph); return ls; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    return TM_OK;
}

}  // namespace tmg

extern "C" tm_status tm_count_batch(tm_graph* g, tm_query* const* qs, int nq, void* stream, uint64_t* totals) {
    if (!g || !qs || nq < 1 || nq > 4096 || !totals) { set_error("bad batch arguments"); return TM_E_INVALID; }
    for (int j = 0; j < nq; ++j)
        if (!qs[j] || qs[j]->g != g) { set_error("null or mismatched query in batch"); return TM_E_INVALID; }
    TM_ENTER(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (g->v.m == 0) {
        for (int j = 0; j < nq; ++j) totals[j] = 0;
        return TM_OK;
    }
    std::vector<const Plan*> plans(nq);
    for (int j = 0; j < nq; ++j) {
        apply_cached_tuning(g, qs[j]);
        plans[j] = &qs[j]->plan;
    }
    std::vector<int> order(nq);
    std::vector<LaunchGroup> groups = occupancy_groups(g, MODE_COUNT, plans.data(), nq, order.data());
    BatchExec* b = cached_exec(g, nq, groups, MODE_COUNT);
    std::lock_guard<std::mutex> use(b->mu);
    tm_status s = b->alloc();
    if (s != TM_OK) return s;
    memset(b->stage, 0, b->ctrl_bytes());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        uint64_t base = 0;
        for (int i = groups[gi].first; i < groups[gi].first + groups[gi].count; ++i) {
            const int j = order[i];
            QueryDev* qd = b->qdev_stage() + i;
            memset(qd, 0, sizeof(QueryDev));
            qd->plan = qs[j]->plan;
            qd->root_begin = 0;
            qd->root_end = (uint64_t)g->v.m;
            qd->n_chunks = n_chunks((uint64_t)g->v.m, qs[j]->plan.tune.chunk_roots);
            qd->chunk_base = base;
            base += qd->n_chunks;
            qd->total = b->counters + j;
        }
        ((Ctrl*)b->stage)[gi].total_chunks = base;
    }
    if (!b->exec) {
        s = capture_batch(g, b);
        if (s != TM_OK) return s;
    }
    TM_CUDA(cudaGraphLaunch(b->exec, st));
    note_launches(1);
    TM_CUDA(cudaStreamSynchronize(st));
    Ctrl sum;
    memset(&sum, 0, sizeof sum);
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const Ctrl& c = ((const Ctrl*)b->stage)[gi];
        sum.donated += c.donated;
        sum.q_reserve += c.q_reserve;
        sum.err |= c.err;
    }
    note_search_stats(sum);
    if (sum.err) { set_error("a bounded device wait timed out"); return TM_E_TIMEOUT; }
    for (int j = 0; j < nq; ++j) totals[j] = b->counters_host[j];
    return TM_OK;
}

extern "C" tm_status tm_enumerate_batch(tm_graph* g, tm_query* const* qs, int nq, void* stream,
                                        int32_t* const* match_devs, const uint64_t* caps, uint64_t* n_written,
                                        uint64_t* totals, double* kernel_ms) {
    if (!g || !qs || nq < 1 || nq > 4096 || !match_devs || !caps || !n_written || !totals) {
        set_error("bad batch arguments");
        return TM_E_INVALID;
    }
    std::vector<const tm_query*> seen(qs, qs + nq);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
        set_error("a query appears twice in the batch (its chunk counts would be shared)");
        return TM_E_INVALID;
    }
    for (int j = 0; j < nq; ++j)
        if (!qs[j] || qs[j]->g != g || (caps[j] > 0 && !match_devs[j])) {
            set_error("null or mismatched query or match buffer in batch");
            return TM_E_INVALID;
        }
    TM_ENTER(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t m = (uint64_t)g->v.m;
    if (kernel_ms) kernel_ms[0] = kernel_ms[1] = 0.0;
    if (m == 0) {
        for (int j = 0; j < nq; ++j) totals[j] = n_written[j] = 0;
        return TM_OK;
    }
    std::vector<const Plan*> plans(nq);
    std::vector<uint64_t> nch(nq);
    for (int j = 0; j < nq; ++j) {
        apply_cached_tuning(g, qs[j]);
        plans[j] = &qs[j]->plan;
        nch[j] = n_chunks(m, qs[j]->plan.tune.chunk_roots);
        // each query's own scratch holds its chunk counts, then their offsets
        tm_status r = scratch_reserve(&qs[j]->scratch, g->device, 1, 1, nch[j], 0);
        if (r != TM_OK) return r;
        TM_CUDA(cudaMemsetAsync(qs[j]->scratch.chunk_cnt, 0, (nch[j] + 2) * 8, st));   // counts + list length
    }
    // pass 1: per-chunk counts of every query, one persistent launch per occupancy group
    std::vector<int> order(nq);
    std::vector<LaunchGroup> cg = occupancy_groups(g, MODE_COUNT, plans.data(), nq, order.data());
    BatchExec* bc = cached_exec(g, nq, cg, MODE_COUNT);
    std::lock_guard<std::mutex> lock_c(bc->mu);
    tm_status s = bc->alloc();
    if (s != TM_OK) return s;
    memset(bc->stage, 0, bc->ctrl_bytes());
    for (size_t gi = 0; gi < cg.size(); ++gi) {
        uint64_t base = 0;
        for (int i = cg[gi].first; i < cg[gi].first + cg[gi].count; ++i) {
            const int j = order[i];
            QueryDev* qd = bc->qdev_stage() + i;
            memset(qd, 0, sizeof(QueryDev));
            qd->plan = qs[j]->plan;
            qd->root_end = m;
            qd->n_chunks = nch[j];
            qd->chunk_base = base;
            base += nch[j];
            qd->total = bc->counters + j;
            qd->chunk_cnt = qs[j]->scratch.chunk_cnt;
        }
        ((Ctrl*)bc->stage)[gi].total_chunks = base;
    }
    if (kernel_ms && !bc->ev[0])
        for (auto& e : bc->ev) TM_CUDA(cudaEventCreate(&e));
    TM_CUDA(cudaMemcpyAsync(bc->head, bc->stage, bc->head_bytes(), cudaMemcpyHostToDevice, st));
    TM_CUDA(cudaMemsetAsync(bc->counters, 0, (size_t)nq * 8, st));
    if (kernel_ms) TM_CUDA(cudaEventRecord(bc->ev[0], st));
    for (size_t gi = 0; gi < cg.size(); ++gi) {
        Scratch v = bc->view(gi);
        TM_CUDA(cudaMemsetAsync(bc->ready, 0, DEFAULT_TASK_CAP, st));
        s = launch_search(g, MODE_COUNT, bc->qdev_dev() + cg[gi].first, cg[gi].count, cg[gi].warp_smem,
                          cg[gi].warps, cg[gi].feat, &v, st);
        if (s != TM_OK) return s;
    }
    if (kernel_ms) TM_CUDA(cudaEventRecord(bc->ev[1], st));
    // pass 2: chunk offsets, and the chunks the fill pass must search
    for (int j = 0; j < nq; ++j) {
        s = exclusive_scan_u64(qs[j]->scratch.chunk_cnt, qs[j]->scratch.chunk_cnt, nch[j] + 1,
                               qs[j]->scratch.scan_tmp, st);
        if (s != TM_OK) return s;
        if (caps[j] > 0) {
            s = list_chunks(qs[j]->scratch.chunk_cnt, nch[j], caps[j], g->num_sms, st);
            if (s != TM_OK) return s;
        }
    }
    // pass 3: rows of the queries with room for some, written from each chunk's
    // offset on the device (chunks past the cap or without matches are skipped)
    std::vector<int> fq;
    for (int j = 0; j < nq; ++j)
        if (caps[j] > 0) fq.push_back(j);
    BatchExec* bf = nullptr;
    std::unique_lock<std::mutex> lock_f;
    if (!fq.empty()) {
        const int nf = (int)fq.size();
        std::vector<const Plan*> fplans(nf);
        for (int i = 0; i < nf; ++i) fplans[i] = plans[fq[i]];
        std::vector<int> forder(nf);
        std::vector<LaunchGroup> fg = occupancy_groups(g, MODE_FILL, fplans.data(), nf, forder.data());
        bf = cached_exec(g, nf, fg, MODE_FILL);
        lock_f = std::unique_lock<std::mutex>(bf->mu);
        s = bf->alloc();
        if (s != TM_OK) return s;
        memset(bf->stage, 0, bf->ctrl_bytes());
        for (size_t gi = 0; gi < fg.size(); ++gi) {
            uint64_t base = 0;
            for (int i = fg[gi].first; i < fg[gi].first + fg[gi].count; ++i) {
                const int j = fq[forder[i]];
                QueryDev* qd = bf->qdev_stage() + i;
                memset(qd, 0, sizeof(QueryDev));
                qd->plan = qs[j]->plan;
                qd->root_end = m;
                qd->n_chunks = nch[j];
                qd->chunk_base = base;
                base += nch[j];
                qd->total = bf->counters + i;
                qd->chunk_off = qs[j]->scratch.chunk_cnt;
                qd->match_out = match_devs[j];
                qd->cap = caps[j];
            }
            ((Ctrl*)bf->stage)[gi].total_chunks = base;
        }
        if (kernel_ms && !bf->ev[0])
            for (auto& e : bf->ev) TM_CUDA(cudaEventCreate(&e));
        TM_CUDA(cudaMemcpyAsync(bf->head, bf->stage, bf->head_bytes(), cudaMemcpyHostToDevice, st));
        if (kernel_ms) TM_CUDA(cudaEventRecord(bf->ev[0], st));
        for (size_t gi = 0; gi < fg.size(); ++gi) {
            Scratch v = bf->view(gi);
            s = launch_search(g, MODE_FILL, bf->qdev_dev() + fg[gi].first, fg[gi].count, fg[gi].warp_smem,
                              fg[gi].warps, fg[gi].feat, &v, st);
            if (s != TM_OK) return s;
        }
        if (kernel_ms) TM_CUDA(cudaEventRecord(bf->ev[1], st));
        TM_CUDA(cudaMemcpyAsync(bf->stage, bf->head, bf->ctrl_bytes(), cudaMemcpyDeviceToHost, st));
    }
    TM_CUDA(cudaMemcpyAsync(bc->counters_host, bc->counters, (size_t)nq * 8, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaMemcpyAsync(bc->stage, bc->head, bc->ctrl_bytes(), cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    Ctrl sum;
    memset(&sum, 0, sizeof sum);
    for (size_t gi = 0; gi < cg.size(); ++gi) {
        const Ctrl& c = ((const Ctrl*)bc->stage)[gi];
        sum.donated += c.donated;
        sum.q_reserve += c.q_reserve;
        sum.err |= c.err;
    }
    for (size_t gi = 0; bf && gi < bf->groups.size(); ++gi) sum.err |= ((const Ctrl*)bf->stage)[gi].err;
    note_search_stats(sum);
    if (sum.err) { set_error("a bounded device wait timed out"); return TM_E_TIMEOUT; }
    if (kernel_ms) {
        float a = 0.f, b = 0.f;
        TM_CUDA(cudaEventElapsedTime(&a, bc->ev[0], bc->ev[1]));
        if (bf) TM_CUDA(cudaEventElapsedTime(&b, bf->ev[0], bf->ev[1]));
        kernel_ms[0] = a;
        kernel_ms[1] = b;
    }
    bool truncated = false;
    for (int j = 0; j < nq; ++j) {
        totals[j] = bc->counters_host[j];
        n_written[j] = std::min<uint64_t>(totals[j], caps[j]);
        truncated |= totals[j] > caps[j];
    }
    return truncated ? TM_E_TRUNCATED : TM_OK;
}

// Release batch executables of a graph (called from tm_graph_free).
void tmg::drop_batches(const tm_graph* g) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batches.erase(g);
}

// ------------------------------------------------------------- autotune

extern "C" tm_status tm_autotune(tm_graph* g, tm_query* q, void* stream, tm_tuning* tuned) {
    if (!g || !q || q->g != g) { set_error("null or mismatched argument"); return TM_E_INVALID; }
    TM_ENTER(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t m = (uint64_t)g->v.m;
    tm_tuning best = q->plan.tune;
    if (m > 0) {
        cudaEvent_t e0, e1;
        TM_CUDA(cudaEventCreate(&e0));
        TM_CUDA(cudaEventCreate(&e1));
        auto time_cfg = [&](const tm_tuning& t, float* ms) -> tm_status {
            q->plan.tune = t;
            float best_ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                tm_status s = run_count(g, q, 0, m, st, nullptr, false, false);
                if (s != TM_OK) return s;
                cudaEventRecord(e1, st);
                TM_CUDA(cudaEventSynchronize(e1));
                float x = 0;
                cudaEventElapsedTime(&x, e0, e1);
                if (rep > 0) best_ms = std::min(best_ms, x);
                if (x > 2000.f) { best_ms = std::min(best_ms, x); break; }
            }
            *ms = best_ms;
            return TM_OK;
        };
        float best_ms;
        tm_status s = time_cfg(best, &best_ms);
        // coordinate descent over the four knobs
        const int warps_c[] = {2, 4, 8};
        const int chunk_c[] = {32, 64, 256};
        const int min_c[] = {128, 512, 4096};
        for (int knob = 0; knob < 4 && s == TM_OK; ++knob) {
            std::vector<tm_tuning> cands;
            for (int i = 0; i < 3; ++i) {
                tm_tuning t = best;
                if (knob == 0) t.warps_per_block = warps_c[i];
                if (knob == 1) t.chunk_roots = chunk_c[i];
                if (knob == 2) { t.split_depth = i; if (t.split_depth > q->plan.k - 1) continue; }
                if (knob == 3) t.split_min = min_c[i];
                cands.push_back(t);
            }
            for (auto& t : cands) {
                float ms;
                s = time_cfg(t, &ms);
                if (s != TM_OK) break;
                if (ms < best_ms * 0.97f) { best_ms = ms; best = t; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        TM_CUDA(cudaStreamSynchronize(st));
        if (s != TM_OK) return s;
        q->plan.tune = best;
        TuneKey key{q->plan.shape_hash, 0};
        int64_t d = q->plan.delta;
        while (d > 0) { key.dbucket++; d >>= 1; }
        std::lock_guard<std::mutex> lk(g->tune_mu);
        g->tuned[key] = best;
    }
    q->explicit_tuning = false;
    if (tuned) *tuned = best;
    return TM_OK;
}

// ----------------------------------------------------------------- status

extern "C" const char* tm_status_str(tm_status s) {
    switch (s) {
        case TM_OK: return "ok";
        case TM_E_INVALID: return "invalid argument";
        case TM_E_OOM: return "out of device memory";
        case TM_E_TRUNCATED: return "truncated: enumeration cap reached";
        case TM_E_TIMEOUT: return "bounded device wait timed out";
        case TM_E_CUDA: return "CUDA error";
        case TM_E_BUSY: return "busy: request not finished";
        case TM_E_ADMISSION: return "request exceeds the serving memory budget";
    }
    return "unknown status";
}

extern "C" const char* tm_last_error(void) { return g_last_error.c_str(); }

extern "C" tm_status tm_inject_alloc_failure(int64_t after) {
    g_alloc_fault.store(after < 0 ? -1 : after);
    return TM_OK;
}

extern "C" tm_status tm_last_search_stats(uint64_t* donated, uint64_t* reserved) {
    if (donated) *donated = g_last_donated;
    if (reserved) *reserved = g_last_reserved;
    return TM_OK;
}

extern "C" uint64_t tm_kernel_launches(void) { return g_launches.load(); }
