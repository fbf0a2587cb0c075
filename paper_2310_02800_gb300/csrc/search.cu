// Persistent warp-cooperative temporal motif search (sm_103a).
//
// The search is the chronological depth-first search of the paper's
// Algorithm 1 (Section 2.2), rooted at every edge, with the per-level plan of
// Section 5.1.2 deciding where candidates come from and which mapped nodes a
// new node must differ from.  The GPU organisation is our own:
//
//  * A warp owns a stack of FRAMES, one per motif edge i >= 1.  Frame i holds
//    up to 64 partial matches of i edges ("parents"), each with its candidate
//    window for edge i: the entries of one time-ordered adjacency list with
//    t in (t_prev, min(t_root + delta, t_prev + gap_{i-1})], located by a
//    binary search for the lower end and a galloping search for the upper end
//    (the cached candidate range of Section 5.1.1 is the window itself).  When
//    the list belongs to an endpoint of the edge just bound, the lower end is
//    the graph's successor word for that edge instead, read together with the
//    candidate; its time gap proves most windows empty without further loads.
//  * The windows of a frame are flattened: lane j of a 32-wide step takes the
//    j-th remaining candidate across all parents, so lanes stay busy even when
//    every individual window is short.  Survivors of a step (structure, label
//    and injectivity checks) are compacted with __ballot_sync into the child
//    frame, which is drained once it holds cap - 32 parents (16 in count
//    frames of 48, 32 in fill frames of 64) or its parent frame is exhausted.  Processing frames in order keeps the emitted matches in
//    lexicographic order of edge ids (used by enumeration).
//  * The last motif edge is never expanded: survivors are counted with
//    __popc(ballot) and added to per-warp accumulators; per-root / per-chunk
//    counts use __match_any_sync groups and one atomic per group.
//  * Load balance (sub-tree-level parallelism, Section 5.2): root edges are
//    claimed in chunks from an atomic cursor; when warps sit idle, a warp at a
//    shallow level donates the upper half of its remaining candidate range to
//    a device task queue (count mode only), and idle warps pop those tasks.
//    Every device-side wait is bounded by a global-timer deadline.
//  * Look-ahead on chords (our addition): when an edge binds the last node of
//    a later motif edge whose node pair no earlier motif edge joins, some
//    graph edge must join their images later in the root's window; the
//    pair-ordered out-list answers that with two searches, and partial
//    matches without one are dropped before their subtrees are searched.
//  * Enumeration is two launches of this kernel: a count launch leaves
//    per-chunk match counts, a device scan turns them into row offsets,
//    list_chunks_kernel lists the chunks holding a match below the cap, and a fill
//    launch searches only the listed chunks again, each writing its rows in
//    lexicographic order from its offset.
//  * The kernel is instantiated per mode (count, enumeration fill), with or
//    without work counters, and per feature set (anti-edges, look-ahead), so
//    a plain motif runs code holding neither.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "tm_internal.cuh"

namespace tmg {

namespace {

constexpr unsigned FULL = 0xffffffffu;
// read the next level's successor words together with each candidate
constexpr bool PREFETCH = true;
constexpr uint32_t INLIST = 0x80000000u;    // window in an in-list
constexpr uint32_t PAIRLIST = 0x40000000u;  // window in the (neighbour, time)-ordered out-list
constexpr uint32_t POSMASK = 0x3FFFFFFFu;
constexpr uint32_t SPAN_FAR = 0xFFFFFFFFu;   // frame window end: recompute from the root
constexpr uint32_t PAIR_MIN_DEG = 1024;     // closing lookups on shorter lists scan the time window
constexpr uint32_t PAIR_MIN_WINDOW = 768;   // ... and so do windows shorter than this
constexpr uint64_t WAIT_NS = 20ull * 1000 * 1000 * 1000;      // idle-wait deadline
constexpr uint64_t READY_NS = 2ull * 1000 * 1000 * 1000;      // publish-wait deadline

__device__ __forceinline__ int64_t sat_add(int64_t a, int64_t b) {
    return (b > 0 && a > INT64_MAX - b) ? INT64_MAX : a + b;
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// first index in [lo, hi) with t[idx] > x
__device__ __forceinline__ uint32_t upper_bound_t(const int64_t* __restrict__ t, uint32_t lo, uint32_t hi, int64_t x) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(t + mid) <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first index in [beg, hi) with t[idx] > lim, searching outward from beg
__device__ __forceinline__ uint32_t gallop_end(const int64_t* __restrict__ t, uint32_t beg, uint32_t hi, int64_t lim) {
    uint32_t a = beg, b = hi, step = 1;
    while (true) {
        uint32_t probe = a + step - 1;
        if (probe >= hi) { b = hi; break; }
        if (__ldg(t + probe) > lim) { b = probe; break; }
        a = probe + 1;
        step <<= 1;
    }
    return upper_bound_t(t, a, b, lim);
}

// End of a time window that starts at beg: the first index in [beg, hi) with
// t[idx] > lim (galloping from beg: O(log of the window length)).
__device__ __forceinline__ uint32_t window_end(const int64_t* __restrict__ t, uint32_t beg, uint32_t hi, int64_t lim) {
    return gallop_end(t, beg, hi, lim);
}

__device__ __forceinline__ uint32_t ceil_log2p1(uint32_t x) { return 32 - __clz(x); }  // ceil(log2(x+1))

// first index in [lo, hi) with a[idx] >= x
__device__ __forceinline__ uint32_t lower_bound_i32(const int32_t* __restrict__ a, uint32_t lo, uint32_t hi, int32_t x) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Edges u -> v with time in [t0, t1], counted from u's pair-ordered out-list.
__device__ __forceinline__ uint32_t pair_count(const GraphView& g, int32_t u, int32_t v, int64_t t0, int64_t t1) {
    uint32_t u0 = __ldg(g.off[0] + u), u1 = __ldg(g.off[0] + u + 1);
    uint32_t ps = lower_bound_i32(g.pnbr, u0, u1, v);
    uint32_t pe = lower_bound_i32(g.pnbr, ps, u1, v + 1);
    if (ps == pe) return 0u;
    uint32_t a = upper_bound_t(g.pt, ps, pe, t0 - 1);   // first time >= t0 (t0 >= 0)
    uint32_t b = upper_bound_t(g.pt, a, pe, t1);
    return b - a;
}

// Whether some edge u -> v has a time in (t0, t1]: u's pair-ordered out-list
// holds the u -> v edges as one time-ordered run (binary search on the
// neighbour, then a galloping search past t0 inside the run).
__device__ __forceinline__ bool pair_after(const GraphView& g, int32_t u, int32_t v, int64_t t0, int64_t t1) {
    if (t1 <= t0) return false;
    const uint32_t u1 = __ldg(g.off[0] + u + 1);
    uint32_t a = lower_bound_i32(g.pnbr, __ldg(g.off[0] + u), u1, v), hi = u1, step = 1;
    while (true) {
        const uint32_t probe = a + step - 1;
        if (probe >= u1) break;                       // hi stays at the list end
        if (__ldg(g.pnbr + probe) != v || __ldg(g.pt + probe) > t0) { hi = probe; break; }
        a = probe + 1;
        step <<= 1;
    }
    while (a < hi) {
        const uint32_t mid = a + ((hi - a) >> 1);
        if (__ldg(g.pnbr + mid) == v && __ldg(g.pt + mid) <= t0) a = mid + 1; else hi = mid;
    }
    return a < u1 && __ldg(g.pnbr + a) == v && __ldg(g.pt + a) <= t1;
}

// ------------------------------------------------------------ frame access

template <int CAP>
struct FrameT {
    using L = FrameLayout<CAP>;
    char* p;
    __device__ int64_t& tprev(int s) const { return ((int64_t*)(p + L::TPREV))[s]; }
    // window end t_root + delta, as its distance from tprev (SPAN_FAR: too far to hold)
    __device__ uint32_t& tspan(int s) const { return ((uint32_t*)(p + L::TEND))[s]; }
    __device__ uint32_t& beg(int s) const { return ((uint32_t*)(p + L::BEG))[s]; }
    __device__ uint32_t& len(int s) const { return ((uint32_t*)(p + L::LEN))[s]; }
    __device__ uint32_t& root(int s) const { return ((uint32_t*)(p + L::ROOT))[s]; }
    __device__ int32_t& node(int j, int s) const { return ((int32_t*)(p + L::NODE))[j * CAP + s]; }
    // eids follow the nb node rows
    __device__ int32_t& eid(int nb, int j, int s) const { return ((int32_t*)(p + L::NODE))[(nb + j) * CAP + s]; }
    // anti-edge attached-edge times, at byte offset `row_off` of the frame
    __device__ int64_t& anti_t(int row_off, int a, int s) const { return ((int64_t*)(p + row_off))[a * CAP + s]; }
};

// ------------------------------------------------------------ per-warp state

// work counters, laid out like tm_work
constexpr int W_ROOTS = 0, W_NODES = 1, W_ENTRIES = 1 + TM_MAX_EDGES, W_PROBE = 1 + 2 * TM_MAX_EDGES,
              W_MATCH = 2 + 2 * TM_MAX_EDGES, W_LEN = 3 + 2 * TM_MAX_EDGES;

struct Acc {             // per-warp accumulators for the current query
    unsigned long long total;      // warp-uniform
    unsigned long long w[W_LEN];   // stats launches; lane-0 values except W_PROBE (per lane)
};

template <int MODE, bool STATS, int FEAT>
struct Search {
    static constexpr bool ANTI = (FEAT & FEAT_ANTI) != 0;   // anti-edge checks compiled in
    static constexpr bool LOOK = (FEAT & FEAT_LOOK) != 0;   // look-ahead checks compiled in
    static constexpr int CAP = MODE == MODE_FILL ? FCAP_FILL : FCAP_COUNT;   // parents per frame
    static constexpr uint32_t DESCEND = CAP - 32;   // a child frame this full is drained next
    using Frame = FrameT<CAP>;
    const GraphView& g;
    const QueryDev* __restrict__ qs;
    Ctrl* ctrl;
    Task* tasks;
    uint8_t* ready;
    uint64_t task_cap;
    char* wbase;              // this warp's shared block
    int lane;
    // current query
    int qi;
    const QueryDev* q;
    int k;
    // level cursors: lane j holds the values for level j
    uint32_t myP, myOff, myT;
    Acc acc;
    // enumerate fill
    unsigned long long out_base, out_local;
    unsigned polls;           // donation checks (warp-uniform)

    __device__ Search(const GraphView& g_, const QueryDev* qs_, Ctrl* c, Task* t, uint8_t* r, uint64_t cap, char* wb)
        : g(g_), qs(qs_), ctrl(c), tasks(t), ready(r), task_cap(cap), wbase(wb) {
        lane = threadIdx.x & 31;
        qi = -1; q = nullptr; k = 0;
        myP = myOff = myT = 0;
        acc.total = 0;
        if (STATS) for (int i = 0; i < W_LEN; ++i) acc.w[i] = 0;
        out_base = out_local = 0;
        polls = 0;
    }

    __device__ uint32_t P(int l) const { return __shfl_sync(FULL, myP, l); }
    __device__ uint32_t Off(int l) const { return __shfl_sync(FULL, myOff, l); }
    __device__ uint32_t T(int l) const { return __shfl_sync(FULL, myT, l); }
    __device__ void setP(int l, uint32_t v) { if (lane == l) myP = v; }
    __device__ void setOff(int l, uint32_t v) { if (lane == l) myOff = v; }
    __device__ void setT(int l, uint32_t v) { if (lane == l) myT = v; }

    // The window end t_root + delta of entry s of frame f (4 bytes per entry
    // instead of 8: rebuilt from the root edge's time when too far from tprev).
    __device__ int64_t tend_of(Frame f, int s) const {
        const uint32_t sp = f.tspan(s);
        return sp != SPAN_FAR ? f.tprev(s) + (int64_t)sp : sat_add(__ldg(g.t + f.root(s)), q->plan.delta);
    }
    __device__ static void set_tend(Frame f, int s, int64_t tprev, int64_t tend) {
        const uint64_t d = (uint64_t)(tend - tprev);   // tprev <= tend
        f.tspan(s) = d < (uint64_t)SPAN_FAR ? (uint32_t)d : SPAN_FAR;
    }

    __device__ Frame frame(int i) const {
        return Frame{wbase + (MODE == MODE_FILL ? q->plan.lv[i].frame_off_fill : q->plan.lv[i].frame_off)};
    }

    __device__ int anti_off(int i) const {
        return MODE == MODE_FILL ? q->plan.lv[i].anti_row_off_fill : q->plan.lv[i].anti_row_off;
    }

    // Anti-edges in `mask` (Section 2.1): true when none of them has an edge in
    // its window.  Slots of the candidate's partial match are the parent's
    // slots [0, nb) plus n0, n1; times: edge `lvl` is the candidate (ct), edge
    // lvl-1 is the parent's tprev, older attached edges come from anti rows.
    __device__ bool anti_clear(unsigned mask, int lvl, Frame pf, int ps, int nb, int32_t n0, int32_t n1, int64_t ct,
                               int64_t tprev, int prow) const {
        const Plan& pl = q->plan;
        auto slot = [&](int s) -> int32_t { return s < nb ? pf.node(s, ps) : (s == nb ? n0 : n1); };
        for (int a = 0; a < pl.n_anti; ++a) {
            if (!(mask & (1u << a))) continue;
            const AntiPlan& ap = pl.anti[a];
            int64_t ti = ap.edge == lvl ? ct : (ap.edge == lvl - 1 ? tprev : pf.anti_t(prow, a, ps));
            uint32_t c = pair_count(g, slot(ap.xs), slot(ap.ys), ti, sat_add(ti, ap.delta));
            if (c > (uint32_t)ap.same_pair) return false;
        }
        return true;
    }

    // Look-ahead of level `lp` for a partial match whose slots are the
    // parent's [0, nb) plus n0, n1, just extended by an edge at time ct:
    // false when a later motif edge between bound nodes has no graph edge left
    // in (ct, tend].
    __device__ bool look_ok(const LevelPlan& lp, Frame pf, int ps, int nb, int32_t n0, int32_t n1, int64_t ct,
                            int64_t tend) const {
        auto slot = [&](int s) -> int32_t { return s < nb ? pf.node(s, ps) : (s == nb ? n0 : n1); };
        for (int l = 0; l < lp.n_look; ++l)
            if (!pair_after(g, slot(lp.look_u[l]), slot(lp.look_v[l]), ct, tend)) return false;
        return true;
    }

    __device__ void flush() {
        if (q == nullptr) return;
        if (lane == 0 && acc.total) atomicAdd(q->total, acc.total);
        if (STATS) {
            for (int i = 0; i < W_LEN; ++i) {
                unsigned long long v = acc.w[i];
                for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(FULL, v, d);
                if (lane == 0 && v && q->work) atomicAdd(q->work + i, v);
                acc.w[i] = 0;
            }
        }
        acc.total = 0;
    }

    __device__ void use_query(int j) {
        if (j == qi) return;
        flush();
        qi = j;
        q = qs + j;
        k = q->plan.k;
    }

    // Window for motif edge `lv_i` of a (child) partial match whose slots are
    // parent slots [0, nb) of frame `pf` at index `ps`, plus new nodes n0, n1
    // at slots nb, nb+1; prev_e is the edge just bound (time tprev).  The
    // window's lower end comes from the successor index when the list belongs
    // to an endpoint of prev_e, else from a binary search; the upper end from
    // a galloping search.  Returns len; beg gets bit 31 for in-lists.
    // The edge just bound sits at position cpos of list cdir (0 out-list, 1 in-list,
    // 2 the edge list itself, 3 a pair-ordered list); prev_e is its edge id when
    // already loaded, else -1.  Successor-index lookups read the position-indexed
    // copy when it covers the continuation, else the edge-indexed one.
    __device__ uint2 successor(int nx, int cdir, uint32_t cpos, int32_t prev_e) const {
        if (cdir == 0 && nx == NX_OUT_SRC) return __ldg(g.pnx[0] + cpos);
        if (cdir == 0 && nx == NX_OUT_DST) return __ldg(g.pnx[1] + cpos);
        if (cdir == 1 && nx == NX_IN_DST) return __ldg(g.pnx[2] + cpos);
        if (cdir == 1 && nx == NX_IN_SRC) return __ldg(g.pnx[3] + cpos);
        return __ldg(g.nxt[nx] + edge_at(cdir, cpos, prev_e));
    }
    // True when successor() is one load (no edge id needed first).
    __device__ static bool successor_direct(int nx, int cdir) {
        if (cdir == 2) return true;
        if (cdir == 0) return nx == NX_OUT_SRC || nx == NX_OUT_DST;
        if (cdir == 1) return nx == NX_IN_DST || nx == NX_IN_SRC;
        return false;
    }
    // Successor words of the lists level `ln` draws its window from, after a
    // candidate edge at position cpos of list cdir, read ahead together with
    // the candidate: only those that take one load.  y == 0 means "not read".
    __device__ void next_words(const LevelPlan& ln, int cdir, uint32_t cpos, uint2& wa, uint2& wb) const {
        wa = make_uint2(0u, 0u);
        wb = make_uint2(0u, 0u);
        if (ln.nx_a >= 0 && successor_direct(ln.nx_a, cdir)) wa = successor(ln.nx_a, cdir, cpos, -1);
        if (ln.kind == CLOSE && ln.nx_b >= 0 && successor_direct(ln.nx_b, cdir)) wb = successor(ln.nx_b, cdir, cpos, -1);
    }
    // True when a list whose successor word is w has no entry in (tprev, lim].
    __device__ static bool word_shows_empty(uint2 w, uint64_t span) {
        return w.y == SUCC_END || (uint64_t)w.y > span;
    }
    __device__ int32_t edge_at(int cdir, uint32_t cpos, int32_t prev_e) const {
        if (prev_e >= 0) return prev_e;
        if (cdir == 0 || cdir == 1) return __ldg(g.aeid[cdir] + cpos);
        if (cdir == 3) return __ldg(g.peid + cpos);
        return (int32_t)cpos;
    }

    __device__ uint32_t locate(int lv_i, Frame pf, int ps, int nb, int32_t n0, int32_t n1, int32_t prev_e,
                               int cdir, uint32_t cpos, int64_t tprev, int64_t tend, uint32_t& beg_out,
                               uint2 wa, uint2 wb) {
        const LevelPlan& lp = q->plan.lv[lv_i];
        auto slot = [&](int s) -> int32_t { return s < nb ? pf.node(s, ps) : (s == nb ? n0 : n1); };
        int64_t lim = min(tend, sat_add(tprev, lp.gap));
        beg_out = 0;
        if (!STATS && lim <= tprev) return 0;
        const uint64_t span = (uint64_t)(lim - tprev);
        // words read ahead: an empty list empties the window (a closing
        // window is drawn from either of two lists)
        if (!STATS && (word_shows_empty(wa, span) || word_shows_empty(wb, span))) return 0;
        const int64_t* tarr;
        uint32_t b, hi, flag = 0;
        int kind = lp.kind;
        if (kind == FREE) {
            tarr = g.t;
            hi = (uint32_t)g.m;
            b = gallop_end(tarr, (uint32_t)edge_at(cdir, cpos, prev_e) + 1u, hi, tprev);
            if (STATS) acc.w[W_PROBE] += ceil_log2p1(hi);
        } else {
            int dir, nx;
            uint32_t lo;
            if (kind == CLOSE) {
                // the shorter of out(phi(x_i)) and in(phi(y_i))
                int32_t u = slot(lp.a), w = slot(lp.b);
                uint32_t u0 = __ldg(g.off[0] + u), u1 = __ldg(g.off[0] + u + 1);
                uint32_t w0 = __ldg(g.off[1] + w), w1 = __ldg(g.off[1] + w + 1);
                if (u1 - u0 <= w1 - w0) { dir = 0; lo = u0; hi = u1; nx = lp.nx_a; }
                else { dir = 1; lo = w0; hi = w1; nx = lp.nx_b; }
                if (!STATS && hi - lo >= PAIR_MIN_DEG) {
                    // a long list: if its time window is long too, take the u -> w
                    // edges straight from u's pair-ordered out-list instead of
                    // scanning the window for one neighbour
                    const int64_t* ta = g.at[dir];
                    uint32_t b0;
                    if (nx >= 0) {
                        const uint2 pw = dir ? wb : wa;
                        const uint2 w = pw.y ? pw : successor(nx, cdir, cpos, prev_e);
                        if (word_shows_empty(w, span)) return 0;
                        b0 = w.x;
                    } else {
                        b0 = upper_bound_t(ta, lo, hi, tprev);
                    }
                    uint32_t e0 = (b0 < hi) ? window_end(ta, b0, hi, lim) : b0;
                    if (e0 - b0 < PAIR_MIN_WINDOW) {
                        beg_out = b0 | (dir ? INLIST : 0u);
                        return e0 - b0;
                    }
                    uint32_t ps = lower_bound_i32(g.pnbr, u0, u1, w);
                    uint32_t pe = lower_bound_i32(g.pnbr, ps, u1, w + 1);
                    uint32_t pb = upper_bound_t(g.pt, ps, pe, tprev);
                    uint32_t pz = (pb < pe) ? window_end(g.pt, pb, pe, lim) : pb;
                    beg_out = pb | PAIRLIST;
                    return pz - pb;
                }
            } else {
                dir = kind == EXT_IN ? 1 : 0;
                int32_t v = slot(lp.a);
                nx = lp.nx_a;
                hi = __ldg(g.off[dir] + v + 1);
                lo = (nx >= 0 && !STATS) ? 0u : __ldg(g.off[dir] + v);
            }
            tarr = g.at[dir];
            flag = dir ? INLIST : 0u;
            if (nx >= 0) {
                const uint2 pw = (kind == CLOSE && dir) ? wb : wa;
                const uint2 w = pw.y ? pw : successor(nx, cdir, cpos, prev_e);
                if (!STATS && word_shows_empty(w, span)) return 0;
                b = w.x;
            } else {
                b = upper_bound_t(tarr, lo, hi, tprev);
            }
            if (STATS) acc.w[W_PROBE] += ceil_log2p1(hi - lo);
        }
        uint32_t e = (b < hi) ? window_end(tarr, b, hi, lim) : b;
        beg_out = b | flag;
        return e - b;
    }

    // Exclusive prefix of the window lengths of a frame's parents, kept in
    // registers: lane j holds parents 2j and 2j+1.
    struct Prefix {
        uint32_t preA, preB, lenA, lenB, tot;
    };
    __device__ Prefix prefix(Frame f, uint32_t np) const {
        const uint32_t a = 2u * lane, b = a + 1u;
        Prefix r;
        r.lenA = a < np ? f.len(a) : 0u;
        r.lenB = b < np ? f.len(b) : 0u;
        uint32_t s = r.lenA + r.lenB, inc = s;
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t u = __shfl_up_sync(FULL, inc, d);
            if (lane >= d) inc += u;
        }
        r.preA = inc - s;
        r.preB = r.preA + r.lenA;
        r.tot = __shfl_sync(FULL, inc, 31);
        return r;
    }

    // The parent whose window holds flattened position x (x < total) and its prefix.
    __device__ void owner(const Prefix& pr, uint32_t x, int& p, uint32_t& pre_p) const {
        bool oa = pr.lenA && pr.preA <= x && x - pr.preA < pr.lenA;
        bool ob = pr.lenB && pr.preB <= x && x - pr.preB < pr.lenB;
        unsigned ba = __ballot_sync(FULL, oa), bb = __ballot_sync(FULL, ob);
        int src = ba ? __ffs(ba) - 1 : __ffs(bb) - 1;
        uint32_t va = __shfl_sync(FULL, pr.preA, src), vb = __shfl_sync(FULL, pr.preB, src);
        p = 2 * src + (ba ? 0 : 1);
        pre_p = ba ? va : vb;
    }

    // Start a frame: its cursor and flattened total.
    __device__ uint32_t begin_frame(int i) {
        Prefix pr = prefix(frame(i), P(i));
        setOff(i, 0);
        setT(i, pr.tot);
        return pr.tot;
    }

    // Emit survivors of the last level (or of the root level when k == 1).
    __device__ void emit(bool ok, uint32_t root, Frame pf, int ps, int nb, int32_t last_eid) {
        unsigned bal = __ballot_sync(FULL, ok);
        if (!bal) return;
        unsigned cnt = __popc(bal);
        if (MODE == MODE_COUNT) {
            acc.total += cnt;
            if (STATS && lane == 0) acc.w[W_MATCH] += cnt;
            if (q->per_root && ok) {
                unsigned grp = __match_any_sync(bal, root);
                if (lane == __ffs(grp) - 1) atomicAdd(q->per_root + (root - q->root_begin), (unsigned long long)__popc(grp));
            }
            if (q->chunk_cnt && ok) {
                uint32_t c = (uint32_t)((root - q->root_begin) / (uint32_t)q->plan.tune.chunk_roots);
                unsigned grp = __match_any_sync(bal, c);
                if (lane == __ffs(grp) - 1) atomicAdd(q->chunk_cnt + c, (unsigned long long)__popc(grp));
            }
        } else {
            unsigned rank = __popc(bal & ((1u << lane) - 1u));
            unsigned long long pos = out_base + out_local + rank;
            if (ok && pos < q->cap) {
                int32_t* o = q->match_out + pos * (unsigned long long)k;
                for (int j = 0; j < k - 1; ++j) o[j] = pf.eid(nb, j, ps);
                o[k - 1] = last_eid;
            }
            out_local += cnt;
        }
    }

    // One 32-candidate step of frame i.
    __device__ void step(int i) {
        const LevelPlan& lp = q->plan.lv[i];
        Frame f = frame(i);
        const int nb = lp.nb;
        const uint32_t np = P(i), off = Off(i), tot = T(i);
        uint32_t idx = off + lane;
        bool act = idx < tot;
        // Lane -> parent without a search: the parent holding `off`, plus the
        // parents whose windows start inside this 32-wide step (a start mask).
        Prefix pr = prefix(f, np);
        int p0;
        uint32_t pre0;
        owner(pr, off, p0, pre0);
        const int a = 2 * lane, b = a + 1;
        unsigned mk = 0;
        if (a > p0 && pr.lenA && pr.preA - off < 32u) mk |= 1u << (pr.preA - off);
        if (b > p0 && pr.lenB && pr.preB - off < 32u) mk |= 1u << (pr.preB - off);
        const unsigned starts = __reduce_or_sync(FULL, mk);
        const unsigned le = starts & ((2u << lane) - 1u);
        const int p = p0 + __popc(le);
        const uint32_t within = le ? (uint32_t)(lane - (31 - __clz(le))) : (off - pre0 + (uint32_t)lane);
        int32_t n0 = -1, n1 = -1, ceid = -1;
        int64_t ct = 0;
        bool ok = act;
        const int kind = lp.kind;
        // the candidate's edge id: written by enumeration and read by edge labels;
        // the next level's successor lookup loads it only if it needs it
        const bool need_eid = (MODE == MODE_FILL) || lp.elabel >= 0;
        int cdir = 2;
        uint32_t pos = 0;
        uint2 wa = make_uint2(0u, 0u), wb = wa;   // next level's successor words, read with the candidate
        if (act) {
            uint32_t bw = f.beg(p);
            pos = (bw & POSMASK) + within;
            cdir = (bw & PAIRLIST) ? 3 : (kind == FREE ? 2 : ((bw & INLIST) ? 1 : 0));
            if (PREFETCH && !STATS && i < k - 1) next_words(q->plan.lv[i + 1], cdir, pos, wa, wb);
            if (bw & PAIRLIST) {
                // closing edge from the pair-ordered list: structure holds by construction
                ct = __ldg(g.pt + pos);
                if (need_eid) ceid = __ldg(g.peid + pos);
            } else if (kind == FREE) {
                ct = __ldg(g.t + pos);
                n0 = __ldg(g.src + pos);
                n1 = __ldg(g.dst + pos);
                ceid = (int32_t)pos;
                ok = n0 != n1;
                for (int j = 0; j < nb; ++j) {
                    int32_t x = f.node(j, p);
                    ok &= (x != n0) && (x != n1);
                }
                if (lp.nl0 >= 0) ok &= g.nlabel[n0] == (uint8_t)lp.nl0;
                if (lp.nl1 >= 0) ok &= g.nlabel[n1] == (uint8_t)lp.nl1;
            } else {
                int dir = (bw & INLIST) ? 1 : 0;
                ct = __ldg(g.at[dir] + pos);
                int32_t nbr = __ldg(g.anbr[dir] + pos);
                if (need_eid) ceid = __ldg(g.aeid[dir] + pos);
                if (kind == CLOSE) {
                    ok = nbr == f.node(dir ? lp.a : lp.b, p);
                } else {
                    n0 = nbr;
                    for (int j = 0; j < nb; ++j) ok &= f.node(j, p) != nbr;
                    if (lp.nl0 >= 0) ok &= g.nlabel[nbr] == (uint8_t)lp.nl0;
                }
            }
            if (lp.elabel >= 0) ok &= g.elabel[ceid] == (uint8_t)lp.elabel;
            if (ANTI && ok && lp.anti_mask)
                ok = anti_clear(lp.anti_mask, i, f, p, nb, n0, n1, ct, f.tprev(p), anti_off(i));
            if (LOOK && ok && lp.n_look) ok = look_ok(lp, f, p, nb, n0, n1, ct, tend_of(f, p));
        }
        uint32_t root = act ? f.root(p) : 0u;
        if (i == k - 1) {
            emit(ok, root, f, p, nb, ceid);
            return;
        }
        // expand survivors into frame i+1
        const int nb_c = q->plan.lv[i + 1].nb;
        uint32_t cbeg = 0, clen = 0;
        int64_t tend = 0;
        if (ok) {
            tend = tend_of(f, p);
            clen = locate(i + 1, f, p, nb, n0, n1, ceid, cdir, pos, ct, tend, cbeg, wa, wb);
        }
        if (STATS) {
            unsigned b = __ballot_sync(FULL, ok);
            uint32_t l = ok ? clen : 0u;
            for (int d = 16; d > 0; d >>= 1) l += __shfl_down_sync(FULL, l, d);
            if (lane == 0) {
                acc.w[W_NODES + (i + 1)] += __popc(b);
                acc.w[W_ENTRIES + (i + 1)] += l;
            }
        }
        bool keep = ok && clen > 0;
        unsigned kb = __ballot_sync(FULL, keep);
        if (!kb) return;
        uint32_t cp = P(i + 1);
        Frame c = frame(i + 1);
        if (keep) {
            int s = (int)(cp + __popc(kb & ((1u << lane) - 1u)));
            for (int j = 0; j < nb; ++j) c.node(j, s) = f.node(j, p);
            if (nb_c > nb) c.node(nb, s) = n0;
            if (nb_c > nb + 1) c.node(nb + 1, s) = n1;
            c.tprev(s) = ct;
            set_tend(c, s, ct, tend);
            c.beg(s) = cbeg;
            c.len(s) = clen;
            c.root(s) = root;
            if (MODE == MODE_FILL) {
                for (int j = 0; j < i; ++j) c.eid(nb_c, j, s) = f.eid(nb, j, p);
                c.eid(nb_c, i, s) = ceid;
            }
            const Plan& pl = q->plan;
            for (int a = 0; ANTI && a < pl.n_anti; ++a) {
                const int e = pl.anti[a].edge;
                if (e == i) c.anti_t(anti_off(i + 1), a, s) = ct;
                else if (e < i) c.anti_t(anti_off(i + 1), a, s) = f.anti_t(anti_off(i), a, p);
            }
        }
        __syncwarp();
        setP(i + 1, cp + __popc(kb));
    }

    // Donate the upper half of frame i's remaining candidates as tasks.
    __device__ void maybe_donate(int i) {
        const uint32_t np = P(i), off = Off(i), tot = T(i);
        const tm_tuning& tu = q->plan.tune;
        if (i > tu.split_depth || tot - off <= (uint32_t)tu.split_min || (ANTI && q->plan.n_anti)) return;
        if ((++polls & 15u) != 1u) return;      // look at the idle count every 16th step
        int idle = 0;
        if (lane == 0) idle = *(volatile int*)&ctrl->idle;
        idle = __shfl_sync(FULL, idle, 0);
        if (idle <= 0) return;
        Frame f = frame(i);
        uint32_t mid = off + ((tot - off) >> 1);
        mid = (mid + 31u) & ~31u;
        if (mid >= tot || mid <= off) return;
        // parent containing mid
        Prefix pr = prefix(f, np);
        int p0;
        uint32_t pre0;
        owner(pr, mid, p0, pre0);
        const int ntask = (int)np - p0;
        // a task is one parent's window range: donate only when the tasks carry
        // split_min candidates each on average, else the queue traffic costs
        // more than the work it moves
        if ((tot - mid) < (uint32_t)ntask * (uint32_t)max(tu.split_min, 32)) return;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctrl->q_reserve, (unsigned long long)ntask);
        base = __shfl_sync(FULL, base, 0);
        if (base + (unsigned long long)ntask > task_cap) {
            // no room: void the reserved slots that exist and keep the work
            for (int j = lane; j < ntask; j += 32)
                if (base + j < task_cap) *(volatile uint8_t*)&ready[base + j] = 2;
            return;
        }
        const int nb = q->plan.lv[i].nb;
        for (int j = lane; j < ntask; j += 32) {
            int p = p0 + j;
            uint32_t len = f.len(p), bw = f.beg(p);
            uint32_t skip = (p == p0) ? (mid - pre0) : 0u;
            Task* t = tasks + base + j;
            t->query = (int16_t)qi;
            t->level = (int16_t)i;
            t->beg = bw + skip;
            t->len = len - skip;
            t->tprev = f.tprev(p);
            t->tend = tend_of(f, p);
            t->root = f.root(p);
            for (int s = 0; s < nb; ++s) t->node[s] = f.node(s, p);
        }
        __threadfence();
        for (int j = lane; j < ntask; j += 32) *(volatile uint8_t*)&ready[base + j] = 1;
        __syncwarp();
        if (lane == 0) {
            f.len(p0) = mid - pre0;
            atomicAdd(&ctrl->donated, (unsigned)ntask);
        }
        __syncwarp();
        setP(i, (uint32_t)p0 + 1);
        setT(i, mid);
    }

    // Drain frame `base` (and everything below it) to completion.
    __device__ void drain(int base) {
        begin_frame(base);
        int lvl = base;
        while (true) {
            if (Off(lvl) < T(lvl)) {
                if (MODE == MODE_COUNT) maybe_donate(lvl);
                if (Off(lvl) < T(lvl)) {
                    step(lvl);
                    setOff(lvl, Off(lvl) + 32);
                    if (lvl < k - 1 && P(lvl + 1) >= DESCEND) { ++lvl; begin_frame(lvl); }
                }
                continue;
            }
            if (lvl < k - 1 && P(lvl + 1) > 0) { ++lvl; begin_frame(lvl); continue; }
            setP(lvl, 0);
            if (lvl == base) break;
            --lvl;
        }
    }

    // Roots [r0, r1) of the current query: level 0 of the search.
    __device__ void roots(uint64_t r0, uint64_t r1, bool flush_at_end) {
        const Plan& pl = q->plan;
        for (uint64_t rb = r0; rb < r1; rb += 32) {
            uint64_t r = rb + lane;
            bool ok = r < r1;
            int32_t s = 0, d = 0;
            int64_t tt = 0;
            uint2 wa = make_uint2(0u, 0u), wb = wa;
            if (ok) {
                if (PREFETCH && !STATS && k > 1) next_words(pl.lv[1], 2, (uint32_t)r, wa, wb);
                s = __ldg(g.src + r);
                d = __ldg(g.dst + r);
                tt = __ldg(g.t + r);
                ok = s != d;
                if (pl.elabel0 >= 0) ok &= g.elabel[r] == (uint8_t)pl.elabel0;
                if (pl.nl_x0 >= 0) ok &= g.nlabel[s] == (uint8_t)pl.nl_x0;
                if (pl.nl_y0 >= 0) ok &= g.nlabel[d] == (uint8_t)pl.nl_y0;
                if (ANTI && ok && pl.anti_mask0)
                    ok = anti_clear(pl.anti_mask0, 0, Frame{wbase}, 0, 0, s, d, tt, tt, 0);
                if (LOOK && ok && pl.lv[0].n_look)
                    ok = look_ok(pl.lv[0], Frame{wbase}, 0, 0, s, d, tt, sat_add(tt, pl.delta));
            }
            if (STATS && lane == 0) acc.w[W_ROOTS] += (r1 - rb < 32ull) ? (unsigned long long)(r1 - rb) : 32ull;
            if (k == 1) {
                emit(ok, (uint32_t)r, Frame{wbase}, 0, 0, (int32_t)r);
                continue;
            }
            uint32_t cbeg = 0, clen = 0;
            int64_t tend = 0;
            if (ok) {
                tend = sat_add(tt, pl.delta);
                clen = locate(1, Frame{wbase}, 0, 0, s, d, (int32_t)r, 2, (uint32_t)r, tt, tend, cbeg, wa, wb);
            }
            if (STATS) {
                unsigned b = __ballot_sync(FULL, ok);
                uint32_t l = ok ? clen : 0u;
                for (int dd = 16; dd > 0; dd >>= 1) l += __shfl_down_sync(FULL, l, dd);
                if (lane == 0) {
                    acc.w[W_NODES + 1] += __popc(b);
                    acc.w[W_ENTRIES + 1] += l;
                }
            }
            bool keep = ok && clen > 0;
            unsigned kb = __ballot_sync(FULL, keep);
            if (kb) {
                uint32_t cp = P(1);
                Frame c = frame(1);
                if (keep) {
                    int sl = (int)(cp + __popc(kb & ((1u << lane) - 1u)));
                    c.node(0, sl) = s;
                    c.node(1, sl) = d;
                    c.tprev(sl) = tt;
                    set_tend(c, sl, tt, tend);
                    c.beg(sl) = cbeg;
                    c.len(sl) = clen;
                    c.root(sl) = (uint32_t)r;
                    if (MODE == MODE_FILL) c.eid(2, 0, sl) = (int32_t)r;
                    for (int a = 0; ANTI && a < pl.n_anti; ++a)
                        if (pl.anti[a].edge == 0) c.anti_t(anti_off(1), a, sl) = tt;
                }
                __syncwarp();
                setP(1, cp + __popc(kb));
                if (cp + __popc(kb) >= DESCEND) drain(1);
            }
        }
        if (flush_at_end && k > 1 && P(1) > 0) drain(1);
    }

    __device__ void run_task(const Task& tk) {
        use_query(tk.query);
        const int i = tk.level;
        const int nb = q->plan.lv[i].nb;
        Frame f = frame(i);
        if (lane == 0) {
            f.tprev(0) = tk.tprev;
            set_tend(f, 0, tk.tprev, tk.tend);
            f.beg(0) = tk.beg;
            f.len(0) = tk.len;
            f.root(0) = tk.root;
            for (int s = 0; s < nb; ++s) f.node(s, 0) = tk.node[s];
        }
        __syncwarp();
        setP(i, 1);
        drain(i);
    }

    // Global chunk c -> query index (chunks of query j are contiguous).
    __device__ int query_of_chunk(uint64_t c, int nq) const {
        int lo = 0, hi = nq;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (qs[mid].chunk_base <= c) lo = mid; else hi = mid;
        }
        return lo;
    }

    __device__ bool try_pop(Task& out) {
        int got = 0;
        unsigned long long h = 0;
        if (lane == 0) {
            for (int attempt = 0; attempt < 64 && !got; ++attempt) {
                h = *(volatile unsigned long long*)&ctrl->q_head;
                unsigned long long r = *(volatile unsigned long long*)&ctrl->q_reserve;
                if (h >= min(r, (unsigned long long)task_cap)) break;
                if (atomicCAS(&ctrl->q_head, h, h + 1) != h) continue;
                uint64_t t0 = now_ns();
                uint8_t st = 0;
                while ((st = *(volatile uint8_t*)&ready[h]) == 0) {
                    if (now_ns() - t0 > READY_NS) { atomicMax(&ctrl->err, (unsigned)TM_E_TIMEOUT); break; }
                    __nanosleep(64);
                }
                if (st == 1) got = 1;
            }
        }
        got = __shfl_sync(FULL, got, 0);
        if (!got) return false;
        h = __shfl_sync(FULL, h, 0);
        __threadfence();
        const uint32_t* src = (const uint32_t*)(tasks + h);
        uint32_t w = lane < 16 ? __ldcg(src + lane) : 0u;
        uint32_t* dst = (uint32_t*)&out;
        for (int j = 0; j < 16; ++j) dst[j] = __shfl_sync(FULL, w, j);
        return true;
    }

    __device__ bool queue_empty() const {
        unsigned long long h = *(volatile unsigned long long*)&ctrl->q_head;
        unsigned long long r = *(volatile unsigned long long*)&ctrl->q_reserve;
        return h >= min(r, (unsigned long long)task_cap);
    }

    __device__ void run(int nq, uint64_t total_chunks) {
        if (MODE == MODE_COUNT && lane == 0) atomicAdd(&ctrl->busy, 1);
        // phase 1: root chunks
        while (true) {
            unsigned long long c = 0;
            if (lane == 0) c = atomicAdd(&ctrl->next_chunk, 1ULL);
            c = __shfl_sync(FULL, c, 0);
            if (c >= total_chunks) break;
            int j = query_of_chunk(c, nq);
            if (j != qi) {
                // frames of the previous query must be empty before switching
                if (MODE == MODE_COUNT && qi >= 0 && k > 1 && P(1) > 0) drain(1);
                use_query(j);
            }
            uint64_t lc = c - q->chunk_base;
            const uint64_t cr = (uint64_t)q->plan.tune.chunk_roots;
            if (MODE == MODE_FILL) {
                // claim index lc -> the lc-th listed chunk (one holding a match whose
                // rows start below the cap); past the list's end the rest of this
                // query is skipped
                if (lc >= q->chunk_off[q->n_chunks + 1]) {
                    unsigned long long nxt = (j + 1 < nq) ? qs[j + 1].chunk_base : total_chunks;
                    if (lane == 0) atomicMax(&ctrl->next_chunk, nxt);
                    continue;
                }
                lc = ((const uint32_t*)(q->chunk_off + q->n_chunks + 2))[lc];
                out_base = q->chunk_off[lc];
                out_local = 0;
            }
            const uint64_t r0 = q->root_begin + lc * cr;
            const uint64_t r1 = min(q->root_end, r0 + cr);
            roots(r0, r1, MODE == MODE_FILL);
        }
        if (MODE == MODE_COUNT && qi >= 0 && k > 1 && P(1) > 0) drain(1);
        // phase 2 (count): help with donated subtrees until no warp holds work
        if (MODE == MODE_COUNT) {
            Task tk;
            while (true) {
                if (try_pop(tk)) { run_task(tk); continue; }
                int leave = 0;
                if (lane == 0) {
                    atomicSub(&ctrl->busy, 1);
                    atomicAdd(&ctrl->idle, 1);
                    uint64_t t0 = now_ns();
                    unsigned ns = 256;
                    while (true) {
                        if (!queue_empty()) { atomicAdd(&ctrl->busy, 1); break; }
                        int b = *(volatile int*)&ctrl->busy;
                        if (b == 0) {
                            // no warp holds work: leave unless a donation landed meanwhile
                            __threadfence();
                            if (queue_empty()) { leave = 1; break; }
                            continue;
                        }
                        if (now_ns() - t0 > WAIT_NS) { leave = 1; break; }
                        __nanosleep(ns);     // back off: waiting warps poll one shared line
                        if (ns < 8192) ns <<= 1;
                    }
                    atomicSub(&ctrl->idle, 1);
                }
                leave = __shfl_sync(FULL, leave, 0);
                if (leave) break;
            }
        }
        flush();
    }
};

template <int MODE, bool STATS, int FEAT>
__global__ void __maxnreg__(56) search_kernel(const __grid_constant__ GraphView g,
                                                     const QueryDev* __restrict__ qs, int nq, int warp_smem,
                                                     Ctrl* ctrl, Task* tasks, uint8_t* ready, uint64_t task_cap) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5;
    Search<MODE, STATS, FEAT> s(g, qs, ctrl, tasks, ready, task_cap, smem + (size_t)warp * warp_smem);
    s.run(nq, ctrl->total_chunks);
}

}  // namespace

namespace {

// The chunks of an enumeration that hold a match and whose rows start below
// the cap, from the scanned row offsets: their ids are appended (in no
// particular order) after the offsets and the list length (zeroed by the
// caller), for the fill pass to claim.
__global__ void list_chunks_kernel(unsigned long long* buf, uint64_t nch, uint64_t cap) {
    const unsigned long long* off = buf;
    unsigned long long* n_list = buf + nch + 1;
    uint32_t* list = (uint32_t*)(buf + nch + 2);
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nch; base += stride) {
        const uint64_t c = base + lane;
        const bool keep = c < nch && off[c + 1] > off[c] && off[c] < cap;
        const unsigned b = __ballot_sync(FULL, keep);
        if (!b) continue;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(n_list, (unsigned long long)__popc(b));
        at = __shfl_sync(FULL, at, 0);
        if (keep) list[at + __popc(b & ((1u << lane) - 1u))] = (uint32_t)c;
    }
}

}  // namespace

tm_status list_chunks(unsigned long long* chunk_buf, uint64_t nch, uint64_t cap, int num_sms, cudaStream_t st) {
    if (nch == 0) return TM_OK;
    const uint64_t blocks = std::min<uint64_t>((nch + 255) / 256, (uint64_t)num_sms * 8);
    list_chunks_kernel<<<(unsigned)blocks, 256, 0, st>>>(chunk_buf, nch, cap);
    note_launches(1);
    TM_CUDA(cudaGetLastError());
    return TM_OK;
}

namespace {
std::mutex g_cfg_mu;
std::unordered_map<uint64_t, int> g_blocks_per_sm;   // (device, kernel, warps, smem) -> resident blocks per SM

// Kernel instances: count and fill for each feature set (anti-edge checks,
// look-ahead checks), and count with work counters (all features).  A query
// runs the instance holding only the code its plan needs.
template <int MODE>
const void* kernel_for(unsigned feat) {
    switch (feat & 3u) {
        case 0: return (const void*)search_kernel<MODE, false, 0>;
        case 1: return (const void*)search_kernel<MODE, false, 1>;
        case 2: return (const void*)search_kernel<MODE, false, 2>;
        default: return (const void*)search_kernel<MODE, false, 3>;
    }
}
const void* kernel_of(Mode mode, bool stats, unsigned feat) {
    if (mode == MODE_FILL) return kernel_for<MODE_FILL>(feat);
    if (stats) return (const void*)search_kernel<MODE_COUNT, true, 3>;
    return kernel_for<MODE_COUNT>(feat);
}

// Resident blocks per SM for one launch shape, computed once per shape.
int blocks_per_sm(const tm_graph* g, const void* fn, int kid, int threads, int smem) {
    uint64_t key = ((uint64_t)g->device << 56) | ((uint64_t)kid << 48) | ((uint64_t)threads << 32) | (uint64_t)smem;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    auto it = g_blocks_per_sm.find(key);
    if (it != g_blocks_per_sm.end()) return it->second;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem);
    cudaGetLastError();
    if (blocks < 1) blocks = 1;
    g_blocks_per_sm[key] = blocks;
    return blocks;
}
}  // namespace

LaunchCfg search_launch_cfg(const tm_graph* g, Mode mode, int max_warp_smem, int warps_per_block) {
    LaunchCfg c;
    c.warps_per_block = std::max(1, std::min(16, warps_per_block));
    // keep the block's frames within the 227 KB of shared memory a block may use
    while (c.warps_per_block > 1 && max_warp_smem * c.warps_per_block > 232448) c.warps_per_block--;
    c.smem_bytes = max_warp_smem * c.warps_per_block;
    int kid = mode == MODE_FILL ? 8 : 0;
    c.grid = blocks_per_sm(g, kernel_of(mode, false, 0u), kid, c.warps_per_block * 32, c.smem_bytes) * g->num_sms;
    return c;
}

tm_status launch_search(const tm_graph* g, Mode mode, const QueryDev* qdev_dev, int nq, int max_warp_smem,
                        int warps_per_block, unsigned feat, const Scratch* s, cudaStream_t st, int grid_override,
                        bool stats) {
    LaunchCfg c = search_launch_cfg(g, mode, max_warp_smem, warps_per_block);
    int grid = grid_override > 0 ? grid_override : c.grid;
    if (mode == MODE_FILL) stats = false;
    const void* fn = kernel_of(mode, stats, feat);
    // the instance's shared-memory limit (set once per launch shape)
    blocks_per_sm(g, fn, (mode == MODE_FILL ? 8 : 0) + (stats ? 4 : 0) + (int)(feat & 3u), c.warps_per_block * 32,
                  c.smem_bytes);
    GraphView v = g->v;
    Ctrl* ctrl = s->ctrl();
    Task* tasks = s->tasks;
    uint8_t* ready = s->ready;
    uint64_t cap = s->task_cap;
    void* args[] = {&v, (void*)&qdev_dev, &nq, &max_warp_smem, &ctrl, &tasks, &ready, &cap};
    TM_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(c.warps_per_block * 32), args, (size_t)c.smem_bytes, st));
    note_launches(1);
    return TM_OK;
}

}  // namespace tmg
