// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tm.h"

namespace tmg {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);

// Kernels this library has launched (all entry points, all threads).
void note_launches(uint64_t n);
tm_status cuda_fail(cudaError_t e, const char* what);

// Every device and pinned-host allocation of the library goes through these,
// so that tm_inject_alloc_failure can make one of them fail like an
// out-of-memory device (cudaErrorMemoryAllocation, nothing allocated).
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
cudaError_t host_alloc_pinned(void** p, size_t bytes);

// Select the device and drop any error another library left on this thread,
// so that only this call's own CUDA errors are reported.
#define TM_ENTER(dev)                                         \
    do {                                                      \
        cudaGetLastError();                                   \
        TM_CUDA(cudaSetDevice(dev));                          \
    } while (0)

#define TM_CUDA(call)                                         \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return tmg::cuda_fail(_e, #call); \
    } while (0)

// ------------------------------------------------------------ device graph

// Device-resident temporal graph (paper Section 2.2): the chronological edge
// list plus out- and in-adjacency in time order, stored column-wise so that a
// binary search touches only the time column and a window scan reads
// contiguous (t, neighbour) runs.
struct GraphView {
    int64_t n, m;
    const int32_t* src;       // by edge id
    const int32_t* dst;
    const int64_t* t;
    const uint8_t* elabel;    // nullable
    const uint8_t* nlabel;    // nullable
    const uint32_t* off[2];   // [0] out, [1] in : n+1 list offsets
    const int64_t* at[2];     // list entry time
    const int32_t* anbr[2];   // list entry neighbour (dst for out, src for in)
    const int32_t* aeid[2];   // list entry edge id
    // successor index, by edge id e = (u, v, t): first position with time > t in
    // out(u), in(v), out(v), in(u).  Each word is {x: absolute position in the
    // list columns, y: time of that entry minus t, saturated at SUCC_FAR, or
    // SUCC_END when the list has no later entry}, so one load both starts a
    // window and, for most windows, proves it empty.
    const uint2* nxt[4];
    // the same, indexed by list position for the common continuations: [0] out-list
    // entry -> next later in that out-list, [1] out-list entry -> out(its neighbour),
    // [2] in-list entry -> next later in that in-list, [3] in-list entry -> in(its neighbour)
    const uint2* pnx[4];
    // out-lists again, ordered by (neighbour, time) within each node (offsets off[0]):
    // the edges u -> v form one contiguous, time-ordered range
    const int32_t* pnbr;
    const int64_t* pt;
    const int32_t* peid;
};

constexpr uint32_t SUCC_END = 0xFFFFFFFFu;   // successor word: no later entry in the list
constexpr uint32_t SUCC_FAR = 0xFFFFFFFEu;   // successor word: time gap >= this

enum SuccKind : int8_t { NX_OUT_SRC = 0, NX_IN_DST = 1, NX_OUT_DST = 2, NX_IN_SRC = 3, NX_NONE = -1 };

struct TuneKey {
    uint64_t shape;     // motif structure hash
    int dbucket;        // floor(log2(delta + 1))
    bool operator==(const TuneKey& o) const { return shape == o.shape && dbucket == o.dbucket; }
};
struct TuneKeyHash {
    size_t operator()(const TuneKey& k) const { return (size_t)(k.shape * 1315423911ULL + (uint64_t)k.dbucket); }
};

}  // namespace tmg

struct tm_graph {
    int device = 0;
    tmg::GraphView v{};
    std::vector<void*> allocs;     // device buffers owned by the graph
    char* slab = nullptr;          // the graph's columns, carved from one allocation
    size_t slab_used = 0, slab_cap = 0;
    int32_t* perm = nullptr;       // device: edge id -> input index
    uint64_t device_bytes = 0;
    int num_sms = 0;
    std::mutex tune_mu;
    std::unordered_map<tmg::TuneKey, tm_tuning, tmg::TuneKeyHash> tuned;
    // serving: device ms one request of a (shape, delta bucket, flavour) takes,
    // learnt from timed launches and shared by every server of this graph
    std::mutex cost_mu;
    std::unordered_map<uint64_t, double> serve_cost_ms;
};

namespace tmg {

// --------------------------------------------------------------- the plan

enum LevelKind : int8_t { EXT_OUT = 0, EXT_IN = 1, CLOSE = 2, FREE = 3 };

// How one search level binds motif edge i (paper Section 5.1.2 "minfo"):
// which mapped node supplies the candidate list, which mapped nodes a new
// node must differ from, and the constraints checked on a candidate.
constexpr int TM_MAX_LOOK = 3;

struct LevelPlan {
    int8_t kind;       // LevelKind
    int8_t a;          // EXT_OUT: slot of x_i; EXT_IN: slot of y_i; CLOSE: slot of x_i
    int8_t b;          // CLOSE: slot of y_i
    int8_t nb;         // slots bound before this level
    int16_t elabel;    // -1 = any
    int16_t nl0;       // label of the (first) new node, -1 = any
    int16_t nl1;       // FREE: label of the second new node (y_i)
    int8_t nx_a;       // SuccKind giving the window start of the list used by EXT / CLOSE(out) levels
    int8_t nx_b;       // SuccKind for the in-list option of a CLOSE level
    uint8_t anti_mask; // anti-edges whose nodes and attached edge are all bound once edge i is
    uint8_t n_look;    // later motif edges (after i+1) whose two nodes are first both bound by edge i
    int8_t look_u[TM_MAX_LOOK];  // their endpoint slots: an edge look_u -> look_v must exist in
    int8_t look_v[TM_MAX_LOOK];  // (t_i, t_root + delta], else no match extends this partial match
    int8_t pad2[4];
    int32_t frame_off;       // byte offset of this level's frame in a warp's shared block (count)
    int32_t frame_off_fill;  // same, enumerate-fill layout (frames also carry edge ids)
    int32_t anti_row_off;    // byte offset of the anti-edge time rows within this level's frame
    int32_t anti_row_off_fill;
    int64_t gap;             // t_i - t_{i-1} bound (INT64_MAX = none)
};

// One temporal anti-edge (paper Section 2.1, Section 5.4.3), checked at the
// level where its two nodes and its attached edge are all bound.
struct AntiPlan {
    int8_t xs, ys;     // slots of the absent edge's endpoints
    int8_t edge;       // attached motif edge i
    int8_t same_pair;  // the attached edge joins the same two nodes (exclude it)
    int32_t pad;
    int64_t delta;     // window [t(e_i), t(e_i) + delta]
};

// Parents per frame (at most two per lane).  A level is descended into once its
// frame holds cap - 32 parents, so one more 32-wide step of its parent level
// always fits.  Count frames hold 48 (descend at 16): the smaller shared
// memory footprint leaves more of each SM's unified L1 / shared memory to L1;
// fill frames carry edge ids and keep 64 (descend at 32).
constexpr int FCAP_COUNT = 48;
constexpr int FCAP_FILL = 64;

struct Plan {
    int32_t k, n_nodes;
    int64_t delta;
    int16_t elabel0, nl_x0, nl_y0, pad0;
    int32_t warp_smem;             // bytes of shared memory a warp needs (count)
    int32_t warp_smem_fill;        // same, enumerate fill
    tm_tuning tune;
    uint64_t shape_hash;
    int32_t n_anti;
    uint8_t anti_mask0;            // anti-edges checked when the root binds edge 0
    uint8_t pad1[3];
    AntiPlan anti[TM_MAX_ANTI];
    LevelPlan lv[TM_MAX_EDGES];    // lv[i] for i = 1..k-1 (lv[0]: only the look-ahead of the root)
};

// Code a plan needs beyond plain search: anti-edge checks, look-ahead checks.
constexpr unsigned FEAT_ANTI = 1u, FEAT_LOOK = 2u;
inline unsigned plan_features(const Plan& p) {
    unsigned f = p.n_anti > 0 ? FEAT_ANTI : 0u;
    for (int i = 0; i < TM_MAX_EDGES; ++i)
        if (p.lv[i].n_look) f |= FEAT_LOOK;
    return f;
}

// Frame field offsets (bytes, relative to frame start), CAP entries each.
//   tprev i64, tend - tprev u32 (0xFFFFFFFF when it does not fit: t_root + delta is
//   then rebuilt from the root edge), beg u32 (bits 31/30: list kind), len u32, root u32,
//   node[nb] i32, eid[i] i32 (enumerate only), anti_t[n_anti] i64 (motifs with
//   anti-edges: time of each anti-edge's attached edge once bound)
template <int CAP>
struct FrameLayout {
    static constexpr int TPREV = 0;
    static constexpr int TEND = TPREV + 8 * CAP;
    static constexpr int BEG = TEND + 4 * CAP;
    static constexpr int LEN = BEG + 4 * CAP;
    static constexpr int ROOT = LEN + 4 * CAP;
    static constexpr int NODE = ROOT + 4 * CAP;
};
// Count frames (no edge ids) or fill frames (edge ids of the bound edges).
inline int frame_bytes(int nb, int level, bool with_eids, int n_anti = 0) {
    if (with_eids)
        return FrameLayout<FCAP_FILL>::NODE + 4 * FCAP_FILL * (nb + level) + 8 * FCAP_FILL * n_anti;
    return FrameLayout<FCAP_COUNT>::NODE + 4 * FCAP_COUNT * nb + 8 * FCAP_COUNT * n_anti;
}
constexpr int WARP_HDR = 128;      // per-warp header: level cursors

tm_status build_plan(const tm_graph* g, const tm_motif* m, Plan* out);
uint64_t plan_shape_hash(const tm_motif* m);

// --------------------------------------------------------- device scratch

// Donated search task: one partial match (its mapped nodes, times and window).
struct Task {
    int16_t query;
    int16_t level;
    uint32_t beg;        // bit 31: in-list
    uint32_t len;
    uint32_t root;
    int64_t tprev;
    int64_t tend;
    int32_t node[TM_MAX_NODES];
};
static_assert(sizeof(Task) == 64, "task is one 64-byte record");

// Per-launch control block.  The root-chunk cursor is claimed by every warp
// many times per launch; the queue and idle counters are polled by waiting
// warps: they sit on separate 128-byte lines so polling never delays claims.
struct Ctrl {
    unsigned long long total_chunks; // root chunks of all queries of the launch
    unsigned long long pad0[15];
    unsigned long long next_chunk;   // root-chunk cursor (own line)
    unsigned long long pad1[15];
    unsigned long long q_reserve;    // task slots reserved by donors
    unsigned long long q_head;       // next task slot to pop
    int busy;                        // warps holding work
    int idle;                        // warps waiting for tasks
    unsigned int err;                // 0 or TM_E_TIMEOUT
    unsigned int donated;            // tasks donated (diagnostic)
    unsigned long long pad2[12];
};
static_assert(sizeof(Ctrl) == 384, "control block is three 128-byte lines");

// Enumeration chunk buffer of a query with nch root chunks: nch + 1 per-chunk
// match counts (scanned in place into row offsets by the caller), then the
// number of chunks holding a match whose rows start below the cap, and those
// chunks' ids (uint32, in no particular order; written by list_chunks after
// the scan).  The fill pass searches only the listed chunks.  The count pass
// needs the counts and the list length zeroed: the first (nch + 2) * 8 bytes.
inline size_t chunk_buf_bytes(uint64_t nch) { return (size_t)(nch + 2) * 8 + (size_t)nch * 4; }

struct QueryDev {                    // one query of a launch
    Plan plan;
    uint64_t root_begin, root_end;
    uint64_t n_chunks;
    uint64_t chunk_base;             // first global chunk index of this query
    unsigned long long* total;       // device counter
    unsigned long long* per_root;    // nullable (indexed by root - root_begin)
    unsigned long long* chunk_cnt;   // nullable (enumerate count pass): chunk buffer, counts + list
    const unsigned long long* chunk_off;  // enumerate fill: chunk buffer, offsets + list
    int32_t* match_out;              // enumerate fill
    uint64_t cap;
    unsigned long long* work;        // nullable: tm_work counters (2 + 2*TM_MAX_EDGES + 1)
};

// Device memory a launch uses beyond its inputs and outputs, plus the pinned
// host staging it is initialised from.  Layout of `head` (device) and `stage`
// (pinned host): one Ctrl, then nq QueryDev records.
struct Scratch {
    int device = 0;
    char* head = nullptr;            // device: Ctrl + QueryDev[qcap]
    char* stage = nullptr;           // pinned host mirror of head
    int qcap = 0;
    Task* tasks = nullptr;
    uint8_t* ready = nullptr;
    uint64_t task_cap = 0;
    unsigned long long* counters = nullptr;   // device: totals, work counters
    unsigned long long* counters_host = nullptr;  // pinned mirror
    uint64_t counters_len = 0;
    unsigned long long* chunk_cnt = nullptr;  // device: enumerate per-chunk counts / offsets
    uint64_t chunk_cap = 0;
    void* scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    Ctrl* ctrl() const { return (Ctrl*)head; }
    QueryDev* qdev() const { return (QueryDev*)(head + sizeof(Ctrl)); }
    Ctrl* ctrl_stage() const { return (Ctrl*)stage; }
    QueryDev* qdev_stage() const { return (QueryDev*)(stage + sizeof(Ctrl)); }
    size_t head_bytes(int nq) const { return sizeof(Ctrl) + (size_t)nq * sizeof(QueryDev); }
};

void drop_batches(const tm_graph* g);

// Record the donation counters of a finished count-mode launch for
// tm_last_search_stats (per calling thread).
void note_search_stats(const Ctrl& c);

// The query's plan with the graph's cached tuning for its shape applied.
void query_plan(tm_query* q, Plan* out);

// The graph a query was compiled for, and the motif it was compiled from.
const tm_graph* query_graph(const tm_query* q);
const tm_motif* query_motif(const tm_query* q);

// List the chunks of a scanned chunk buffer that the fill pass must search.
tm_status list_chunks(unsigned long long* chunk_buf, uint64_t nch, uint64_t cap, int num_sms, cudaStream_t st);

tm_status scratch_reserve(Scratch* s, int device, int nq, uint64_t counters_len, uint64_t chunks,
                          uint64_t task_cap);
void scratch_free(Scratch* s);

enum Mode { MODE_COUNT = 0, MODE_FILL = 1 };

struct LaunchCfg {
    int warps_per_block;
    int grid;
    int smem_bytes;      // per block
};

// Queries that share one persistent launch.  A launch has one frame size and
// one block size for all its warps, so a query with large frames (a deep motif)
// would lower the occupancy of every other query of the launch; queries whose
// own launch shape allows the same resident blocks per SM go together instead.
struct LaunchGroup {
    int first, count;    // positions in the grouped order
    int warp_smem;       // frame bytes per warp (largest of the group)
    int warps;           // warps per block
    unsigned feat;       // union of the group's plan features
};
// Groups of nq plans for `mode`; order[i] = index of the query at grouped position i.
std::vector<LaunchGroup> occupancy_groups(const tm_graph* g, Mode mode, const Plan* const* plans, int nq,
                                          int* order);

// Launch the persistent search over nq queries (qdev already on the device).
// Ctrl (incl. total_chunks) and qdev must already be initialised on the stream.
// `feat` selects the kernel instance: the union of plan_features() over the
// nq queries (an instance without a feature a query needs gives wrong counts).
tm_status launch_search(const tm_graph* g, Mode mode, const QueryDev* qdev_dev, int nq,
                        int max_warp_smem, int warps_per_block, unsigned feat,
                        const Scratch* s, cudaStream_t st, int grid_override = 0, bool stats = false);

LaunchCfg search_launch_cfg(const tm_graph* g, Mode mode, int max_warp_smem, int warps_per_block);

// ------------------------------------------------------------- primitives

// Exclusive prefix sum of n uint64 values (in place allowed).  Needs
// scan_temp_bytes(n) bytes of device temp.
size_t scan_temp_bytes(uint64_t n);
tm_status exclusive_scan_u64(const unsigned long long* in, unsigned long long* out, uint64_t n,
                             void* temp, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
// keys/vals are double-buffered: on return *_a holds the result.
tm_status radix_sort_pairs(uint64_t* keys_a, uint64_t* keys_b, uint32_t* vals_a, uint32_t* vals_b,
                           uint64_t n, int bits, void* temp, size_t temp_bytes, cudaStream_t st);
tm_status radix_sort_pairs32(uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a, uint32_t* vals_b,
                             uint64_t n, int bits, void* temp, size_t temp_bytes, cudaStream_t st);
size_t radix_temp_bytes(uint64_t n);

}  // namespace tmg
