/*
 * tm.h -- C ABI of the GB300 temporal-motif mining library (libtmgb300.so).
 *
 * Problem (paper Section 2.1): a temporal graph is a set of directed edges
 * (u, v, t); a motif is k edges (x_i -> y_i) over motif nodes, matched in
 * strictly increasing time with first-to-last span <= delta, optional per-gap
 * bounds t_{i+1} - t_i <= gap_i (fine-grained delta-temporal motif) and
 * optional label equalities on edges and nodes (Section 5.4.1).  Matches are
 * isomorphic: motif nodes map injectively to graph nodes.  Output is a count
 * or the list of matches (Section 2.1, "two flavors of output").
 *
 * Conventions for every call:
 *   - Every call returns tm_status; no C++ exception crosses this boundary.
 *   - On an error status, outputs are left untouched, except TM_E_TRUNCATED
 *     (non-fatal, see tm_enumerate).
 *   - "device pointer" means memory of the graph's CUDA device (cudaMalloc,
 *     a torch CUDA tensor's data_ptr, ...); "host pointer" means pageable or
 *     pinned host memory.  Caller-owned buffers stay caller-owned.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return host-visible results synchronise that stream
 *     before returning.
 *   - Edge ids: edges are ranked by (t, input index); edge id = rank.  Every
 *     edge id the library reports refers to this order (tm_graph_edge_perm
 *     maps it back to input positions).
 *   - Limits: n_edges < 2^30 - 1, n_nodes < 2^31 - 1, timestamps >= 0
 *     (int64 seconds or any unit), k <= 8 motif edges, <= 8 motif nodes.
 */
#ifndef TM_H
#define TM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TM_OK = 0,
    TM_E_INVALID = 1,    /* bad argument, graph or motif */
    TM_E_OOM = 2,        /* device allocation failed */
    TM_E_TRUNCATED = 3,  /* non-fatal: enumeration hit its cap; total is exact */
    TM_E_TIMEOUT = 4,    /* a bounded device wait ran out (result discarded) */
    TM_E_CUDA = 5,       /* CUDA runtime error */
    TM_E_BUSY = 6,       /* serve poll: request not finished yet */
    TM_E_ADMISSION = 7   /* serve: request can never fit the memory budget */
} tm_status;

#define TM_MAX_EDGES 8
#define TM_MAX_NODES 8
#define TM_MAX_ANTI 4

/* Input edge list (paper Section 2.2: a chronologically ordered temporal edge
 * list; here any order is accepted and the library sorts it).
 *   src, dst : int32[n_edges], node ids in [0, n_nodes)
 *   t        : int64[n_edges], >= 0
 *   elabel   : uint8[n_edges] or NULL     (edge labels)
 *   nlabel   : uint8[n_nodes] or NULL     (node labels)
 *   on_device: 0 = all pointers are host pointers, 1 = device pointers.
 * The library copies what it needs; the caller may free these after load. */
typedef struct {
    int64_t n_nodes;
    int64_t n_edges;
    const int32_t* src;
    const int32_t* dst;
    const int64_t* t;
    const uint8_t* elabel;
    const uint8_t* nlabel;
    int32_t on_device;
} tm_edges;

/* Motif query (Section 2.1 definitions; Section 4.3 query constraints).
 *   k          : motif edges, 1..8, listed in temporal order
 *   n_nodes    : motif nodes, 2..8; every node must appear in some edge
 *   esrc/edst  : x_i, y_i of motif edge i, x_i != y_i
 *   delta      : t(e_{k-1}) - t(e_0) <= delta, delta >= 0 (inclusive)
 *   gap[i]     : t(e_{i+1}) - t(e_i) <= gap[i]; INT64_MAX = unconstrained
 *   elabel[i]  : required label of edge i, -1 = any (needs graph elabel)
 *   nlabel[j]  : required label of motif node j, -1 = any (needs graph nlabel)
 *   n_anti     : temporal anti-edges, 0..4 (Section 2.1, Section 5.4.3).
 *                Anti-edge a forbids any graph edge other than e_i, with
 *                i = anti_edge[a], from phi(anti_src[a]) to phi(anti_dst[a])
 *                at a time in the closed window [t(e_i), t(e_i) + anti_delta[a]].
 *                Both nodes must appear in some motif edge; anti_delta >= 0.
 * Edge times within a match are strictly increasing; graph self-loops never
 * match (motif edges join distinct nodes). */
typedef struct {
    int32_t k;
    int32_t n_nodes;
    uint8_t esrc[TM_MAX_EDGES];
    uint8_t edst[TM_MAX_EDGES];
    int64_t delta;
    int64_t gap[TM_MAX_EDGES - 1];
    int16_t elabel[TM_MAX_EDGES];
    int16_t nlabel[TM_MAX_NODES];
    int32_t n_anti;
    uint8_t anti_src[TM_MAX_ANTI];
    uint8_t anti_dst[TM_MAX_ANTI];
    uint8_t anti_edge[TM_MAX_ANTI];
    int64_t anti_delta[TM_MAX_ANTI];
} tm_motif;

/* Execution knobs for one query shape (see tm_autotune).
 *   warps_per_block : 1..16 (reduced automatically when the block's search
 *                     frames would not fit in shared memory)
 *   chunk_roots     : root edges a warp claims at a time (multiple of 32)
 *   split_depth     : deepest search level whose remaining candidates may be
 *                     donated to idle warps: level i holds the candidate windows
 *                     of motif edge i (1 = the root edges' windows, up to k-1);
 *                     0 or -1 disables donation (always off for motifs with
 *                     anti-edges)
 *   split_min       : a donation moves, on average, at least this many
 *                     candidates per donated task */
typedef struct {
    int32_t warps_per_block;
    int32_t chunk_roots;
    int32_t split_depth;
    int32_t split_min;
} tm_tuning;

/* Work of one query's search tree: used as the numerator of the bandwidth
 * roofline.  nodes[i] = partial matches of i edges that locate a window for
 * edge i; entries[i] = candidates in those windows; probe_sectors = sum over
 * located windows of ceil(log2(list length + 1)).  For motifs without chords
 * (no later edge between nodes that no earlier edge joins) this is the tree of
 * the paper's Algorithm 1 (Section 2.2); otherwise the tree after the search's
 * look-ahead pruning, which drops partial matches whose later chords have no
 * graph edge left in the window. */
typedef struct {
    uint64_t roots;
    uint64_t nodes[TM_MAX_EDGES];
    uint64_t entries[TM_MAX_EDGES];
    uint64_t probe_sectors;
    uint64_t matches;
} tm_work;

typedef struct tm_graph tm_graph;
typedef struct tm_query tm_query;
typedef struct tm_server tm_server;

/* Build the device-resident graph (paper Section 4.2 data loader; Section 2.2
 * layout): stable sort by (t, input index), then per-node out- and in-lists of
 * (neighbour, edge id, t) in time order.  Runs on `device`, ordered on
 * `stream`; returns after the build has finished.  *out is library-owned. */
tm_status tm_graph_load(const tm_edges* edges, int device, void* stream, tm_graph** out);

/* Release a graph and its device memory.  NULL is accepted. */
tm_status tm_graph_free(tm_graph* g);

/* Sizes of a loaded graph (any pointer may be NULL). */
tm_status tm_graph_info(const tm_graph* g, int64_t* n_nodes, int64_t* n_edges, uint64_t* device_bytes);

/* Edge id -> input index.  out_perm: int64[n_edges], host pointer. */
tm_status tm_graph_edge_perm(const tm_graph* g, int64_t* out_perm);

/* Validate a motif against a graph and build its search plan (Section 5.1.2:
 * per-level candidate source, mapped-node checks and constraints).  Returns
 * TM_E_INVALID for a malformed motif or label constraints the graph cannot
 * evaluate.  The query owns its scratch memory: one query must not run on two
 * streams at the same time. */
tm_status tm_query_compile(const tm_graph* g, const tm_motif* motif, tm_query** out);
/* A graph must outlive the queries and servers made from it; a query may be
 * freed before or after its graph. */
tm_status tm_query_free(tm_query* q);

/* Override / read the execution knobs of a query. */
tm_status tm_query_set_tuning(tm_query* q, const tm_tuning* tuning);
tm_status tm_query_get_tuning(const tm_query* q, tm_tuning* tuning);

/* Count matches (Section 2.1; search of Algorithm 1 rooted at every edge).
 *   total        : host pointer, receives the exact count
 *   per_root_dev : device pointer uint64[n_edges] or NULL; entry r receives the
 *                  number of matches whose first edge is edge id r
 * Synchronises the stream. */
tm_status tm_count(tm_graph* g, tm_query* q, void* stream, uint64_t* total, uint64_t* per_root_dev);

/* Count only matches whose first edge id lies in [root_begin, root_end)
 * (one shard of the root space; Section 5.3.1 partitions roots by time).
 * per_root_dev, if given, has root_end - root_begin entries. */
tm_status tm_count_roots(tm_graph* g, tm_query* q, int64_t root_begin, int64_t root_end,
                         void* stream, uint64_t* total, uint64_t* per_root_dev);

/* Enumerate matches (Section 2.1 enumeration flavour, with the user-given
 * match limit of Section 4.3).
 *   match_dev : device pointer int32[cap * k]; row j = the k edge ids of one
 *               match in motif-edge order
 *   cap       : rows available
 * Rows are the lexicographically smallest min(cap, total) matches, in
 * lexicographic order of (e_0, ..., e_{k-1}).  *total is always exact.
 * Returns TM_E_TRUNCATED (non-fatal) when total > cap, with *n_written = cap.
 * Synchronises the stream. */
tm_status tm_enumerate(tm_graph* g, tm_query* q, void* stream, int32_t* match_dev, uint64_t cap,
                       uint64_t* n_written, uint64_t* total);

/* Enumerate nq queries together (Section 2.1 enumeration flavour, many
 * queries at once): one multi-query count pass (per-chunk counts of every
 * query), a per-query scan of those counts into row offsets, and one
 * multi-query fill pass that writes each query's rows from the offsets on the
 * device, with a single stream synchronisation at the end.  Queries are grouped
 * by the occupancy their launch shape allows (one persistent launch per group
 * and pass).  Per query j (all arrays have nq entries):
 *   match_devs[j] : device pointer int32[caps[j] * k_j] (may be NULL if caps[j] == 0)
 *   caps[j]       : rows available (host array)
 *   n_written[j], totals[j] : host arrays; receive min(total, cap) and the exact total
 * Rows are as for tm_enumerate (the lexicographically first min(cap, total)).
 *   kernel_ms : host double[2] or NULL; receives the device time of the count
 *               launches and of the fill launches (CUDA events on the stream)
 * Returns TM_E_TRUNCATED (non-fatal) when any query had more matches than its
 * cap, TM_E_INVALID for nq outside [1, 4096] or a query given twice.  Uses each
 * query's own scratch (as tm_enumerate does) and batch buffers cached on the
 * graph by batch shape; calls with the same shape from two host threads are
 * serialised.  On TM_E_TIMEOUT the outputs are untouched but rows may have been
 * written.  Synchronises the stream. */
tm_status tm_enumerate_batch(tm_graph* g, tm_query* const* qs, int nq, void* stream, int32_t* const* match_devs,
                             const uint64_t* caps, uint64_t* n_written, uint64_t* totals, double* kernel_ms);

/* Count nq queries in one persistent launch (replayed from a captured CUDA
 * graph).  totals: host pointer uint64[nq].  Queries may differ in size,
 * shape, delta and constraints.  Synchronises the stream. */
tm_status tm_count_batch(tm_graph* g, tm_query* const* qs, int nq, void* stream, uint64_t* totals);

/* Device timing of this query's search launches.  tm_query_profile(q, 1)
 * makes later tm_count / tm_enumerate calls record CUDA events around the
 * search kernel (count pass) and the enumeration fill kernel on the caller's
 * stream; tm_query_last_ms reads the last call's durations in milliseconds
 * (fill_ms = 0 when the last call had no fill pass).  Only valid after the
 * call has returned. */
tm_status tm_query_profile(tm_query* q, int enable);
tm_status tm_query_last_ms(const tm_query* q, double* search_ms, double* fill_ms);

/* Test hook for the bounded device waits.  kind 1: the next tm_count /
 * tm_count_roots / tm_query_work call on q stages a task-queue slot that no
 * warp ever publishes; the warp that pops it gives up after its ~2 s bounded
 * wait, the kernel finishes normally and the call returns TM_E_TIMEOUT (the
 * CUDA context stays usable).  kind 0 clears a pending fault. */
tm_status tm_query_inject_fault(tm_query* q, int kind);

/* Test hook for out-of-memory handling (failure injected on the host, no
 * GPU fault): the device or pinned-host allocation that this library makes
 * after `after` further successful ones fails as if the device were out of
 * memory, and the call that made it returns TM_E_OOM with its outputs
 * untouched (a served request completes with status TM_E_OOM).  Process-wide;
 * one failure per arming; after < 0 disarms.  Every later call is unaffected. */
tm_status tm_inject_alloc_failure(int64_t after);

/* Number of CUDA kernels (and CUDA-graph replays) this library has launched
 * since it was loaded, over all threads. */
uint64_t tm_kernel_launches(void);

/* Ablation: count with the paper's GPU baseline design (Section 3.2) -- one
 * thread per search tree following Algorithm 1, candidate lists located by
 * binary search at every visit (no cached ranges), structural checks by
 * scanning the motif-to-graph map, no work sharing -- on this library's graph
 * layout.  Same result as tm_count (motifs without anti-edges; TM_E_INVALID
 * otherwise).  kernel_ms (nullable, host) receives the kernel's device time.
 * Synchronises the stream. */
tm_status tm_count_baseline(tm_graph* g, tm_query* q, void* stream, uint64_t* total, double* kernel_ms);

/* Pick tm_tuning for this query's shape by timing candidate settings on the
 * resident graph; the choice is cached per shape in the graph and applied to
 * q.  tuned (nullable, host) receives it. */
tm_status tm_autotune(tm_graph* g, tm_query* q, void* stream, tm_tuning* tuned);

/* Measure the algorithm-independent work counters of a query (host pointer). */
tm_status tm_query_work(tm_graph* g, tm_query* q, void* stream, tm_work* out);

/* Batched count that allocates nothing (the paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at query
 * time -- real-time loops that reserve all of their memory up front, processes
 * under a fixed memory cap or an allocator that forbids cudaMalloc after
 * start-up, plug-ins whose host framework owns every allocation).
 * Same result as tm_count_batch: the same persistent multi-query count kernel,
 * but its scratch (control block, launch records, donated-task queue) lives in
 * one file-scope __device__ array of TM_NOALLOC_SCRATCH_BYTES bytes that every
 * GPU loading this library holds until the process exits; no cudaMalloc,
 * cudaFree or other allocating call is made.
 *   qs, nq     : compiled queries of graph g, 1 <= nq <= TM_NOALLOC_MAX_QUERIES
 *                (TM_E_INVALID beyond that, with a message naming the limit)
 *   totals_dev : device pointer uint64[nq], caller-owned; receives the counts
 * The task queue has TM_NOALLOC_TASKS slots per call: slots are not reused
 * within a call, so once a call has donated that many subtrees, further
 * donations stay with the donating warp (results are unchanged).
 * The launch records are staged in a static host buffer of about 60 KB (not on
 * the caller's stack); the call's own stack use is under 1 KB.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * previous call's contents; each call rewrites and clears what it uses.  Calls
 * that overlap on the GPU (two streams, two host threads) race on the array
 * and must be serialised by the caller.  Synchronises the stream. */
#define TM_NOALLOC_MAX_QUERIES 64
#define TM_NOALLOC_TASKS 4096
#define TM_NOALLOC_SCRATCH_BYTES (320 * 1024)
tm_status tm_count_batch_noalloc(tm_graph* g, tm_query* const* qs, int nq, void* stream, uint64_t* totals_dev);

/* ------------------------------------------------------------- serving --
 * A request loop over one resident graph: submitted queries are admitted
 * while their memory (match buffer + per-request scratch) fits the budget,
 * batched into persistent search launches on several streams, and completed
 * asynchronously.  Requests that arrive while others run are admitted as
 * streams and memory free up (continuous batching).
 *
 * Batches are formed by expected cost: the graph keeps, per motif shape,
 * delta bucket and flavour (count / enumerate), an estimate of the device time
 * one request takes, learnt from the launches every server of the graph has
 * timed.  The oldest admissible request leads each batch; a leader expected
 * to take at least long_ms (or never seen) runs alone, and short requests
 * behind it join while the batch's expected time stays within batch_ms.
 * Short batches run on high-priority streams. */
typedef struct {
    uint64_t mem_budget_bytes;   /* device bytes for match buffers + scratch (0 = 4 GiB) */
    int32_t streams;             /* concurrent batches in flight (0 = 2) */
    int32_t max_batch;           /* queries per launched batch (0 = 16) */
    int32_t grid_pct;            /* share of the full persistent grid each launch uses, 1..100 (0 = 100) */
    int32_t policy;              /* 0 = batches by expected cost (above); 1 = arrival order, any mix */
    double long_ms;              /* expected device ms from which a request runs alone (0 = 1.0) */
    double batch_ms;             /* expected device ms a batch of short requests may hold (0 = 2.0) */
} tm_serve_cfg;

typedef struct {
    tm_status status;            /* TM_OK or TM_E_TRUNCATED on success */
    uint64_t total;              /* exact match count */
    uint64_t n_written;          /* rows in matches (enumerate requests) */
    const int32_t* matches_dev;  /* device pointer, int32[n_written * k]; valid until release */
    int32_t k;
    double submit_to_done_ms;    /* host wall time from submit to completion */
} tm_result;

tm_status tm_serve_start(tm_graph* g, const tm_serve_cfg* cfg, tm_server** out);

/* Queue a request.  The query must stay alive until its result is released;
 * enumerate = 1 requests up to cap matches (cap >= 1).  *ticket identifies it.
 * TM_E_ADMISSION if the request alone exceeds the memory budget.  Thread-safe. */
tm_status tm_serve_submit(tm_server* s, tm_query* q, int enumerate, uint64_t cap, uint64_t* ticket);

/* TM_E_BUSY while the request runs; TM_OK with *out filled when finished.
 * Thread-safe. */
tm_status tm_serve_poll(tm_server* s, uint64_t ticket, tm_result* out);

/* Block until the request finishes (bounded by timeout_ms; TM_E_TIMEOUT after). */
tm_status tm_serve_wait(tm_server* s, uint64_t ticket, int64_t timeout_ms, tm_result* out);

/* Free a finished request's match buffer and bookkeeping. */
tm_status tm_result_release(tm_server* s, uint64_t ticket);

/* Drain in-flight work, stop the loop and free the server. */
tm_status tm_serve_stop(tm_server* s);

/* Static description of a status code. */
const char* tm_status_str(tm_status s);

/* Message of the last error on the calling thread ("" if none). */
const char* tm_last_error(void);

/* Load-balancing diagnostics of the last count-mode search launch made by the
 * calling thread (tm_count, tm_count_roots, tm_query_work, the count pass of
 * tm_enumerate, tm_count_batch, tm_count_batch_noalloc).  Both pointers are
 * host pointers and may be NULL.
 *   donated  : subtrees handed to idle warps through the device task queue
 *              (the sub-tree-level parallelism of Section 5.2)
 *   reserved : task slots the launch's donors reserved; a value above the
 *              queue's capacity means some donations found it full and their
 *              work stayed with the donating warp */
tm_status tm_last_search_stats(uint64_t* donated, uint64_t* reserved);

#ifdef __cplusplus
}
#endif
#endif
