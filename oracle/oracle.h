/*
 * CPU oracle for temporal motif mining -- test infrastructure only.
 * Private to oracle/: the CUDA library has its own, unrelated header.
 * See oracle.c for the definition it follows (paper Section 2.1, Algorithm 1).
 */
#ifndef TM_ORACLE_H
#define TM_ORACLE_H
#include <stdint.h>

#define OR_MAX_EDGES 8
#define OR_MAX_NODES 8
#define OR_MAX_ANTI 4

typedef struct {
    int32_t k;                     /* motif edges, in temporal order */
    int32_t n_nodes;               /* motif nodes 0..n_nodes-1 */
    uint8_t esrc[OR_MAX_EDGES];    /* x_i */
    uint8_t edst[OR_MAX_EDGES];    /* y_i */
    int64_t delta;                 /* first-to-last span bound (inclusive) */
    int64_t gap[OR_MAX_EDGES - 1]; /* t_{i+1} - t_i bound, INT64_MAX = none */
    int16_t elabel[OR_MAX_EDGES];  /* -1 = any */
    int16_t nlabel[OR_MAX_NODES];  /* -1 = any */
    int32_t n_anti;                /* temporal anti-edges (Section 2.1) */
    uint8_t anti_src[OR_MAX_ANTI]; /* motif node of the absent edge's source */
    uint8_t anti_dst[OR_MAX_ANTI];
    uint8_t anti_edge[OR_MAX_ANTI];/* motif edge it is attached to */
    int64_t anti_delta[OR_MAX_ANTI];
} or_motif;

typedef struct {
    uint64_t roots;                     /* root edges tried */
    uint64_t nodes[OR_MAX_EDGES];       /* [i]: partial matches of i edges that located a window for edge i */
    uint64_t entries[OR_MAX_EDGES];     /* [i]: window entries in (t_prev, limit] scanned for edge i */
    uint64_t probes;                    /* binary-search probes */
    uint64_t matches;
} or_work;

typedef struct or_graph or_graph;

or_graph* or_graph_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int64_t* t, const uint8_t* elabel, const uint8_t* nlabel);
void or_graph_free(or_graph* g);
int64_t or_graph_edges(const or_graph* g);
void or_graph_sorted(const or_graph* g, int32_t* src, int32_t* dst, int64_t* t, int64_t* perm);

/* per_root (nullable) has root_end - root_begin entries */
int or_count(const or_graph* g, const or_motif* q, int64_t root_begin, int64_t root_end,
             uint64_t* total, uint64_t* per_root, or_work* work);
/* first min(cap, total) matches in lexicographic order, k int32 edge ids each */
int or_enumerate(const or_graph* g, const or_motif* q, int32_t* out, uint64_t cap,
                 uint64_t* n_written, uint64_t* total);
/* the same over the matches whose first edge id lies in [root_begin, root_end) */
int or_enumerate_roots(const or_graph* g, const or_motif* q, int64_t root_begin, int64_t root_end,
                       int32_t* out, uint64_t cap, uint64_t* n_written, uint64_t* total);
#endif
