/*
 * CPU ORACLE for temporal motif mining -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded, deliberately slow.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load this file's library; the CUDA
 * library never links or calls it, and the two share no code or headers.
 *
 * What it computes (paper Section 2.1, "Problem definition"):
 *   edges are ordered by (t, input index); edge id = rank in that order
 *   (the paper assumes a temporally ordered edge list).  A match of a motif
 *   with k edges (x_i -> y_i), i = 0..k-1, is a k-tuple of edge ids
 *   (e_0, ..., e_{k-1}) with
 *     1. t(e_0) < t(e_1) < ... < t(e_{k-1})           (delta-temporal motif)
 *     2. t(e_{k-1}) - t(e_0) <= delta                  (delta-temporal motif)
 *     3. t(e_{i+1}) - t(e_i) <= gap_i                  (fine-grained motif)
 *     4. an injective map phi: motif nodes -> graph nodes with
 *        src(e_i) = phi(x_i), dst(e_i) = phi(y_i)     (isomorphism semantics)
 *     5. label equalities on edges / nodes where given (Section 5.4.1)
 *     6. for every temporal anti-edge (x', y', delta') attached to motif edge i:
 *        no graph edge other than e_i goes from phi(x') to phi(y') at a time in
 *        the closed interval [t(e_i), t(e_i) + delta']       (Section 2.1)
 *
 * How: the chronological depth-first search of Algorithm 1 (Section 2.2,
 * Mackey et al.), with its execution context MapMG / MapGM / eCount / eStack,
 * its four candidate-list cases of GetCandidateEdgeList, the StructConstraints
 * node-consistency test, and the book-keeping update / rollback.  Readings
 * where the printed algorithm is glitched or silent:
 *   - node id 0 is a valid mapping (the printed "u_G > 0" means "mapped");
 *   - the time limit t' = t(root) + delta is set when the root is bound and
 *     is inclusive (the definition's "<= delta" wins over the listing's "<");
 *     the sum saturates at INT64_MAX;
 *   - candidates must be strictly later than the previous level's edge, in
 *     time (equal timestamps never appear in one match);
 *   - a graph self-loop never maps to a motif edge between distinct motif nodes
 *     (injectivity); motifs with self-loops are rejected;
 *   - when both endpoints are mapped the candidate list is N_out(phi(x)) if
 *     deg_out(phi(x)) <= deg_in(phi(y)), else N_in(phi(y)) (the listing leaves
 *     the choice open; the smaller list is the cheap one);
 *   - the fine-grained limit for edge i is t(e_{i-1}) + gap_{i-1}, saturating.
 * Algorithm 1 has no anti-edges; here they are tested on each complete match,
 * straight from their definition, before the match is counted.
 * Iterating every candidate list in ascending edge id makes the enumeration
 * come out in lexicographic order of (e_0, ..., e_{k-1}).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

struct or_graph {
    int64_t n, m;
    int32_t* src;      /* by edge id */
    int32_t* dst;
    int64_t* t;
    uint8_t* elabel;   /* nullable */
    uint8_t* nlabel;   /* nullable */
    int64_t* perm;     /* edge id -> input index */
    int64_t* out_off;  /* n+1 */
    int64_t* out_eid;  /* edge ids, ascending within a node */
    int64_t* in_off;
    int64_t* in_eid;
};

/* ------------------------------------------------------------ graph build */

static const int64_t* g_sort_t;
static int cmp_time_then_index(const void* a, const void* b) {
    int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
    if (g_sort_t[ia] < g_sort_t[ib]) return -1;
    if (g_sort_t[ia] > g_sort_t[ib]) return 1;
    return (ia > ib) - (ia < ib);
}

or_graph* or_graph_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const int64_t* t, const uint8_t* elabel, const uint8_t* nlabel) {
    if (n < 0 || m < 0) return NULL;
    for (int64_t i = 0; i < m; ++i)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || t[i] < 0) return NULL;
    or_graph* g = (or_graph*)calloc(1, sizeof(or_graph));
    g->n = n; g->m = m;
    size_t mm = (size_t)(m > 0 ? m : 1), nn = (size_t)(n > 0 ? n : 1);
    g->perm = (int64_t*)malloc(mm * sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) g->perm[i] = i;
    g_sort_t = t;
    qsort(g->perm, (size_t)m, sizeof(int64_t), cmp_time_then_index);
    g->src = (int32_t*)malloc(mm * sizeof(int32_t));
    g->dst = (int32_t*)malloc(mm * sizeof(int32_t));
    g->t = (int64_t*)malloc(mm * sizeof(int64_t));
    if (elabel) g->elabel = (uint8_t*)malloc(mm);
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = g->perm[e];
        g->src[e] = src[i]; g->dst[e] = dst[i]; g->t[e] = t[i];
        if (elabel) g->elabel[e] = elabel[i];
    }
    if (nlabel) { g->nlabel = (uint8_t*)malloc(nn); memcpy(g->nlabel, nlabel, (size_t)n); }
    /* CSR by counting sort in edge-id order: each node's list ascends in id */
    g->out_off = (int64_t*)calloc(nn + 1, sizeof(int64_t));
    g->in_off = (int64_t*)calloc(nn + 1, sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) { g->out_off[g->src[e] + 1]++; g->in_off[g->dst[e] + 1]++; }
    for (int64_t v = 0; v < n; ++v) { g->out_off[v + 1] += g->out_off[v]; g->in_off[v + 1] += g->in_off[v]; }
    g->out_eid = (int64_t*)malloc(mm * sizeof(int64_t));
    g->in_eid = (int64_t*)malloc(mm * sizeof(int64_t));
    int64_t* fo = (int64_t*)malloc(nn * sizeof(int64_t));
    int64_t* fi = (int64_t*)malloc(nn * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) { fo[v] = g->out_off[v]; fi[v] = g->in_off[v]; }
    for (int64_t e = 0; e < m; ++e) { g->out_eid[fo[g->src[e]]++] = e; g->in_eid[fi[g->dst[e]]++] = e; }
    free(fo); free(fi);
    return g;
}

void or_graph_free(or_graph* g) {
    if (!g) return;
    free(g->src); free(g->dst); free(g->t); free(g->elabel); free(g->nlabel); free(g->perm);
    free(g->out_off); free(g->out_eid); free(g->in_off); free(g->in_eid);
    free(g);
}

int64_t or_graph_edges(const or_graph* g) { return g->m; }

void or_graph_sorted(const or_graph* g, int32_t* src, int32_t* dst, int64_t* t, int64_t* perm) {
    for (int64_t e = 0; e < g->m; ++e) {
        if (src) src[e] = g->src[e];
        if (dst) dst[e] = g->dst[e];
        if (t) t[e] = g->t[e];
        if (perm) perm[e] = g->perm[e];
    }
}

/* ----------------------------------------------------------------- search */

typedef struct {
    const or_graph* g;
    const or_motif* q;
    /* Algorithm 1 execution context */
    int64_t map_mg[OR_MAX_NODES];   /* motif node -> graph node, -1 unmapped */
    int32_t* map_gm;                /* graph node -> motif node, -1 unmapped */
    int32_t* ecount;                /* graph node -> mapped edges touching it */
    int64_t estack[OR_MAX_EDGES];
    int64_t t_limit;                /* t' */
    /* outputs */
    uint64_t count;
    uint64_t cap, written;
    int32_t* out;
    or_work* work;
} ctx_t;

static int64_t sat_add(int64_t a, int64_t b) {
    if (b > 0 && a > INT64_MAX - b) return INT64_MAX;
    return a + b;
}

/* UpdateDataStructures: map both endpoints, count mapped edges per node */
static void update(ctx_t* c, int level, int64_t e) {
    int32_t u = c->g->src[e], v = c->g->dst[e];
    int xm = c->q->esrc[level], ym = c->q->edst[level];
    c->map_mg[xm] = u; c->map_mg[ym] = v;
    c->map_gm[u] = xm; c->map_gm[v] = ym;
    c->ecount[u] += 1; c->ecount[v] += 1;
    c->estack[level] = e;
}

/* RollbackDataStructures: free a node when its last mapped edge is removed */
static void rollback(ctx_t* c, int level) {
    int64_t e = c->estack[level];
    int32_t u = c->g->src[e], v = c->g->dst[e];
    c->ecount[u] -= 1; c->ecount[v] -= 1;
    if (c->ecount[u] == 0) { c->map_mg[c->map_gm[u]] = -1; c->map_gm[u] = -1; }
    if (c->ecount[v] == 0) { c->map_mg[c->map_gm[v]] = -1; c->map_gm[v] = -1; }
}

/* StructConstraints plus the label tests of Section 5.4.1 */
static int consistent(const ctx_t* c, int level, int64_t e, int64_t uG, int64_t vG) {
    const or_graph* g = c->g;
    int32_t u2 = g->src[e], v2 = g->dst[e];
    int xm = c->q->esrc[level], ym = c->q->edst[level];
    int u_ok = (uG == u2) || (uG < 0 && c->map_gm[u2] < 0);
    int v_ok = (vG == v2) || (vG < 0 && c->map_gm[v2] < 0);
    if (!u_ok || !v_ok) return 0;
    /* two unmapped motif nodes may not land on the same graph node */
    if (u2 == v2) return 0;
    if (c->q->elabel[level] >= 0 && (!g->elabel || g->elabel[e] != (uint8_t)c->q->elabel[level])) return 0;
    if (uG < 0 && c->q->nlabel[xm] >= 0 && (!g->nlabel || g->nlabel[u2] != (uint8_t)c->q->nlabel[xm])) return 0;
    if (vG < 0 && c->q->nlabel[ym] >= 0 && (!g->nlabel || g->nlabel[v2] != (uint8_t)c->q->nlabel[ym])) return 0;
    return 1;
}

/* first position in list[lo, hi) whose edge time is > tprev */
static int64_t upper_by_time(const or_graph* g, const int64_t* list, int64_t lo, int64_t hi,
                             int64_t tprev, or_work* w) {
    int64_t a = lo, b = hi;
    while (a < b) {
        int64_t mid = a + (b - a) / 2;
        int64_t e = list ? list[mid] : mid;
        if (w) w->probes++;
        if (g->t[e] <= tprev) a = mid + 1; else b = mid;
    }
    return a;
}

/* condition 6: is some edge other than e_i from phi(x') to phi(y') inside
 * [t(e_i), t(e_i) + delta'] for an anti-edge (x', y', delta') attached to e_i? */
static int anti_edge_present(const ctx_t* c, int a) {
    const or_graph* g = c->g;
    const or_motif* q = c->q;
    int64_t ei = c->estack[q->anti_edge[a]];
    int64_t u = c->map_mg[q->anti_src[a]], v = c->map_mg[q->anti_dst[a]];
    int64_t t0 = g->t[ei], t1 = sat_add(t0, q->anti_delta[a]);
    for (int64_t p = g->out_off[u]; p < g->out_off[u + 1]; ++p) {
        int64_t e = g->out_eid[p];
        if (e == ei || g->dst[e] != v) continue;
        if (g->t[e] >= t0 && g->t[e] <= t1) return 1;
    }
    return 0;
}

static void emit(ctx_t* c) {
    int k = c->q->k;
    for (int a = 0; a < c->q->n_anti; ++a)
        if (anti_edge_present(c, a)) return;
    if (c->out && c->written < c->cap) {
        for (int i = 0; i < k; ++i) c->out[c->written * (uint64_t)k + (uint64_t)i] = (int32_t)c->estack[i];
        c->written++;
    }
    c->count++;
}

static void dfs(ctx_t* c, int level) {
    const or_graph* g = c->g;
    const or_motif* q = c->q;
    if (level == q->k) { emit(c); return; }
    int xm = q->esrc[level], ym = q->edst[level];
    int64_t uG = c->map_mg[xm], vG = c->map_mg[ym];
    int64_t tprev = g->t[c->estack[level - 1]];
    int64_t lim = c->t_limit;
    int64_t glim = sat_add(tprev, q->gap[level - 1]);
    if (glim < lim) lim = glim;
    /* GetCandidateEdgeList */
    const int64_t* list; int64_t lo, hi;
    if (uG >= 0 && vG >= 0) {
        int64_t dout = g->out_off[uG + 1] - g->out_off[uG];
        int64_t din = g->in_off[vG + 1] - g->in_off[vG];
        if (dout <= din) { list = g->out_eid; lo = g->out_off[uG]; hi = g->out_off[uG + 1]; }
        else { list = g->in_eid; lo = g->in_off[vG]; hi = g->in_off[vG + 1]; }
    } else if (uG >= 0) {
        list = g->out_eid; lo = g->out_off[uG]; hi = g->out_off[uG + 1];
    } else if (vG >= 0) {
        list = g->in_eid; lo = g->in_off[vG]; hi = g->in_off[vG + 1];
    } else {
        list = NULL; lo = 0; hi = g->m;           /* all edges of E_G */
    }
    if (c->work) c->work->nodes[level]++;
    int64_t p = upper_by_time(g, list, lo, hi, tprev, c->work);
    for (; p < hi; ++p) {
        int64_t e = list ? list[p] : p;
        if (g->t[e] > lim) break;
        if (c->work) c->work->entries[level]++;
        if (!consistent(c, level, e, uG, vG)) continue;
        update(c, level, e);
        dfs(c, level + 1);
        rollback(c, level);
    }
}

static int check_motif(const or_motif* q) {
    if (q->k < 1 || q->k > OR_MAX_EDGES || q->n_nodes < 2 || q->n_nodes > OR_MAX_NODES) return 0;
    if (q->delta < 0) return 0;
    for (int i = 0; i < q->k; ++i) {
        if (q->esrc[i] >= q->n_nodes || q->edst[i] >= q->n_nodes) return 0;
        if (q->esrc[i] == q->edst[i]) return 0;
    }
    for (int i = 0; i + 1 < q->k; ++i) if (q->gap[i] < 0) return 0;
    if (q->n_anti < 0 || q->n_anti > OR_MAX_ANTI) return 0;
    for (int a = 0; a < q->n_anti; ++a) {
        if (q->anti_src[a] >= q->n_nodes || q->anti_dst[a] >= q->n_nodes) return 0;
        int used_x = 0, used_y = 0;   /* both ends must be nodes some motif edge binds */
        for (int i = 0; i < q->k; ++i) {
            used_x |= q->esrc[i] == q->anti_src[a] || q->edst[i] == q->anti_src[a];
            used_y |= q->esrc[i] == q->anti_dst[a] || q->edst[i] == q->anti_dst[a];
        }
        if (!used_x || !used_y) return 0;
        if (q->anti_src[a] == q->anti_dst[a] || q->anti_edge[a] >= q->k || q->anti_delta[a] < 0) return 0;
    }
    return 1;
}

static int search(const or_graph* g, const or_motif* q, int64_t r0, int64_t r1,
                  uint64_t* total, uint64_t* per_root, int32_t* out, uint64_t cap,
                  uint64_t* n_written, or_work* work) {
    if (!check_motif(q)) return 1;
    if (r0 < 0) r0 = 0;
    if (r1 > g->m) r1 = g->m;
    ctx_t c;
    memset(&c, 0, sizeof c);
    c.g = g; c.q = q; c.out = out; c.cap = cap; c.work = work;
    size_t nn = (size_t)(g->n > 0 ? g->n : 1);
    c.map_gm = (int32_t*)malloc(nn * sizeof(int32_t));
    c.ecount = (int32_t*)calloc(nn, sizeof(int32_t));
    for (int64_t v = 0; v < g->n; ++v) c.map_gm[v] = -1;
    for (int i = 0; i < OR_MAX_NODES; ++i) c.map_mg[i] = -1;
    if (work) work->roots += (uint64_t)(r1 > r0 ? r1 - r0 : 0);
    for (int64_t r = r0; r < r1; ++r) {
        uint64_t before = c.count;
        if (consistent(&c, 0, r, -1, -1)) {
            update(&c, 0, r);
            c.t_limit = sat_add(g->t[r], q->delta);
            dfs(&c, 1);
            rollback(&c, 0);
        }
        if (per_root) per_root[r - r0] = c.count - before;
    }
    if (total) *total = c.count;
    if (n_written) *n_written = c.written;
    if (work) work->matches += c.count;
    free(c.map_gm); free(c.ecount);
    return 0;
}

int or_count(const or_graph* g, const or_motif* q, int64_t root_begin, int64_t root_end,
             uint64_t* total, uint64_t* per_root, or_work* work) {
    return search(g, q, root_begin, root_end, total, per_root, NULL, 0, NULL, work);
}

int or_enumerate(const or_graph* g, const or_motif* q, int32_t* out, uint64_t cap,
                 uint64_t* n_written, uint64_t* total) {
    return search(g, q, 0, g->m, total, NULL, out, cap, n_written, NULL);
}

int or_enumerate_roots(const or_graph* g, const or_motif* q, int64_t root_begin, int64_t root_end,
                       int32_t* out, uint64_t cap, uint64_t* n_written, uint64_t* total) {
    return search(g, q, root_begin, root_end, total, NULL, out, cap, n_written, NULL);
}
