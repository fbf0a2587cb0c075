// Ablation: the paper's GPU baseline design (Section 3.2), rebuilt on this
// library's graph layout so that the search-kernel design can be compared with
// it on the same GB300 and the same inputs.
//
// One thread expands one search tree (root edge), depth first, exactly in the
// order of Algorithm 1: at each level the candidate list is located by binary
// search for t > t_prev in the mapped endpoint's time-ordered list (or the
// whole edge list); a candidate is accepted after the structural test
// (consistency with the mapped nodes, found by scanning the motif-to-graph map
// MapMG -- the baseline keeps no graph-to-motif map), the time limits and the
// labels.  On backtrack the list is located again by binary search (the
// baseline caches no candidate ranges).  Per-thread work is whatever its tree
// holds: no sharing between threads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "tm_internal.cuh"

namespace tmg {

namespace {

__device__ __forceinline__ int64_t bl_sat_add(int64_t a, int64_t b) {
    return (b > 0 && a > INT64_MAX - b) ? INT64_MAX : a + b;
}

__device__ __forceinline__ uint32_t bl_upper(const int64_t* __restrict__ t, uint32_t lo, uint32_t hi, int64_t x) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(t + mid) <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct BaselineMotif {
    int32_t k, n_nodes;
    uint8_t esrc[TM_MAX_EDGES], edst[TM_MAX_EDGES];
    int64_t delta;
    int64_t gap[TM_MAX_EDGES - 1];
    int16_t elabel[TM_MAX_EDGES], nlabel[TM_MAX_NODES];
};

__global__ void baseline_kernel(const __grid_constant__ GraphView g, const __grid_constant__ BaselineMotif q,
                                unsigned long long* total) {
    unsigned long long found = 0;
    const int k = q.k;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < g.m; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t map[TM_MAX_NODES];            // MapMG: motif node -> graph node, -1 unmapped
        int owner[TM_MAX_NODES];              // level that mapped the motif node
        int32_t stack_e[TM_MAX_EDGES];        // eStack: matched edge per level
        uint32_t cur[TM_MAX_EDGES];           // candidate cursor per level (a list position)
        for (int j = 0; j < TM_MAX_NODES; ++j) { map[j] = -1; owner[j] = -1; }
        // level 0: the root
        int32_t s = g.src[r], d = g.dst[r];
        if (s == d) continue;
        if (q.elabel[0] >= 0 && g.elabel[r] != (uint8_t)q.elabel[0]) continue;
        if (q.nlabel[q.esrc[0]] >= 0 && g.nlabel[s] != (uint8_t)q.nlabel[q.esrc[0]]) continue;
        if (q.nlabel[q.edst[0]] >= 0 && g.nlabel[d] != (uint8_t)q.nlabel[q.edst[0]]) continue;
        if (k == 1) { ++found; continue; }
        map[q.esrc[0]] = s; owner[q.esrc[0]] = 0;
        map[q.edst[0]] = d; owner[q.edst[0]] = 0;
        stack_e[0] = (int32_t)r;
        const int64_t tlim = bl_sat_add(g.t[r], q.delta);
        int lvl = 1;
        bool fresh = true;          // entering lvl for the first time (cursor at list start)
        while (lvl >= 1) {
            // RollbackDataStructures: forget what this level mapped for its previous candidate
            for (int j = 0; j < q.n_nodes; ++j)
                if (owner[j] == lvl) { map[j] = -1; owner[j] = -1; }
            const int x = q.esrc[lvl], y = q.edst[lvl];
            const int32_t uG = map[x], vG = map[y];
            const int64_t tprev = g.t[stack_e[lvl - 1]];
            const int64_t lim = min(tlim, bl_sat_add(tprev, q.gap[lvl - 1]));
            // GetCandidateEdgeList, located anew (binary search) every time
            int dir;
            uint32_t lo, hi;
            const int64_t* tarr;
            if (uG >= 0 && vG >= 0) {
                uint32_t du = g.off[0][uG + 1] - g.off[0][uG], dv = g.off[1][vG + 1] - g.off[1][vG];
                if (du <= dv) { dir = 0; lo = g.off[0][uG]; hi = g.off[0][uG + 1]; }
                else { dir = 1; lo = g.off[1][vG]; hi = g.off[1][vG + 1]; }
                tarr = g.at[dir];
            } else if (uG >= 0) {
                dir = 0; lo = g.off[0][uG]; hi = g.off[0][uG + 1]; tarr = g.at[0];
            } else if (vG >= 0) {
                dir = 1; lo = g.off[1][vG]; hi = g.off[1][vG + 1]; tarr = g.at[1];
            } else {
                dir = 2; lo = 0; hi = (uint32_t)g.m; tarr = g.t;
            }
            uint32_t p = bl_upper(tarr, lo, hi, tprev);
            if (!fresh) p = max(p, cur[lvl] + 1);      // continue after the candidate just explored
            bool advanced = false;
            for (; p < hi; ++p) {
                const int64_t te = __ldg(tarr + p);
                if (te > lim) break;
                int32_t e, us, vs;
                if (dir == 2) { e = (int32_t)p; us = g.src[p]; vs = g.dst[p]; }
                else {
                    e = g.aeid[dir][p];
                    int32_t nb = g.anbr[dir][p];
                    us = dir == 0 ? uG : nb;
                    vs = dir == 0 ? nb : vG;
                }
                if (us == vs) continue;
                // StructConstraints by scanning MapMG
                bool ok = true;
                if (uG >= 0) ok &= us == uG;
                if (vG >= 0) ok &= vs == vG;
                for (int j = 0; j < q.n_nodes && ok; ++j) {
                    if (map[j] < 0) continue;
                    if (uG < 0 && map[j] == us) ok = false;
                    if (vG < 0 && map[j] == vs) ok = false;
                }
                if (!ok) continue;
                if (q.elabel[lvl] >= 0 && g.elabel[e] != (uint8_t)q.elabel[lvl]) continue;
                if (uG < 0 && q.nlabel[x] >= 0 && g.nlabel[us] != (uint8_t)q.nlabel[x]) continue;
                if (vG < 0 && q.nlabel[y] >= 0 && g.nlabel[vs] != (uint8_t)q.nlabel[y]) continue;
                if (lvl == k - 1) { ++found; continue; }
                // NextLevel: map, push, descend
                cur[lvl] = p;
                stack_e[lvl] = e;
                if (uG < 0) { map[x] = us; owner[x] = lvl; }
                if (vG < 0) { map[y] = vs; owner[y] = lvl; }
                advanced = true;
                break;
            }
            if (advanced) { ++lvl; fresh = true; }
            else { --lvl; fresh = false; }
        }
    }
    for (int o = 16; o > 0; o >>= 1) found += __shfl_down_sync(0xffffffffu, found, o);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(total, found);
}

}  // namespace

}  // namespace tmg

using namespace tmg;

extern "C" tm_status tm_count_baseline(tm_graph* g, tm_query* q, void* stream, uint64_t* total, double* kernel_ms) {
    if (!g || !q || !total || query_graph(q) != g) { set_error("null or mismatched argument"); return TM_E_INVALID; }
    const tm_motif* m = query_motif(q);
    if (m->n_anti > 0) { set_error("the baseline kernel has no anti-edges"); return TM_E_INVALID; }
    TM_ENTER(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    BaselineMotif bm;
    memset(&bm, 0, sizeof bm);
    bm.k = m->k; bm.n_nodes = m->n_nodes; bm.delta = m->delta;
    for (int i = 0; i < TM_MAX_EDGES; ++i) { bm.esrc[i] = m->esrc[i]; bm.edst[i] = m->edst[i]; bm.elabel[i] = m->elabel[i]; }
    for (int i = 0; i < TM_MAX_EDGES - 1; ++i) bm.gap[i] = m->gap[i];
    for (int j = 0; j < TM_MAX_NODES; ++j) bm.nlabel[j] = m->nlabel[j];
    unsigned long long* d_total = nullptr;
    TM_CUDA(dev_malloc_async((void**)&d_total, sizeof(unsigned long long), st));
    TM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), st));
    cudaEvent_t e0, e1;
    TM_CUDA(cudaEventCreate(&e0));
    TM_CUDA(cudaEventCreate(&e1));
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, baseline_kernel, 256, 0);
    int grid = std::max(1, blocks) * g->num_sms;
    TM_CUDA(cudaEventRecord(e0, st));
    if (g->v.m > 0) {
        baseline_kernel<<<grid, 256, 0, st>>>(g->v, bm, d_total);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
    }
    TM_CUDA(cudaEventRecord(e1, st));
    unsigned long long h = 0;
    TM_CUDA(cudaMemcpyAsync(&h, d_total, sizeof h, cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaFreeAsync(d_total, st));
    TM_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *total = h;
    if (kernel_ms) *kernel_ms = ms;
    return TM_OK;
}
