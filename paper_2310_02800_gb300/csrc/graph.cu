// Graph ingest (paper Section 4.2 data loader, Section 2.2 layout), on the GPU:
//   1. validate ids / times and find the time range (one reduction kernel)
//   2. stable radix sort by time with the input index as payload -> edge ids
//      (skipped when the input is already in time order)
//   3. gather the edge columns into edge-id order
//   4. per direction: degree histogram + exclusive scan -> list offsets;
//      stable radix sort of (endpoint, edge id) -> lists in time order;
//      gather (t, neighbour) columns for the lists.
//   5. out-lists re-ordered by (neighbour, time): closing-edge lookups
//   6. successor index: per edge, the first later position in its four lists
#include <cuda_runtime.h>

#include <algorithm>

#include "tm_internal.cuh"

namespace tmg {

namespace {

struct Check {
    unsigned long long tmin, tmax;
    unsigned long long bad;       // count of out-of-range ids / negative times
    unsigned long long descents;  // count of t[i] > t[i+1]
};

__global__ void check_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                             const int64_t* __restrict__ t, int64_t m, int64_t n, Check* out) {
    unsigned long long tmin = ~0ULL, tmax = 0, bad = 0, desc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = src[i], d = dst[i];
        int64_t ti = t[i];
        if (s < 0 || s >= n || d < 0 || d >= n || ti < 0) bad++;
        unsigned long long u = (unsigned long long)(ti < 0 ? 0 : ti);
        tmin = min(tmin, u);
        tmax = max(tmax, u);
        if (i + 1 < m && t[i + 1] < ti) desc++;
    }
    for (int d = 16; d > 0; d >>= 1) {
        tmin = min(tmin, __shfl_down_sync(0xffffffffu, tmin, d));
        tmax = max(tmax, __shfl_down_sync(0xffffffffu, tmax, d));
        bad += __shfl_down_sync(0xffffffffu, bad, d);
        desc += __shfl_down_sync(0xffffffffu, desc, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&out->tmin, tmin);
        atomicMax(&out->tmax, tmax);
        if (bad) atomicAdd(&out->bad, bad);
        if (desc) atomicAdd(&out->descents, desc);
    }
}

__global__ void time_keys_kernel(const int64_t* __restrict__ t, int64_t m, unsigned long long tmin,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = (uint64_t)t[i] - tmin;
        vals[i] = (uint32_t)i;
    }
}

__global__ void iota_kernel(uint32_t* __restrict__ v, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

__global__ void gather_edges_kernel(const uint32_t* __restrict__ perm, int64_t m, const int32_t* __restrict__ src,
                                    const int32_t* __restrict__ dst, const int64_t* __restrict__ t,
                                    const uint8_t* __restrict__ el, int32_t* __restrict__ src_o,
                                    int32_t* __restrict__ dst_o, int64_t* __restrict__ t_o, uint8_t* __restrict__ el_o,
                                    int32_t* __restrict__ perm_o) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t i = perm[e];
        src_o[e] = src[i];
        dst_o[e] = dst[i];
        t_o[e] = t[i];
        if (el) el_o[e] = el[i];
        perm_o[e] = (int32_t)i;
    }
}

// Degree histogram.  Lanes of a warp holding the same node add once for the
// group: on power-law inputs a hub takes a large share of all endpoints, and
// one atomic per edge on its counter serialises.  blockDim is a multiple of 32.
__global__ void degree_kernel(const int32_t* __restrict__ node, int64_t m, unsigned long long* __restrict__ deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const int64_t e = base + threadIdx.x;
        const unsigned act = __ballot_sync(0xffffffffu, e < m);
        if (e >= m) continue;
        const int32_t v = node[e];
        const unsigned grp = __match_any_sync(act, v);
        if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&deg[v], (unsigned long long)__popc(grp));
    }
}

__global__ void node_keys_kernel(const int32_t* __restrict__ node, int64_t m, uint32_t* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        keys[e] = (uint32_t)node[e];
        vals[e] = (uint32_t)e;
    }
}

__global__ void offsets_kernel(const unsigned long long* __restrict__ off64, int64_t n1, uint32_t* __restrict__ off) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
        off[i] = (uint32_t)off64[i];
}

__global__ void list_columns_kernel(const uint32_t* __restrict__ eids, int64_t m, const int64_t* __restrict__ t,
                                    const int32_t* __restrict__ other, int64_t* __restrict__ at,
                                    int32_t* __restrict__ anbr, int32_t* __restrict__ aeid,
                                    uint32_t* __restrict__ pos_of_edge) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = eids[i];
        at[i] = t[e];
        anbr[i] = other[e];
        aeid[i] = (int32_t)e;
        pos_of_edge[e] = (uint32_t)i;
    }
}

// Successor index by list position (see GraphView::pnx): the words of the
// edge at each list position.
__global__ void successor_by_position_kernel(int64_t m, const int32_t* __restrict__ aeid_out,
                                             const int32_t* __restrict__ aeid_in, const uint2* __restrict__ so_src,
                                             const uint2* __restrict__ so_dst, const uint2* __restrict__ si_dst,
                                             const uint2* __restrict__ si_src, uint2* __restrict__ p_out_same,
                                             uint2* __restrict__ p_out_dst, uint2* __restrict__ p_in_same,
                                             uint2* __restrict__ p_in_src) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t eo = aeid_out[i], ei = aeid_in[i];
        p_out_same[i] = so_src[eo];
        p_out_dst[i] = so_dst[eo];
        p_in_same[i] = si_dst[ei];
        p_in_src[i] = si_src[ei];
    }
}

__global__ void keys_by_perm_kernel(const int32_t* __restrict__ node, const uint32_t* __restrict__ perm, int64_t m,
                                    uint32_t* __restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)node[perm[i]];
}

__global__ void pair_columns_kernel(const uint32_t* __restrict__ eids, int64_t m, const int64_t* __restrict__ t,
                                    const int32_t* __restrict__ dst, int32_t* __restrict__ pnbr,
                                    int64_t* __restrict__ pt, int32_t* __restrict__ peid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = eids[i];
        pnbr[i] = dst[e];
        pt[i] = t[e];
        peid[i] = (int32_t)e;
    }
}

// first index in [lo, hi) with t[idx] > x
__device__ __forceinline__ uint32_t first_later(const int64_t* __restrict__ t, uint32_t lo, uint32_t hi, int64_t x) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (t[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first index in [beg, hi) with t[idx] > x, searching outward from beg
__device__ __forceinline__ uint32_t first_later_from(const int64_t* __restrict__ t, uint32_t beg, uint32_t hi,
                                                     int64_t x) {
    uint32_t a = beg, b = hi, step = 1;
    while (true) {
        uint32_t probe = a + step - 1;
        if (probe >= hi) { b = hi; break; }
        if (t[probe] > x) { b = probe; break; }
        a = probe + 1;
        step <<= 1;
    }
    return first_later(t, a, b, x);
}

// Successor word for the first entry of a list [.., hi) at position p that is
// later than time te: {p, gap to its time} (SUCC_END when p == hi).
__device__ __forceinline__ uint2 succ_word(const int64_t* __restrict__ t, uint32_t p, uint32_t hi, int64_t te) {
    if (p >= hi) return make_uint2(p, SUCC_END);
    const uint64_t d = (uint64_t)(t[p] - te);
    return make_uint2(p, d < SUCC_FAR ? (uint32_t)d : SUCC_FAR);
}

// Successor index: for every edge e = (u, v, t), the first position after t in
// each of the four lists that touch it: out(u), in(v) (where e itself sits,
// so the search starts just past e), out(v) and in(u), with the time gap to
// that entry.  A search level whose candidate list belongs to an endpoint of
// the previous level's edge reads its window start here instead of
// binary-searching the list, and skips the window when the gap already
// exceeds it.
__global__ void successor_kernel(int64_t m, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                 const int64_t* __restrict__ t, const uint32_t* __restrict__ off_out,
                                 const int64_t* __restrict__ at_out, const uint32_t* __restrict__ off_in,
                                 const int64_t* __restrict__ at_in, const uint32_t* __restrict__ pos_out,
                                 const uint32_t* __restrict__ pos_in, uint2* __restrict__ so_src,
                                 uint2* __restrict__ si_dst, uint2* __restrict__ so_dst,
                                 uint2* __restrict__ si_src) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        const int64_t te = t[e];
        uint32_t hi = off_out[u + 1];
        so_src[e] = succ_word(at_out, first_later_from(at_out, pos_out[e] + 1, hi, te), hi, te);
        hi = off_in[v + 1];
        si_dst[e] = succ_word(at_in, first_later_from(at_in, pos_in[e] + 1, hi, te), hi, te);
        hi = off_out[v + 1];
        so_dst[e] = succ_word(at_out, first_later(at_out, off_out[v], hi, te), hi, te);
        hi = off_in[u + 1];
        si_src[e] = succ_word(at_in, first_later(at_in, off_in[u], hi, te), hi, te);
    }
}

int bits_for(unsigned long long x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

struct Pool {  // temporary device allocations, stream-ordered, freed at scope exit
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Pool(cudaStream_t s) : st(s) {}
    ~Pool() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <typename T>
    tm_status get(T** out, size_t count) {
        void* p = nullptr;
        if (dev_malloc_async(&p, std::max<size_t>(count * sizeof(T), 16), st) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed during graph build");
            return TM_E_OOM;
        }
        ptrs.push_back(p);
        *out = (T*)p;
        return TM_OK;
    }
};

// Graph storage is one allocation (one cudaMalloc at load, one cudaFree at
// free, instead of one per column: ~2 ms less per load/free cycle of a
// 10M-edge graph), carved into 256-byte aligned columns.
constexpr size_t COL_ALIGN = 256;
inline size_t col_bytes(size_t count, size_t elem) {
    return (std::max<size_t>(count * elem, 16) + COL_ALIGN - 1) & ~(COL_ALIGN - 1);
}

// Bytes of every column build() takes with owned(), in the same order.
size_t storage_bytes(int64_t n, int64_t m, bool node_labels, bool edge_labels) {
    size_t b = 0;
    if (node_labels) b += col_bytes(n, 1);
    b += col_bytes(m, 4) * 2 + col_bytes(m, 8) + col_bytes(m, 4);           // src, dst, t, perm
    if (edge_labels) b += col_bytes(m, 1);
    b += 2 * (col_bytes(n + 1, 4) + col_bytes(m, 8) + col_bytes(m, 4) * 2);  // out / in lists
    b += col_bytes(m, 4) + col_bytes(m, 8) + col_bytes(m, 4);               // pair-ordered list
    b += 8 * col_bytes(m, sizeof(uint2));                                     // successor words
    return b;
}

tm_status reserve_storage(tm_graph* g, size_t bytes) {
    void* p = nullptr;
    if (dev_malloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed for graph storage");
        return TM_E_OOM;
    }
    g->allocs.push_back(p);
    g->device_bytes += bytes;
    g->slab = (char*)p;
    g->slab_used = 0;
    g->slab_cap = bytes;
    return TM_OK;
}

template <typename T>
tm_status owned(tm_graph* g, T** out, size_t count) {
    const size_t bytes = col_bytes(count, sizeof(T));
    if (g->slab_used + bytes > g->slab_cap) {
        set_error("graph storage layout does not match the columns built");
        return TM_E_INVALID;
    }
    *out = (T*)(g->slab + g->slab_used);
    g->slab_used += bytes;
    return TM_OK;
}

#define TRY(x)                              \
    do {                                    \
        tm_status _s = (x);                 \
        if (_s != TM_OK) return _s;         \
    } while (0)

int grid_for(int64_t m, int sms) {
    int64_t g = (m + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

tm_status build(tm_graph* g, const tm_edges* e, cudaStream_t st) {
    const int64_t m = e->n_edges, n = e->n_nodes;
    const int sms = g->num_sms;
    Pool tmp(st);
    const int32_t *src = e->src, *dst = e->dst;
    const int64_t* t = e->t;
    const uint8_t* el = e->elabel;
    if (!e->on_device && m > 0) {
        int32_t *s2, *d2;
        int64_t* t2;
        TRY(tmp.get(&s2, m));
        TRY(tmp.get(&d2, m));
        TRY(tmp.get(&t2, m));
        TM_CUDA(cudaMemcpyAsync(s2, src, m * 4, cudaMemcpyHostToDevice, st));
        TM_CUDA(cudaMemcpyAsync(d2, dst, m * 4, cudaMemcpyHostToDevice, st));
        TM_CUDA(cudaMemcpyAsync(t2, t, m * 8, cudaMemcpyHostToDevice, st));
        src = s2; dst = d2; t = t2;
        if (el) {
            uint8_t* e2;
            TRY(tmp.get(&e2, m));
            TM_CUDA(cudaMemcpyAsync(e2, el, m, cudaMemcpyHostToDevice, st));
            el = e2;
        }
    }
    GraphView& v = g->v;
    v.n = n; v.m = m;
    TRY(reserve_storage(g, storage_bytes(n, m, e->nlabel != nullptr, el != nullptr)));
    // node labels
    if (e->nlabel) {
        uint8_t* nl;
        TRY(owned(g, &nl, n));
        TM_CUDA(cudaMemcpyAsync(nl, e->nlabel, n, e->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        v.nlabel = nl;
    }
    // 1. validate
    Check* chk;
    TRY(tmp.get(&chk, 1));
    Check init{~0ULL, 0ULL, 0ULL, 0ULL};
    TM_CUDA(cudaMemcpyAsync(chk, &init, sizeof(Check), cudaMemcpyHostToDevice, st));
    if (m > 0) {
        check_kernel<<<grid_for(m, sms), 256, 0, st>>>(src, dst, t, m, n, chk);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
    }
    Check hc;
    TM_CUDA(cudaMemcpyAsync(&hc, chk, sizeof(Check), cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    if (hc.bad) {
        set_error("edge endpoint out of [0, n_nodes) or negative timestamp");
        return TM_E_INVALID;
    }
    // 2. time order
    uint32_t *perm_a, *perm_b;
    TRY(tmp.get(&perm_a, m));
    TRY(tmp.get(&perm_b, m));
    size_t rtemp_bytes = radix_temp_bytes((uint64_t)m);
    void* rtemp;
    TRY(tmp.get((char**)&rtemp, rtemp_bytes));
    if (m > 0 && hc.descents > 0) {
        uint64_t *ka, *kb;
        TRY(tmp.get(&ka, m));
        TRY(tmp.get(&kb, m));
        time_keys_kernel<<<grid_for(m, sms), 256, 0, st>>>(t, m, hc.tmin, ka, perm_a);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
        TRY(radix_sort_pairs(ka, kb, perm_a, perm_b, (uint64_t)m, bits_for(hc.tmax - hc.tmin), rtemp, rtemp_bytes, st));
    } else if (m > 0) {
        iota_kernel<<<grid_for(m, sms), 256, 0, st>>>(perm_a, m);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
    }
    // 3. edge columns in edge-id order
    int32_t *s_o, *d_o, *p_o;
    int64_t* t_o;
    uint8_t* el_o = nullptr;
    TRY(owned(g, &s_o, m));
    TRY(owned(g, &d_o, m));
    TRY(owned(g, &t_o, m));
    TRY(owned(g, &p_o, m));
    if (el) TRY(owned(g, &el_o, m));
    if (m > 0) {
        gather_edges_kernel<<<grid_for(m, sms), 256, 0, st>>>(perm_a, m, src, dst, t, el, s_o, d_o, t_o, el_o, p_o);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
    }
    v.src = s_o; v.dst = d_o; v.t = t_o; v.elabel = el_o;
    g->perm = p_o;
    // 4. adjacency lists
    unsigned long long* deg;
    TRY(tmp.get(&deg, n + 1));
    size_t stemp_bytes = scan_temp_bytes((uint64_t)(n + 1));
    void* stemp;
    TRY(tmp.get((char**)&stemp, stemp_bytes));
    uint32_t *nk_a, *nk_b, *pos_edge[2];
    TRY(tmp.get(&nk_a, m));
    TRY(tmp.get(&nk_b, m));
    TRY(tmp.get(&pos_edge[0], m));
    TRY(tmp.get(&pos_edge[1], m));
    int nbits = bits_for((unsigned long long)(n > 0 ? n - 1 : 0));
    for (int dir = 0; dir < 2; ++dir) {
        const int32_t* key_node = dir == 0 ? s_o : d_o;
        const int32_t* other = dir == 0 ? d_o : s_o;
        uint32_t* off;
        int64_t* at;
        int32_t *anbr, *aeid;
        TRY(owned(g, &off, n + 1));
        TRY(owned(g, &at, m));
        TRY(owned(g, &anbr, m));
        TRY(owned(g, &aeid, m));
        TM_CUDA(cudaMemsetAsync(deg, 0, (n + 1) * sizeof(unsigned long long), st));
        if (m > 0) {
            degree_kernel<<<grid_for(m, sms), 256, 0, st>>>(key_node, m, deg);
            note_launches(1);
            TM_CUDA(cudaGetLastError());
        }
        TRY(exclusive_scan_u64(deg, deg, (uint64_t)(n + 1), stemp, st));
        offsets_kernel<<<grid_for(n + 1, sms), 256, 0, st>>>(deg, n + 1, off);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
        if (m > 0) {
            node_keys_kernel<<<grid_for(m, sms), 256, 0, st>>>(key_node, m, nk_a, perm_a);
            note_launches(1);
            TM_CUDA(cudaGetLastError());
            TRY(radix_sort_pairs32(nk_a, nk_b, perm_a, perm_b, (uint64_t)m, nbits, rtemp, rtemp_bytes, st));
            list_columns_kernel<<<grid_for(m, sms), 256, 0, st>>>(perm_a, m, t_o, other, at, anbr, aeid,
                                                                   pos_edge[dir]);
            note_launches(1);
            TM_CUDA(cudaGetLastError());
        }
        v.off[dir] = off; v.at[dir] = at; v.anbr[dir] = anbr; v.aeid[dir] = aeid;
    }
    // 5. pair-ordered out-lists: stable sorts of the time-ordered edge ids by
    //    destination, then by source, give (source, destination, time) order
    {
        int32_t *pn, *pe;
        int64_t* ptm;
        TRY(owned(g, &pn, m));
        TRY(owned(g, &ptm, m));
        TRY(owned(g, &pe, m));
        if (m > 0) {
            node_keys_kernel<<<grid_for(m, sms), 256, 0, st>>>(d_o, m, nk_a, perm_a);
            note_launches(1);
            TM_CUDA(cudaGetLastError());
            TRY(radix_sort_pairs32(nk_a, nk_b, perm_a, perm_b, (uint64_t)m, nbits, rtemp, rtemp_bytes, st));
            keys_by_perm_kernel<<<grid_for(m, sms), 256, 0, st>>>(s_o, perm_a, m, nk_a);
            note_launches(1);
            TM_CUDA(cudaGetLastError());
            TRY(radix_sort_pairs32(nk_a, nk_b, perm_a, perm_b, (uint64_t)m, nbits, rtemp, rtemp_bytes, st));
            pair_columns_kernel<<<grid_for(m, sms), 256, 0, st>>>(perm_a, m, t_o, d_o, pn, ptm, pe);
            note_launches(1);
            TM_CUDA(cudaGetLastError());
        }
        v.pnbr = pn; v.pt = ptm; v.peid = pe;
    }
    // 6. successor index (window starts for lists that touch the previous edge)
    uint2* nx[4];
    for (int j = 0; j < 4; ++j) TRY(owned(g, &nx[j], m));
    if (m > 0) {
        successor_kernel<<<grid_for(m, sms), 256, 0, st>>>(m, s_o, d_o, t_o, v.off[0], v.at[0], v.off[1], v.at[1],
                                                           pos_edge[0], pos_edge[1], nx[NX_OUT_SRC], nx[NX_IN_DST],
                                                           nx[NX_OUT_DST], nx[NX_IN_SRC]);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
    }
    for (int j = 0; j < 4; ++j) v.nxt[j] = nx[j];
    uint2* px[4];
    for (int j = 0; j < 4; ++j) TRY(owned(g, &px[j], m));
    if (m > 0) {
        successor_by_position_kernel<<<grid_for(m, sms), 256, 0, st>>>(
            m, v.aeid[0], v.aeid[1], nx[NX_OUT_SRC], nx[NX_OUT_DST], nx[NX_IN_DST], nx[NX_IN_SRC], px[0], px[1], px[2],
            px[3]);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
    }
    for (int j = 0; j < 4; ++j) v.pnx[j] = px[j];
    TM_CUDA(cudaStreamSynchronize(st));
    return TM_OK;
}

}  // namespace

}  // namespace tmg

using namespace tmg;

extern "C" tm_status tm_graph_load(const tm_edges* e, int device, void* stream, tm_graph** out) {
    if (!e || !out) { set_error("null argument"); return TM_E_INVALID; }
    if (e->n_edges < 0 || e->n_nodes < 0 || e->n_edges >= 0x3FFFFFFF || e->n_nodes >= 0x7FFFFFFF) {
        set_error("n_edges / n_nodes out of range");
        return TM_E_INVALID;
    }
    if (e->n_edges > 0 && (!e->src || !e->dst || !e->t || e->n_nodes < 1)) {
        set_error("missing edge columns");
        return TM_E_INVALID;
    }
    int ndev = 0;
    TM_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) { set_error("bad device"); return TM_E_INVALID; }
    TM_ENTER(device);
    tm_graph* g = new tm_graph();
    g->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete g; return cuda_fail(cudaGetLastError(), "props"); }
    g->num_sms = prop.multiProcessorCount;
    // keep up to 2 GiB of freed build temporaries in the device's stream-ordered
    // pool, so loading graphs one after another does not go back to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = 0;
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (keep < (2ull << 30)) {
            keep = 2ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    cudaGetLastError();
    tm_status s = build(g, e, (cudaStream_t)stream);
    if (s != TM_OK) {
        tm_graph_free(g);
        return s;
    }
    *out = g;
    return TM_OK;
}

extern "C" tm_status tm_graph_free(tm_graph* g) {
    if (!g) return TM_OK;
    cudaSetDevice(g->device);
    drop_batches(g);
    for (void* p : g->allocs) cudaFree(p);
    delete g;
    return TM_OK;
}

extern "C" tm_status tm_graph_info(const tm_graph* g, int64_t* n_nodes, int64_t* n_edges, uint64_t* device_bytes) {
    if (!g) { set_error("null graph"); return TM_E_INVALID; }
    if (n_nodes) *n_nodes = g->v.n;
    if (n_edges) *n_edges = g->v.m;
    if (device_bytes) *device_bytes = g->device_bytes;
    return TM_OK;
}

extern "C" tm_status tm_graph_edge_perm(const tm_graph* g, int64_t* out_perm) {
    if (!g || (!out_perm && g->v.m > 0)) { set_error("null argument"); return TM_E_INVALID; }
    if (g->v.m == 0) return TM_OK;
    TM_ENTER(g->device);
    std::vector<int32_t> tmp((size_t)g->v.m);
    TM_CUDA(cudaMemcpy(tmp.data(), g->perm, g->v.m * 4, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < g->v.m; ++i) out_perm[i] = tmp[i];
    return TM_OK;
}
