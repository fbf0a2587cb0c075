// Device building blocks for graph ingest and enumeration offsets:
// an exclusive prefix sum and a stable LSD radix sort of (key, value) pairs.
#include <cuda_runtime.h>

#include "tm_internal.cuh"

namespace tmg {

// ------------------------------------------------------------------- scan

namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

// Exclusive scan of one block's thread totals; returns this thread's prefix,
// and the block total in *total.
__device__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* total) {
    __shared__ unsigned long long warp_sum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = warp_incl_scan(v);
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < SCAN_THREADS / 32 ? warp_sum[lane] : 0ULL;
        unsigned long long wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) warp_sum[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    unsigned long long r = warp_sum[warp] + inc - v;
    __syncthreads();
    return r;
}

__global__ void scan_reduce_kernel(const unsigned long long* __restrict__ in, uint64_t n,
                                   unsigned long long* __restrict__ partial) {
    __shared__ unsigned long long red[SCAN_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    unsigned long long s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        uint64_t i = base + (uint64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// Block-level exclusive scan of one tile plus the tile's carried-in offset.
__global__ void scan_down_kernel(const unsigned long long* __restrict__ in, unsigned long long* out, uint64_t n,
                                 const unsigned long long* __restrict__ partial_scanned) {
    __shared__ unsigned long long tile[SCAN_TILE];
    __shared__ unsigned long long tot;
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int li = j * SCAN_THREADS + threadIdx.x;
        uint64_t i = base + li;
        tile[li] = i < n ? in[i] : 0ULL;
    }
    __syncthreads();
    unsigned long long loc[SCAN_ITEMS];
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        loc[j] = tile[threadIdx.x * SCAN_ITEMS + j];
        s += loc[j];
    }
    unsigned long long pre = block_excl_scan(s, &tot);
    unsigned long long carry = partial_scanned ? partial_scanned[blockIdx.x] : 0ULL;
    pre += carry;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        tile[threadIdx.x * SCAN_ITEMS + j] = pre;
        pre += loc[j];
    }
    __syncthreads();
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int li = j * SCAN_THREADS + threadIdx.x;
        uint64_t i = base + li;
        if (i < n) out[i] = tile[li];
    }
}

uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
}  // namespace

size_t scan_temp_bytes(uint64_t n) {
    size_t bytes = 0;
    uint64_t len = n;
    while (len > (uint64_t)SCAN_TILE) {
        len = ceil_div(len, SCAN_TILE);
        bytes += ((len * 8 + 255) / 256) * 256;
    }
    return bytes + 256;
}

tm_status exclusive_scan_u64(const unsigned long long* in, unsigned long long* out, uint64_t n, void* temp,
                             cudaStream_t st) {
    if (n == 0) return TM_OK;
    uint64_t nb = ceil_div(n, SCAN_TILE);
    if (nb == 1) {
        scan_down_kernel<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
        return TM_OK;
    }
    unsigned long long* partial = (unsigned long long*)temp;
    void* rest = (char*)temp + ((nb * 8 + 255) / 256) * 256;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, partial);
    note_launches(1);
    TM_CUDA(cudaGetLastError());
    tm_status s = exclusive_scan_u64(partial, partial, nb, rest, st);
    if (s != TM_OK) return s;
    scan_down_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, partial);
    note_launches(1);
    TM_CUDA(cudaGetLastError());
    return TM_OK;
}

// ------------------------------------------------------------ radix sort

namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_BINS = 256;

template <typename K>
__global__ void radix_hist_kernel(const K* __restrict__ keys, uint64_t n, int shift, uint64_t ntiles,
                                  unsigned long long* __restrict__ counts) {
    __shared__ unsigned int h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ITEMS; ++j) {
        uint64_t i = base + (uint64_t)j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)((keys[i] >> shift) & 0xFF)], 1u);
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items keep their input order within a digit.  A tile is
// processed in rounds of RS_THREADS consecutive items; within a round an
// item's rank among equal digits = (equal digits in earlier warps) + (equal
// digits in earlier lanes of its own warp, from __match_any_sync).
template <typename K>
__global__ void radix_scatter_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
                                     uint32_t* __restrict__ vout, uint64_t n, int shift, uint64_t ntiles,
                                     const unsigned long long* __restrict__ offsets) {
    __shared__ unsigned long long base_d[RS_BINS];
    __shared__ unsigned int wc[RS_WARPS][RS_BINS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base_d[threadIdx.x] = offsets[(uint64_t)threadIdx.x * ntiles + blockIdx.x];
    uint64_t tile0 = (uint64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < RS_ITEMS; ++j) {
        for (int x = threadIdx.x; x < RS_WARPS * (RS_BINS + 1); x += RS_THREADS) (&wc[0][0])[x] = 0;
        __syncthreads();
        uint64_t i = tile0 + (uint64_t)j * RS_THREADS + threadIdx.x;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        uint32_t val = valid ? vin[i] : 0u;
        unsigned d = valid ? (unsigned)((key >> shift) & 0xFF) : (unsigned)RS_BINS;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (rank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned before = 0;
            for (int w = 0; w < warp; ++w) before += wc[w][d];
            uint64_t pos = base_d[d] + before + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        {
            unsigned tot = 0;
            for (int w = 0; w < RS_WARPS; ++w) tot += wc[w][threadIdx.x];
            base_d[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}
}  // namespace

size_t radix_temp_bytes(uint64_t n) {
    uint64_t ntiles = ceil_div(n > 0 ? n : 1, RS_TILE);
    uint64_t cnt = ntiles * RS_BINS;
    return ((cnt * 8 + 255) / 256) * 256 + scan_temp_bytes(cnt);
}

template <typename K>
tm_status radix_sort_pairs_t(K* keys_a, K* keys_b, uint32_t* vals_a, uint32_t* vals_b, uint64_t n, int bits,
                             void* temp, size_t temp_bytes, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return TM_OK;
    if (temp_bytes < radix_temp_bytes(n)) return TM_E_INVALID;
    uint64_t ntiles = ceil_div(n, RS_TILE);
    uint64_t cnt = ntiles * RS_BINS;
    unsigned long long* counts = (unsigned long long*)temp;
    void* scan_tmp = (char*)temp + ((cnt * 8 + 255) / 256) * 256;
    K *ki = keys_a, *ko = keys_b;
    uint32_t *vi = vals_a, *vo = vals_b;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        radix_hist_kernel<K><<<(unsigned)ntiles, RS_THREADS, 0, st>>>(ki, n, shift, ntiles, counts);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
        tm_status s = exclusive_scan_u64(counts, counts, cnt, scan_tmp, st);
        if (s != TM_OK) return s;
        radix_scatter_kernel<K><<<(unsigned)ntiles, RS_THREADS, 0, st>>>(ki, vi, ko, vo, n, shift, ntiles, counts);
        note_launches(1);
        TM_CUDA(cudaGetLastError());
        K* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
    }
    if (ki != keys_a) {
        TM_CUDA(cudaMemcpyAsync(keys_a, ki, n * sizeof(K), cudaMemcpyDeviceToDevice, st));
        TM_CUDA(cudaMemcpyAsync(vals_a, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    return TM_OK;
}

tm_status radix_sort_pairs(uint64_t* keys_a, uint64_t* keys_b, uint32_t* vals_a, uint32_t* vals_b, uint64_t n,
                           int bits, void* temp, size_t temp_bytes, cudaStream_t st) {
    return radix_sort_pairs_t<uint64_t>(keys_a, keys_b, vals_a, vals_b, n, bits, temp, temp_bytes, st);
}

tm_status radix_sort_pairs32(uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a, uint32_t* vals_b, uint64_t n,
                             int bits, void* temp, size_t temp_bytes, cudaStream_t st) {
    return radix_sort_pairs_t<uint32_t>(keys_a, keys_b, vals_a, vals_b, n, bits, temp, temp_bytes, st);
}

}  // namespace tmg
