// Batched count that allocates no memory.
//
// Some callers cannot allocate device memory when they want to run a query:
// real-time loops that reserve all of their memory up front, processes that
// run under a fixed memory cap or an allocator that forbids cudaMalloc after
// start-up, and plug-ins whose host framework owns every allocation.
// tm_count_batch_noalloc serves them.  It runs the same persistent multi-query
// count kernel as tm_count_batch, but the kernel's scratch -- the control
// block, the per-query launch records and the task queue for donated subtrees
// -- lives in one fixed, file-scope __device__ array instead of buffers
// obtained from cudaMalloc.  The caller passes the graph, the compiled queries
// and the device array that receives the totals.
//
// The array is g_noalloc_scratch below: TM_NOALLOC_SCRATCH_BYTES bytes, present
// on every GPU that loads this library until the process exits.  It holds at
// most TM_NOALLOC_MAX_QUERIES launch records and TM_NOALLOC_TASKS task slots,
// which one call uses up as it donates (slots are not reused within a call).
// The launch records are staged in a file-scope host buffer (not on the
// caller's stack, which may be small in a plug-in's threads); a mutex guards
// it while the records are copied out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "tm_internal.cuh"

namespace tmg {

namespace {

constexpr int NOALLOC_MAX_QUERIES = TM_NOALLOC_MAX_QUERIES;
constexpr uint64_t NOALLOC_TASKS = TM_NOALLOC_TASKS;

// byte layout of the static array
constexpr size_t OFF_CTRL = 0;
constexpr size_t OFF_QDEV = 512;
constexpr size_t OFF_READY = (OFF_QDEV + NOALLOC_MAX_QUERIES * sizeof(QueryDev) + 255) / 256 * 256;
constexpr size_t OFF_TASKS = (OFF_READY + NOALLOC_TASKS + 255) / 256 * 256;
constexpr size_t NOALLOC_END = OFF_TASKS + NOALLOC_TASKS * sizeof(Task);
static_assert(NOALLOC_END <= TM_NOALLOC_SCRATCH_BYTES, "static scratch layout exceeds its stated size");
static_assert(sizeof(Ctrl) <= OFF_QDEV, "control block overlaps the launch records");

// The scratch itself.  In host code this name is only a host-side stand-in
// for the symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TM_NOALLOC_SCRATCH_BYTES];

// Host staging of the control block and launch records (about 60 KB).
struct Stage {
    Ctrl ctrl;
    unsigned char pad[OFF_QDEV - sizeof(Ctrl)];
    QueryDev q[NOALLOC_MAX_QUERIES];
};
Stage g_stage;
std::mutex g_stage_mu;

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_dev[MAX_DEVICES] = {nullptr};

// Once per device, with that device current: the array's device address.
tm_status scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= MAX_DEVICES) {
        set_error("device index beyond the no-alloc set-up table");
        return TM_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_dev[device] = (unsigned char*)p;
    }
    *out = g_scratch_dev[device];
    return TM_OK;
}

}  // namespace

}  // namespace tmg

using namespace tmg;

extern "C" tm_status tm_count_batch_noalloc(tm_graph* g, tm_query* const* qs, int nq, void* stream,
                                            uint64_t* totals_dev) {
    if (!g || !qs || !totals_dev) { set_error("null argument"); return TM_E_INVALID; }
    if (nq < 1 || nq > NOALLOC_MAX_QUERIES) {
        set_error("tm_count_batch_noalloc: nq must be in [1, " + std::to_string(NOALLOC_MAX_QUERIES) +
                  "], the capacity of its static scratch");
        return TM_E_INVALID;
    }
    TM_ENTER(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    tm_status s = scratch_address(g->device, &base);
    if (s != TM_OK) return s;
    const uint64_t m = (uint64_t)g->v.m;
    int warp_smem = 16, warps = 1;
    unsigned feat = 0;
    for (int j = 0; j < nq; ++j)
        if (!qs[j] || query_graph(qs[j]) != g) { set_error("null or mismatched query in batch"); return TM_E_INVALID; }
    // Every call reuses the array: clear the caller's totals, then rewrite the
    // control block and the launch records and clear the task-ready flags.
    TM_CUDA(cudaMemsetAsync(totals_dev, 0, (size_t)nq * sizeof(uint64_t), st));
    if (m == 0) return cudaStreamSynchronize(st) == cudaSuccess ? TM_OK : cuda_fail(cudaGetLastError(), "sync");
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        memset(&g_stage.ctrl, 0, sizeof(Ctrl));
        uint64_t chunk_base = 0;
        for (int j = 0; j < nq; ++j) {
            QueryDev& qd = g_stage.q[j];
            memset(&qd, 0, sizeof(QueryDev));
            query_plan(qs[j], &qd.plan);
            qd.root_begin = 0;
            qd.root_end = m;
            qd.n_chunks = (m + (uint64_t)qd.plan.tune.chunk_roots - 1) / (uint64_t)qd.plan.tune.chunk_roots;
            qd.chunk_base = chunk_base;
            chunk_base += qd.n_chunks;
            qd.total = (unsigned long long*)totals_dev + j;
            warp_smem = std::max(warp_smem, qd.plan.warp_smem);
            warps = std::max(warps, qd.plan.tune.warps_per_block);
            feat |= plan_features(qd.plan);
        }
        g_stage.ctrl.total_chunks = chunk_base;
        // pageable source: the copy has left this buffer when the call returns
        TM_CUDA(cudaMemcpyAsync(base + OFF_CTRL, &g_stage, OFF_QDEV + (size_t)nq * sizeof(QueryDev),
                                cudaMemcpyHostToDevice, st));
    }
    TM_CUDA(cudaMemsetAsync(base + OFF_READY, 0, NOALLOC_TASKS, st));
    Scratch view;                       // points into the static array; never freed
    view.device = g->device;
    view.head = (char*)(base + OFF_CTRL);
    view.qcap = NOALLOC_MAX_QUERIES;
    view.tasks = (Task*)(base + OFF_TASKS);
    view.ready = base + OFF_READY;
    view.task_cap = NOALLOC_TASKS;
    s = launch_search(g, MODE_COUNT, (const QueryDev*)(base + OFF_QDEV), nq, warp_smem, warps, feat, &view, st);
    if (s != TM_OK) return s;
    Ctrl done;
    TM_CUDA(cudaMemcpyAsync(&done, base + OFF_CTRL, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    TM_CUDA(cudaStreamSynchronize(st));
    note_search_stats(done);
    if (done.err) { set_error("a bounded device wait timed out"); return TM_E_TIMEOUT; }
    return TM_OK;
}
