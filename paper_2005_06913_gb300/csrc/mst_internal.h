// mst_internal.h — host-side declarations shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mst.h"
#include "mst_common.cuh"

namespace mst {

// The status a solve reports for a set of device status bits (host and
// device): a bounded wait that gave up outranks everything, then an internal
// check, then bad input, then a disconnected graph.
__host__ __device__ inline mst_status status_code(uint32_t bits)
{
    if (bits & ST_TIMEOUT)
        return MST_ERR_TIMEOUT;
    if (bits & ST_INTERNAL)
        return MST_ERR_INTERNAL;
    if (bits & (ST_BAD_VERTEX | ST_NAN | ST_BAD_OFFSETS))
        return MST_ERR_INVALID_ARG;
    if (bits & ST_DISCONNECTED)
        return MST_ERR_DISCONNECTED;
    return MST_OK;
}

// ------------------------------------------------------------ single graph

// Workspace and captured round loop of the single-graph solver.
struct Single {
    Ws ws{};
    void *base = nullptr;   // one cudaMalloc carved into the Ws arrays
    size_t bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid_tiles = 0;     // persistent grid of the tile kernels
    int grid_stream = 0;    // grid of the grid-stride kernels
    int grid_fused = 0;     // co-resident grid of the fused cooperative kernel
    int fused_blocks_per_sm = 4;  // CTAs per SM of the fused kernel (clamped by occupancy)
    int fused_threads = 256;      // threads per CTA of the fused kernel
    int schedule = 0;       // 0 fused, shape per solve; 1 fused, fixed shape; 2 CUDA graph
    int sms = 0;            // multiprocessors of the device
    uint64_t solves = 0;    // solves since the descriptors were last cleared
    uint32_t wait_limit = 0;  // polls of a grid-barrier wait before it gives up (0: default)
};

struct KernelProfile {
    std::string name;
    int launches;
    double ms;
    double bytes;
};

// Workspace bytes for capacities (n_cap, m_cap).
size_t single_bytes(uint32_t n_cap, uint32_t m_cap);
// Allocates (or grows) the workspace and rebuilds the graph.
cudaError_t single_reserve(Single &s, int device, uint32_t n, uint32_t m);
void single_release(Single &s);
// Queues one solve on `stream` (arguments already validated).
// Device copy of a solve's inputs that the fused kernel writes while its
// round-0 find-min reads them from mapped host memory.
struct InputCopy {
    int32_t *src;
    int32_t *dst;
    void *w;
};

cudaError_t single_launch(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                          uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n,
                          uint32_t m, cudaStream_t stream, int grid = 0, const InputCopy *copy = nullptr);
double single_alg_bytes(const Ctl &c);
// Row of every entry of an adjacency CSR (mst_csr.cu); a malformed offset
// table marks entry 0 with row -1.
cudaError_t csr_rows(const int64_t *row_ptr, const int32_t *col, uint32_t n, uint32_t nnz,
                     bool symmetric, int32_t *rows, int num_sms, cudaStream_t stream);
// Per-phase times of the last fused solve (its own phase log; synchronous).
cudaError_t single_phase_profile(Single &s, cudaStream_t stream, std::vector<KernelProfile> &prof);
// Replays a solve kernel by kernel between CUDA events (synchronous).
cudaError_t single_profile(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                           uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n, uint32_t m,
                           cudaStream_t stream, std::vector<KernelProfile> &prof);

// ------------------------------------------------------------------ batched

// One graph of a descriptor-list batch (the serving path): caller buffers,
// sizes, weight type and the graph's offsets into the batch workspace.
struct GraphDesc {
    const int32_t *src, *dst;
    const void *w;
    int32_t *out;
    int64_t *out_count;
    uint32_t n, m, wt, pad;
    uint64_t ws_vo, ws_eo;
};

// Per-size-bucket schedule of the batched solver.
struct BatchedConfig {
    int schedule = 0;       // 1 block per graph, 2 warp per small graph
    int block_threads = 0;  // 0 = automatic
    int blocks_per_sm = 0;  // CTAs per SM (sets the shared memory per CTA)
    int warp_max_m = 0;     // graphs with at most this many edges go to warps
};

struct Batched {
    void *base = nullptr;
    size_t bytes = 0;
    uint64_t n_cap = 0, m_cap = 0;
    int32_t g_cap = 0;
    void *ctl = nullptr;    // batched control words (inside base)
    int schedule = 0;       // forced schedule (0 = autotuned/default)
    int block_threads = 0;  // forced block size (0 = autotuned/default)
    std::map<int, BatchedConfig> tuned;  // size bucket -> choice
    bool tuned_loaded = false;
    int32_t last_G = 0;     // graphs of the last batched launch (per-graph status)
};

size_t batched_bytes(int32_t G, uint64_t n, uint64_t m);
cudaError_t batched_reserve(Batched &b, int32_t G, uint64_t n, uint64_t m);
void batched_release(Batched &b);
cudaError_t batched_launch(Batched &b, int device, uint32_t wt, int32_t G, const int64_t *vtx_off,
                           const int64_t *edge_off, uint64_t total_n, uint64_t total_m,
                           const int32_t *src, const int32_t *dst, const void *w, int32_t *out,
                           int64_t *out_counts, cudaStream_t stream);
uint32_t batched_status_bits(Batched &b, cudaStream_t stream, cudaError_t *err);
// Status bits of each graph of the last batched launch (synchronises `stream`).
cudaError_t batched_graph_status(Batched &b, cudaStream_t stream, int32_t G, uint32_t *bits);
// Status bits of each graph of a finished descriptor batch run in `ws_base`.
cudaError_t desc_batch_graph_status(void *ws_base, int32_t G, uint64_t total_n, uint64_t total_m,
                                    uint32_t *bits);
// Workspace bytes of a descriptor batch with these totals.
size_t desc_batch_bytes(int32_t G, uint64_t total_n, uint64_t total_m);
// Solves a descriptor batch in caller-provided workspace `ws_base` (of
// desc_batch_bytes bytes); `descs` is a device array of G entries.
cudaError_t batched_launch_desc(const Batched &tuning, int device, void *ws_base, int32_t G,
                                const GraphDesc *descs, uint64_t total_n, uint64_t total_m,
                                cudaStream_t stream);
// Device status bits of a descriptor batch run in `ws_base`.
cudaError_t desc_batch_status(void *ws_base, uint32_t *bits, cudaStream_t stream);
cudaError_t batched_autotune(Batched &b, int device, uint32_t wt, int32_t G,
                             const int64_t *vtx_off, const int64_t *edge_off, uint64_t total_n,
                             uint64_t total_m, const int32_t *src, const int32_t *dst,
                             const void *w, int32_t *out, int64_t *out_counts, const char *path,
                             cudaStream_t stream);

// ------------------------------------------------------------------ serving

struct Request {
    uint64_t ticket;
    uint32_t wt;
    int32_t n;
    int64_t m;
    const int32_t *src, *dst;
    const void *w;
    int32_t *out;
    int64_t *out_count;
    double t_submit_us;
    size_t footprint;
};

struct Server;

// ------------------------------------------------------------------ handle

enum LastKind { LAST_NONE = 0, LAST_SINGLE = 1, LAST_BATCHED = 2 };

}  // namespace mst

// Arguments of the last single-graph solve (for mst_profile_last_solve).
struct LastSolve {
    const int32_t *src = nullptr, *dst = nullptr;
    const void *w = nullptr;
    int32_t *out = nullptr;
    int64_t *out_count = nullptr;
    uint32_t n = 0, m = 0, wt = 0;
    bool valid = false;
};

struct mst_handle_s {
    int device = 0;
    LastSolve last_solve;
    void *staging = nullptr;  // device staging of mst_solve_host
    size_t staging_bytes = 0;
    int32_t *csr_rows = nullptr;  // row of each CSR entry (mst_solve_csr)
    size_t csr_cap = 0;           // entries
    cudaStream_t copy_stream[2] = {nullptr, nullptr};  // its input copies run side by side
    cudaEvent_t copy_event[3] = {nullptr, nullptr, nullptr};
    size_t budget = 0;  // 0 = unlimited
    int num_sms = 0;
    mst::Single single;
    mst::Batched batched;
    mst::LastKind last = mst::LAST_NONE;
    mst::Server *server = nullptr;
};

namespace mst {
mst_status status_from_bits(uint32_t bits);
double now_us();
mst_status server_start(mst_handle h, int streams, int max_batch);
mst_status server_submit(mst_handle h, const Request &r, uint64_t *ticket);
mst_status server_poll(mst_handle h, uint64_t ticket, int *done, double *latency_us);
mst_status server_drain(mst_handle h);
mst_status server_stop(mst_handle h);
}  // namespace mst
