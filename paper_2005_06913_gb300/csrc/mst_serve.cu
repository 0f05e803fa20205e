// mst_serve.cu — continuous-batching server over the batched solver.
//
// A host thread owns up to S CUDA streams ("slots").  Submitted graphs wait
// in a FIFO queue.  Whenever a slot is free, the thread takes queued requests
// in arrival order, as many as fit max_batch and the memory budget (each
// request needs workspace for its edge list and vertex arrays), builds a
// descriptor list in pinned host memory, and launches one batched solve on
// the slot's stream with workspace from the stream-ordered allocator.  When
// the slot's completion event fires, the requests are marked done (their
// latency is completion minus submit time) and the memory is released.  So
// requests that arrive while other batches run on the GPU are admitted as
// soon as a slot and memory free up, and their solves overlap on the device.
// Large requests (more than kServeBigM edges) are not batched: one CTA per
// graph would take tens of milliseconds on them.  Medium ones (more than
// kServeMidM edges) wait for the fused lane too unless its queue is long.
// The lane runs one fused multi-CTA single-graph solve at a time, on a
// slot's stream, in the server's one lane workspace: on the whole
// co-resident grid when nothing else is in flight, else on half of it,
// while other slots keep serving batches.  Lane requests that queued up
// meanwhile are solved together in the next launch, as one union graph.
// Each request's result is the same as a solve of that graph alone: the
// minimum spanning tree under the (weight, edge id) order is unique.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <unordered_map>

#include "mst_internal.h"

namespace mst {

constexpr int64_t kServeBigM = 131072;  // larger requests always get the fused kernel
constexpr int64_t kServeMidM = 16384;   // larger ones wait for it ...
constexpr int kServeLaneDepth = 4;       // ... unless this many are ahead of them

// One request of a fused-lane union (see k_lane_gather).
struct LaneDesc {
    const int32_t *src, *dst;
    const uint32_t *w;
    int32_t *out;
    int64_t *out_count;
    uint32_t n, m;
    uint32_t vbase, ebase;  // the request's first vertex and edge in the union
};

struct Slot {
    bool big = false;             // the request in flight is a large one
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    GraphDesc *h_desc = nullptr;  // pinned host descriptors
    GraphDesc *d_desc = nullptr;  // device copy
    int cap = 0;
    void *ws = nullptr;           // workspace of the batch in flight
    size_t ws_bytes = 0;
    uint64_t total_n = 0, total_m = 0;  // the batch's totals (locate per-graph status)
    LaneDesc *h_lane = nullptr;   // pinned host descriptors of a lane union
    int lane_k = 0;               // requests in the lane union in flight (0: one request)
    std::vector<uint64_t> tickets;
    bool busy = false;
};

struct Outcome {
    bool done = false;
    double latency_us = 0.0;
    mst_status status = MST_OK;
};

struct Server {
    mst_handle h = nullptr;
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Outcome> results;
    std::unordered_map<uint64_t, double> submit_us;
    std::vector<Slot> slots;
    Single lane;  // fused-kernel workspace of the (single) large-request lane
    void *ubuf = nullptr;  // the lane union's copies of its requests, descriptors, flags
    size_t ubuf_bytes = 0;
    std::vector<std::pair<void *, size_t>> retired;  // outgrown lane workspaces, freed at
                                                     // stop (or when memory runs short)
    int max_batch = 256;
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    int inflight = 0;
    bool big_inflight = false;  // a fused single-graph solve is running
    bool stop = false;
    cudaError_t error = cudaSuccess;
};

// ------------------------------------------------------- the fused lane's unions
//
// Requests queued for the fused lane are solved together: their graphs are
// copied side by side into one union graph (vertex ids shifted by the
// request's vertex base, edge ids by its edge base), the fused kernel
// solves the union once, and each request's ids are cut back out of the
// union's ascending output.  The minimum spanning forest of a disjoint
// union is the union of the graphs' own forests (no edge joins two
// requests), and an edge's order (weight, id) within its request is the
// same in the union, so each request gets exactly the tree it gets alone;
// the union pays the fused kernel's per-round barriers once for all of them.

constexpr int kLaneBatch = 16;            // requests per union at most
constexpr int64_t kLaneMaxM = 1ll << 25;  // edges per union at most (unless one request alone)
constexpr uint32_t kLaneMaxN = 1u << 24;  // vertices the lane is sized for up front

// Copies request blockIdx.y into the union.  An edge with an endpoint out of
// range becomes a self-loop (the solve ignores both alike) and a NaN weight
// is copied as is (it sorts after every other weight, alone or in the
// union); either is recorded in the request's flag, so the request, and
// only it, reports MST_ERR_INVALID_ARG.
__global__ void k_lane_gather(const LaneDesc *d, uint32_t wt, int32_t *us, int32_t *ud,
                              uint32_t *uw, uint32_t *flags)
{
    const LaneDesc q = d[blockIdx.y];
    bool bad = false;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q.m; i += gridDim.x * blockDim.x) {
        uint32_t u = (uint32_t)__ldg(q.src + i), v = (uint32_t)__ldg(q.dst + i);
        const uint32_t x = __ldg(q.w + i);
        if (u >= q.n || v >= q.n) {
            bad = true;
            u = v = 0;
        }
        if (wt && (x & 0x7fffffffu) > 0x7f800000u)
            bad = true;
        us[q.ebase + i] = (int32_t)(q.vbase + u);
        ud[q.ebase + i] = (int32_t)(q.vbase + v);
        uw[q.ebase + i] = x;
    }
    if (__syncthreads_or(bad ? 1 : 0) && threadIdx.x == 0)
        atomicOr(&flags[blockIdx.y], 1u);
}

// First position of ids[0..cnt) (ascending) that is >= x.
__device__ __forceinline__ uint32_t lower_pos(const int32_t *ids, uint32_t cnt, uint32_t x)
{
    uint32_t lo = 0, hi = cnt;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint32_t)ids[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Cuts request blockIdx.x's ids out of the union's output and records its
// status: MST_ERR_INVALID_ARG if flagged, MST_ERR_DISCONNECTED if its ids do
// not span it, else MST_OK (a wait that ran out is reported from the
// union's own status word, for every request of the union).
__global__ void k_lane_scatter(const LaneDesc *d, const int32_t *uo, const int64_t *ucnt,
                               const uint32_t *flags, int32_t *stat)
{
    __shared__ uint32_t s_lo, s_hi;
    const LaneDesc q = d[blockIdx.x];
    if (threadIdx.x == 0) {
        const uint32_t total = (uint32_t)*ucnt;
        s_lo = lower_pos(uo, total, q.ebase);
        s_hi = lower_pos(uo, total, q.ebase + q.m);
    }
    __syncthreads();
    const uint32_t lo = s_lo, k = s_hi - s_lo;
    const uint32_t cap = q.n > 0 ? q.n - 1 : 0;
    for (uint32_t i = threadIdx.x; i < k && i < cap; i += blockDim.x)
        q.out[i] = uo[lo + i] - (int32_t)q.ebase;
    if (threadIdx.x == 0) {
        *q.out_count = (int64_t)(k < cap ? k : cap);
        int32_t code = MST_OK;
        if (flags[blockIdx.x])
            code = MST_ERR_INVALID_ARG;
        else if (k > cap)
            code = MST_ERR_INTERNAL;
        else if (q.n > 0 && k != cap)
            code = MST_ERR_DISCONNECTED;
        stat[blockIdx.x] = code;
    }
}

// Layout of the lane union's buffer: descriptors, flags and statuses of up
// to kLaneBatch requests, the union's count, copies of its edge arrays and
// its output.
static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
static size_t union_head()
{
    return al256(sizeof(LaneDesc) * kLaneBatch) + 2 * al256(4 * kLaneBatch) + al256(8);
}
static size_t union_bytes(uint64_t n_u, uint64_t m_u)
{
    return union_head() + 3 * al256(4 * m_u) + al256(4 * (n_u > 0 ? n_u : 1));
}
static int32_t *union_stat(void *base)
{
    return (int32_t *)((char *)base + al256(sizeof(LaneDesc) * kLaneBatch) + al256(4 * kLaneBatch));
}

// Workspace of one request inside a batch (edge list, vertex arrays, bits).
static size_t request_bytes(uint32_t n, uint32_t m)
{
    return (size_t)m * 16 + (size_t)n * 28 + ((size_t)m / 32 + 2) * 4 + 64;
}

// Each request gets the status of its own solve, as mst_solve_ex would
// report it for that graph alone (a forest is MST_ERR_DISCONNECTED, a bad
// vertex id or NaN weight MST_ERR_INVALID_ARG), never a batch-mate's.
static void complete_slot(Server &S, Slot &sl)
{
    const double t = now_us();
    std::vector<uint32_t> bits(sl.tickets.size(), 0u);
    cudaError_t e = cudaSuccess;
    std::vector<int32_t> lane_stat;
    if (sl.big) {
        e = cudaMemcpy(bits.data(), &S.lane.ws.ctl->status, sizeof(uint32_t),
                       cudaMemcpyDeviceToHost);
        if (sl.lane_k > 0 && e == cudaSuccess) {  // a union: each request's own status
            lane_stat.resize(sl.lane_k);
            e = cudaMemcpy(lane_stat.data(), union_stat(S.ubuf), sl.lane_k * sizeof(int32_t),
                           cudaMemcpyDeviceToHost);
        }
    } else {
        if (!bits.empty())
            e = desc_batch_graph_status(sl.ws, (int32_t)bits.size(), sl.total_n, sl.total_m,
                                        bits.data());
        cudaFreeAsync(sl.ws, sl.stream);
    }
    std::lock_guard<std::mutex> lk(S.mu);
    for (size_t i = 0; i < sl.tickets.size(); i++) {
        const uint64_t tk = sl.tickets[i];
        Outcome &o = S.results[tk];
        o.done = true;
        o.latency_us = t - S.submit_us[tk];
        if (e != cudaSuccess)
            o.status = MST_ERR_CUDA;
        else if (!lane_stat.empty())  // a wait that ran out concerns the whole union
            o.status = (bits[0] & (ST_TIMEOUT | ST_INTERNAL))
                           ? status_from_bits(bits[0] & (ST_TIMEOUT | ST_INTERNAL))
                           : (mst_status)lane_stat[i];
        else
            o.status = status_from_bits(bits[i]);
        S.submit_us.erase(tk);
    }
    if (!sl.big)
        S.in_use -= sl.ws_bytes;
    else
        S.big_inflight = false;
    S.inflight--;
    sl.tickets.clear();
    sl.ws = nullptr;
    sl.ws_bytes = 0;
    sl.big = false;
    sl.lane_k = 0;
    sl.busy = false;
    S.cv.notify_all();
}

// Takes queued requests for one launch (lock held).  Large requests form
// their own FIFO lane with at most one in flight; that lane also takes the
// oldest medium request, which one CTA of a batch would solve several times
// slower.  A medium request goes to a batch only when kServeLaneDepth
// requests for the lane are queued ahead of it.  The fused kernel's grid
// barrier needs all of its CTAs resident at once, and two fused grids that
// are each partly resident would wait on each other until the barrier gives
// up.  One fused grid next to batched kernels (which never wait on anything)
// always completes.  Small requests are batched in arrival order, passing
// large ones that wait for the lane.  Requests that can never fit the budget
// are completed at once with MST_ERR_BUDGET.
static void reject(Server &S, std::deque<Request>::iterator it)
{
    Outcome &o = S.results[it->ticket];
    o.done = true;
    o.status = MST_ERR_BUDGET;
    S.submit_us.erase(it->ticket);
}

static std::vector<Request> take_batch(Server &S, Slot &sl, size_t budget, bool *big)
{
    std::vector<Request> batch;
    *big = false;
    if (!S.big_inflight) {
        for (auto it = S.pending.begin(); it != S.pending.end();) {
            if (it->m <= kServeMidM) {
                ++it;
                continue;
            }
            const bool large = it->m > kServeBigM;  // else a batch may take it
            const size_t have = S.lane.base ? S.lane.bytes : 0;
            const size_t need = single_bytes((uint32_t)std::max<int64_t>(it->n, 1024),
                                             (uint32_t)std::max<int64_t>(it->m, 1024));
            if (budget && need > budget && large) {  // can never be admitted
                reject(S, it);
                it = S.pending.erase(it);
                continue;
            }
            if (budget && need > have && S.in_use + need > budget && !S.retired.empty()) {
                for (auto &r : S.retired) {  // rare: free outgrown workspaces (waits for the GPU)
                    cudaFree(r.first);
                    S.in_use -= r.second;
                }
                S.retired.clear();
            }
            if (budget && need > have && S.in_use + need > budget) {
                ++it;  // wait for memory (a medium one goes to a batch instead)
                continue;
            }
            batch.push_back(*it);
            it = S.pending.erase(it);
            *big = true;
            // more requests of the same weight type join the union, in
            // arrival order, while it stays within kLaneBatch requests,
            // kLaneMaxM edges and the memory budget
            int64_t n_u = batch[0].n, m_u = batch[0].m;
            const size_t have_u = S.ubuf ? S.ubuf_bytes : 0;
            for (auto jt = it; jt != S.pending.end() && (int)batch.size() < kLaneBatch;) {
                if (jt->m <= kServeMidM || jt->wt != batch[0].wt || m_u + jt->m > kLaneMaxM ||
                    n_u + jt->n > (int64_t)INT32_MAX) {
                    ++jt;
                    continue;
                }
                const int64_t n2 = n_u + jt->n, m2 = m_u + jt->m;
                const size_t need2 = single_bytes((uint32_t)std::max<int64_t>(n2, 1024),
                                                  (uint32_t)std::max<int64_t>(m2, 1024));
                const size_t needu = union_bytes((uint64_t)n2, (uint64_t)m2);
                const size_t grow =
                    (need2 > have ? need2 - have : 0) + (needu > have_u ? needu - have_u : 0);
                if (budget && S.in_use + grow > budget) {
                    ++jt;
                    continue;
                }
                batch.push_back(*jt);
                jt = S.pending.erase(jt);
                n_u = n2;
                m_u = m2;
            }
            return batch;
        }
    }
    size_t bytes = 4096 + 64 * 4;  // control block and order list slack
    int lane_ahead = 0;            // requests queued for the lane so far
    for (auto it = S.pending.begin(); it != S.pending.end() && (int)batch.size() < S.max_batch;) {
        if (it->m > kServeBigM || (it->m > kServeMidM && lane_ahead < kServeLaneDepth)) {
            lane_ahead += it->m > kServeMidM ? 1 : 0;
            ++it;
            continue;
        }
        const size_t need = request_bytes((uint32_t)it->n, (uint32_t)it->m);
        if (budget && need + 4096 > budget) {  // can never be admitted
            reject(S, it);
            it = S.pending.erase(it);
            continue;
        }
        if (budget && S.in_use + bytes + need > budget)
            break;
        bytes += need;
        batch.push_back(*it);
        it = S.pending.erase(it);
    }
    return batch;
}

// A large request on the slot's fused-kernel workspace (grown if needed).
// The lane's requests: one alone is solved in place; several are solved as
// one union graph (see k_lane_gather / k_lane_scatter).
static cudaError_t launch_lane(Server &S, Slot &sl, const std::vector<Request> &reqs, bool alone);

static cudaError_t launch_big(Server &S, Slot &sl, const Request &r, bool alone)
{
    const uint32_t n = (uint32_t)r.n, m = (uint32_t)r.m;
    Single &lane = S.lane;
    if (!lane.base || n > lane.ws.n_cap || m > lane.ws.m_cap) {
        // The old workspace is kept until the server stops: freeing it now
        // would wait for every stream of the device, batches included.  The
        // new one grows geometrically (within the budget), so this happens
        // a few times per server at most.
        uint32_t n2 = n, m2 = m;
        if (lane.base) {
            S.retired.emplace_back(lane.base, lane.bytes);
            lane.base = nullptr;
            n2 = std::max<uint64_t>(n, std::min<uint64_t>(2ull * lane.ws.n_cap, 0x7fffffffu));
            m2 = std::max<uint64_t>(m, std::min<uint64_t>(2ull * lane.ws.m_cap, 0x7fffffffu));
            const size_t budget = S.h->budget;
            if (budget && S.in_use + single_bytes(n2, m2) > budget) {
                n2 = n;
                m2 = m;
            }
        }
        lane.schedule = 1;  // fixed shape: the grid is chosen per launch below
        lane.fused_blocks_per_sm = 4;
        lane.fused_threads = 256;
        cudaError_t e = single_reserve(lane, S.h->device, n2, m2);
        std::lock_guard<std::mutex> lk(S.mu);
        S.in_use += lane.base ? lane.bytes : 0;
        if (e != cudaSuccess)
            return e;
    }
    if (n == 0)
        return cudaMemsetAsync(r.out_count, 0, sizeof(int64_t), sl.stream);
    // the whole co-resident grid when nothing else runs, else half of it
    // (two CTAs per SM), which leaves room for batches on the other slots
    const int grid = alone ? lane.grid_fused : lane.grid_fused / 2;
    cudaError_t e = single_launch(lane, r.src, r.dst, r.w, r.wt, r.out, r.out_count, n, m,
                                  sl.stream, grid);
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.done, sl.stream);
    sl.tickets.assign(1, r.ticket);
    return e;
}

static cudaError_t launch_lane(Server &S, Slot &sl, const std::vector<Request> &reqs, bool alone)
{
    if (reqs.size() == 1)
        return launch_big(S, sl, reqs[0], alone);
    const int k = (int)reqs.size();
    uint64_t n_u = 0, m_u = 0;
    for (const Request &r : reqs) {
        n_u += (uint64_t)r.n;
        m_u += (uint64_t)r.m;
    }
    // the union's buffer (an outgrown one is kept until the server stops, as
    // the lane workspaces are: freeing it now would wait for every stream)
    const size_t need = union_bytes(n_u, m_u);
    if (!S.ubuf || need > S.ubuf_bytes) {
        std::lock_guard<std::mutex> lk(S.mu);
        const size_t grow = std::max(need, 2 * S.ubuf_bytes);
        if (S.ubuf)
            S.retired.emplace_back(S.ubuf, S.ubuf_bytes);
        S.ubuf = nullptr;
        S.ubuf_bytes = 0;
        cudaError_t e = cudaMalloc(&S.ubuf, grow);
        if (e != cudaSuccess) {
            S.ubuf = nullptr;
            return e;
        }
        S.ubuf_bytes = grow;
        S.in_use += grow;
    }
    if (!sl.h_lane) {
        cudaError_t e = cudaMallocHost((void **)&sl.h_lane, sizeof(LaneDesc) * kLaneBatch);
        if (e != cudaSuccess) {
            sl.h_lane = nullptr;
            return e;
        }
    }
    char *p = (char *)S.ubuf;
    LaneDesc *d_desc = (LaneDesc *)p;
    p += al256(sizeof(LaneDesc) * kLaneBatch);
    uint32_t *flags = (uint32_t *)p;
    p += al256(4 * kLaneBatch);
    int32_t *stat = (int32_t *)p;
    p += al256(4 * kLaneBatch);
    int64_t *ucnt = (int64_t *)p;
    p += al256(8);
    int32_t *us = (int32_t *)p;
    p += al256(4 * m_u);
    int32_t *ud = (int32_t *)p;
    p += al256(4 * m_u);
    uint32_t *uw = (uint32_t *)p;
    p += al256(4 * m_u);
    int32_t *uo = (int32_t *)p;
    uint32_t vb = 0, eb = 0, max_m = 1;
    for (int i = 0; i < k; i++) {
        const Request &r = reqs[i];
        sl.h_lane[i] = LaneDesc{r.src, r.dst, (const uint32_t *)r.w, r.out, r.out_count,
                                (uint32_t)r.n, (uint32_t)r.m, vb, eb};
        vb += (uint32_t)r.n;
        eb += (uint32_t)r.m;
        max_m = std::max<uint32_t>(max_m, (uint32_t)r.m);
    }
    cudaError_t e = cudaMemcpyAsync(d_desc, sl.h_lane, sizeof(LaneDesc) * k,
                                    cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(flags, 0, 4 * kLaneBatch, sl.stream);
    if (e != cudaSuccess)
        return e;
    const uint32_t gx = std::min<uint32_t>((max_m + 1023) / 1024, 256);
    k_lane_gather<<<dim3(gx, k), 256, 0, sl.stream>>>(d_desc, reqs[0].wt, us, ud, uw, flags);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    // the union, solved by the fused kernel in the lane workspace
    Request u = reqs[0];
    u.n = (int32_t)n_u;
    u.m = (int64_t)m_u;
    u.src = us;
    u.dst = ud;
    u.w = uw;
    u.out = uo;
    u.out_count = ucnt;
    e = launch_big(S, sl, u, alone);
    if (e != cudaSuccess)
        return e;
    k_lane_scatter<<<k, 256, 0, sl.stream>>>(d_desc, uo, ucnt, flags, stat);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.done, sl.stream);  // after the cut-out
    sl.tickets.clear();
    for (const Request &r : reqs)
        sl.tickets.push_back(r.ticket);
    sl.lane_k = k;
    return e;
}

static cudaError_t launch_batch(Server &S, Slot &sl, std::vector<Request> &batch)
{
    const int G = (int)batch.size();
    if (G > sl.cap) {
        if (sl.h_desc)
            cudaFreeHost(sl.h_desc);
        if (sl.d_desc)
            cudaFree(sl.d_desc);
        sl.cap = std::max(G, 2 * sl.cap);
        cudaError_t e = cudaMallocHost((void **)&sl.h_desc, sizeof(GraphDesc) * sl.cap);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&sl.d_desc, sizeof(GraphDesc) * sl.cap);
        if (e != cudaSuccess)
            return e;
    }
    uint64_t vo = 0, eo = 0;
    for (int i = 0; i < G; i++) {
        const Request &r = batch[i];
        GraphDesc &d = sl.h_desc[i];
        d.src = r.src;
        d.dst = r.dst;
        d.w = r.w;
        d.out = r.out;
        d.out_count = r.out_count;
        d.n = (uint32_t)r.n;
        d.m = (uint32_t)r.m;
        d.wt = r.wt;
        d.pad = 0;
        d.ws_vo = vo;
        d.ws_eo = eo;
        vo += (uint64_t)r.n;
        eo += (uint64_t)r.m;
    }
    const size_t bytes = desc_batch_bytes(G, vo, eo);
    cudaError_t e = cudaMallocAsync(&sl.ws, bytes, sl.stream);
    if (e != cudaSuccess)
        return e;
    sl.ws_bytes = bytes;
    sl.total_n = vo;
    sl.total_m = eo;
    e = cudaMemcpyAsync(sl.d_desc, sl.h_desc, sizeof(GraphDesc) * G, cudaMemcpyHostToDevice,
                        sl.stream);
    if (e == cudaSuccess)
        e = batched_launch_desc(S.h->batched, S.h->device, sl.ws, G, sl.d_desc, vo, eo, sl.stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.done, sl.stream);
    sl.tickets.clear();
    for (const Request &r : batch)
        sl.tickets.push_back(r.ticket);
    return e;
}

static void server_loop(Server *Sp)
{
    Server &S = *Sp;
    cudaSetDevice(S.h->device);
    const size_t budget = S.h->budget;
    for (;;) {
        // retire finished batches
        for (Slot &sl : S.slots)
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess)
                complete_slot(S, sl);
        std::unique_lock<std::mutex> lk(S.mu);
        if (S.stop && S.pending.empty() && S.inflight == 0)
            break;
        Slot *free_slot = nullptr;
        for (Slot &sl : S.slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        std::vector<Request> batch;
        bool big = false;
        if (free_slot && !S.pending.empty())
            batch = take_batch(S, *free_slot, budget, &big);
        if (batch.empty()) {
            S.cv.notify_all();
            // nothing to launch: wait for a submit or poll the busy slots soon
            S.cv.wait_for(lk, std::chrono::microseconds(S.inflight ? 20 : 2000));
            continue;
        }
        size_t bytes = 0;
        if (!big)
            for (const Request &r : batch)
                bytes += request_bytes((uint32_t)r.n, (uint32_t)r.m);
        if (!big)
            S.in_use += bytes + 4096;
        const bool alone = S.inflight == 0;
        S.inflight++;
        S.big_inflight |= big;
        free_slot->busy = true;
        free_slot->big = big;
        lk.unlock();
        cudaError_t e =
            big ? launch_lane(S, *free_slot, batch, alone) : launch_batch(S, *free_slot, batch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> g(S.mu);
            S.error = e;
            for (const Request &r : batch) {
                Outcome &o = S.results[r.ticket];
                o.done = true;
                o.status = e == cudaErrorMemoryAllocation ? MST_ERR_OOM : MST_ERR_CUDA;
            }
            if (!big)
                S.in_use -= bytes + 4096;
            else
                S.big_inflight = false;
            S.inflight--;
            free_slot->busy = false;
            free_slot->big = false;
            free_slot->lane_k = 0;
            free_slot->tickets.clear();
            if (free_slot->ws) {
                cudaFreeAsync(free_slot->ws, free_slot->stream);
                free_slot->ws = nullptr;
            }
        } else if (!big) {
            free_slot->ws_bytes = bytes + 4096;  // the admission charge
        }
    }
}

mst_status server_start(mst_handle h, int streams, int max_batch)
{
    if (h->server)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    Server *S = new Server();
    S->h = h;
    S->max_batch = max_batch;
    S->slots.resize(streams);
    for (Slot &sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            delete S;
            return MST_ERR_CUDA;
        }
    }
    // The lane's workspace and the union buffer are sized up front for the
    // largest union (when the budget leaves room for them four times over):
    // growing them later calls cudaMalloc, which can wait for the whole
    // device, so every request in flight would see the stall (measured: at
    // 2,000 graphs/s on the C5 shape, p99 41 ms with growth on demand).
    const size_t lane_b = single_bytes(kLaneMaxN, (uint32_t)kLaneMaxM);
    const size_t union_b = union_bytes(kLaneMaxN, (uint64_t)kLaneMaxM);
    if (!h->budget || 4 * (lane_b + union_b) <= h->budget) {
        S->lane.schedule = 1;
        S->lane.fused_blocks_per_sm = 4;
        S->lane.fused_threads = 256;
        if (single_reserve(S->lane, h->device, kLaneMaxN, (uint32_t)kLaneMaxM) == cudaSuccess &&
            cudaMalloc(&S->ubuf, union_b) == cudaSuccess) {
            S->ubuf_bytes = union_b;
            S->in_use += S->lane.bytes + union_b;
        } else {  // no room: grow on demand instead
            cudaGetLastError();
            single_release(S->lane);
            S->ubuf = nullptr;
        }
    }
    for (Slot &sl : S->slots)
        if (cudaMallocHost((void **)&sl.h_lane, sizeof(LaneDesc) * kLaneBatch) != cudaSuccess) {
            cudaGetLastError();
            sl.h_lane = nullptr;
        }
    h->server = S;
    S->thr = std::thread(server_loop, S);
    return MST_OK;
}

mst_status server_submit(mst_handle h, const Request &r, uint64_t *ticket)
{
    Server *S = h->server;
    if (!S)
        return MST_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop)
        return MST_ERR_INVALID_ARG;
    Request q = r;
    q.ticket = S->next_ticket++;
    S->submit_us[q.ticket] = q.t_submit_us;
    S->results[q.ticket] = Outcome();
    S->pending.push_back(q);
    *ticket = q.ticket;
    S->cv.notify_all();
    return MST_OK;
}

mst_status server_poll(mst_handle h, uint64_t ticket, int *done, double *latency_us)
{
    Server *S = h->server;
    if (!S)
        return MST_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end())
        return MST_ERR_INVALID_ARG;
    *done = it->second.done ? 1 : 0;
    if (!it->second.done)
        return MST_OK;
    if (latency_us)
        *latency_us = it->second.latency_us;
    const mst_status st = it->second.status;
    S->results.erase(it);
    return st;
}

mst_status server_drain(mst_handle h)
{
    Server *S = h->server;
    if (!S)
        return MST_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv.wait(lk, [&] { return S->pending.empty() && S->inflight == 0; });
    return S->error == cudaSuccess ? MST_OK : MST_ERR_CUDA;
}

mst_status server_stop(mst_handle h)
{
    Server *S = h->server;
    if (!S)
        return MST_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    S->thr.join();
    cudaSetDevice(h->device);
    for (Slot &sl : S->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        if (sl.done)
            cudaEventDestroy(sl.done);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
        if (sl.h_desc)
            cudaFreeHost(sl.h_desc);
        if (sl.d_desc)
            cudaFree(sl.d_desc);
        if (sl.h_lane)
            cudaFreeHost(sl.h_lane);
    }
    single_release(S->lane);
    if (S->ubuf)
        cudaFree(S->ubuf);
    for (auto &r : S->retired)
        cudaFree(r.first);
    const mst_status st = S->error == cudaSuccess ? MST_OK : MST_ERR_CUDA;
    delete S;
    h->server = nullptr;
    return st;
}

}  // namespace mst
