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
// The lane solves one such request at a time, on a slot's stream, with the
// fused multi-CTA single-graph kernel in the server's one lane workspace:
// on the whole co-resident grid when nothing else is in flight, else on
// half of it, while other slots keep serving batches.
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
    if (sl.big) {
        e = cudaMemcpy(bits.data(), &S.lane.ws.ctl->status, sizeof(uint32_t),
                       cudaMemcpyDeviceToHost);
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
        o.status = e != cudaSuccess ? MST_ERR_CUDA : status_from_bits(bits[i]);
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
            S.pending.erase(it);
            *big = true;
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
            big ? launch_big(S, *free_slot, batch[0], alone) : launch_batch(S, *free_slot, batch);
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
    }
    single_release(S->lane);
    for (auto &r : S->retired)
        cudaFree(r.first);
    const mst_status st = S->error == cudaSuccess ? MST_OK : MST_ERR_CUDA;
    delete S;
    h->server = nullptr;
    return st;
}

}  // namespace mst
