// mst_api.cu — the extern "C" entry points of libmst (see include/mst.h):
// argument validation, handle and workspace ownership, status reporting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <chrono>
#include <new>

#include "mst_internal.h"

namespace mst {

double now_us()
{
    using namespace std::chrono;
    return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

mst_status status_from_bits(uint32_t bits) { return status_code(bits); }

static mst_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return MST_OK;
    if (e == cudaErrorMemoryAllocation)
        return MST_ERR_OOM;
    return MST_ERR_CUDA;
}

}  // namespace mst

using namespace mst;

extern "C" {

const char *mst_status_string(mst_status s)
{
    switch (s) {
    case MST_OK: return "MST_OK";
    case MST_ERR_INVALID_ARG: return "MST_ERR_INVALID_ARG";
    case MST_ERR_OOM: return "MST_ERR_OOM";
    case MST_ERR_CUDA: return "MST_ERR_CUDA";
    case MST_ERR_DISCONNECTED: return "MST_ERR_DISCONNECTED";
    case MST_ERR_TIMEOUT: return "MST_ERR_TIMEOUT";
    case MST_ERR_BUDGET: return "MST_ERR_BUDGET";
    case MST_ERR_INTERNAL: return "MST_ERR_INTERNAL";
    }
    return "MST_ERR_UNKNOWN";
}

mst_status mst_create(mst_handle *h, int device, size_t mem_budget_bytes)
{
    if (!h)
        return MST_ERR_INVALID_ARG;
    *h = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess)
        return MST_ERR_CUDA;
    mst_handle_s *p = new (std::nothrow) mst_handle_s();
    if (!p)
        return MST_ERR_OOM;
    p->device = device;
    p->budget = mem_budget_bytes;
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, device);
    *h = p;
    return MST_OK;
}

mst_status mst_destroy(mst_handle h)
{
    if (!h)
        return MST_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    if (h->server)
        server_stop(h);
    cudaDeviceSynchronize();
    single_release(h->single);
    batched_release(h->batched);
    if (h->staging)
        cudaFree(h->staging);
    if (h->csr_rows)
        cudaFree(h->csr_rows);
    for (cudaStream_t cs : h->copy_stream)
        if (cs)
            cudaStreamDestroy(cs);
    for (cudaEvent_t ev : h->copy_event)
        if (ev)
            cudaEventDestroy(ev);
    delete h;
    return MST_OK;
}

// Bytes the handle holds outside the single and batched workspaces: the
// host-buffer staging and the CSR row buffer (all counted in the budget).
static size_t aux_bytes(const mst_handle h)
{
    return h->staging_bytes + h->csr_cap * sizeof(int32_t);
}

static mst_status check_graph_args(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                   const void *w, int32_t *out, int64_t *out_count)
{
    if (n < 0 || m < 0 || m > INT32_MAX)
        return MST_ERR_INVALID_ARG;
    if (!out_count)
        return MST_ERR_INVALID_ARG;
    if (m > 0 && (!src || !dst || !w))
        return MST_ERR_INVALID_ARG;
    if (n > 1 && !out)
        return MST_ERR_INVALID_ARG;
    if (n == 0 && m > 0)
        return MST_ERR_INVALID_ARG;  // no vertex id can be valid
    return MST_OK;
}

// One single-graph solve (arguments already checked, device set).  With
// `copy`, src/dst/w are mapped host memory that round 0 reads once while
// writing the device copy the later phases use.
static mst_status solve_single(mst_handle h, mst_weight_type wt, int32_t n, int64_t m,
                               const int32_t *src, const int32_t *dst, const void *w,
                               int32_t *out_edge_ids, int64_t *out_count, cudaStream_t s,
                               const InputCopy *copy)
{
    if (n == 0) {
        // nothing to do: zero edges, status cleared
        h->last = LAST_SINGLE;
        if (h->single.base) {
            if (cudaMemsetAsync(&h->single.ws.ctl->status, 0, sizeof(uint32_t), s) != cudaSuccess)
                return MST_ERR_CUDA;
        }
        return cuda_status(cudaMemsetAsync(out_count, 0, sizeof(int64_t), s));
    }
    const uint32_t nn = (uint32_t)n, mm = (uint32_t)m;
    if (!h->single.base || nn > h->single.ws.n_cap || mm > h->single.ws.m_cap) {
        uint32_t n_cap = nn > h->single.ws.n_cap ? nn : h->single.ws.n_cap;
        uint32_t m_cap = mm > h->single.ws.m_cap ? mm : h->single.ws.m_cap;
        if (h->budget && single_bytes(n_cap < 1024 ? 1024 : n_cap, m_cap < 1024 ? 1024 : m_cap) +
                                 h->batched.bytes + aux_bytes(h) > h->budget)
            return MST_ERR_BUDGET;
        cudaStreamSynchronize(s);  // workspace may be in use by earlier work
        cudaError_t e = single_reserve(h->single, h->device, nn, mm);
        if (e != cudaSuccess) {
            single_release(h->single);
            cudaGetLastError();
            return cuda_status(e);
        }
    }
    h->last = LAST_SINGLE;
    if (copy)  // a replay reads the device copy
        h->last_solve = LastSolve{copy->src, copy->dst, copy->w, out_edge_ids, out_count, nn, mm,
                                  (uint32_t)wt, true};
    else
        h->last_solve = LastSolve{src, dst, w, out_edge_ids, out_count, nn, mm, (uint32_t)wt, true};
    return cuda_status(single_launch(h->single, src, dst, w, (uint32_t)wt, out_edge_ids, out_count,
                                     nn, mm, s, 0, copy));
}

mst_status mst_solve_ex(mst_handle h, mst_weight_type wt, int32_t n, int64_t m,
                        const int32_t *src, const int32_t *dst, const void *w,
                        int32_t *out_edge_ids, int64_t *out_count, void *stream)
{
    if (!h || (wt != MST_W_U32 && wt != MST_W_F32))
        return MST_ERR_INVALID_ARG;
    mst_status st = check_graph_args(n, m, src, dst, w, out_edge_ids, out_count);
    if (st != MST_OK)
        return st;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    return solve_single(h, wt, n, m, src, dst, w, out_edge_ids, out_count, (cudaStream_t)stream,
                        nullptr);
}

mst_status mst_solve_csr(mst_handle h, mst_weight_type wt, int32_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col, const void *w,
                         uint32_t flags, int32_t *out_edge_ids, int64_t *out_count, void *stream)
{
    if (!h || (wt != MST_W_U32 && wt != MST_W_F32) || (flags & ~(uint32_t)MST_CSR_SYMMETRIC))
        return MST_ERR_INVALID_ARG;
    mst_status st = check_graph_args(n, nnz, col, col, w, out_edge_ids, out_count);
    if (st != MST_OK)
        return st;
    if (nnz > 0 && !row_ptr)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if ((size_t)nnz > h->csr_cap) {
        const size_t bytes = (size_t)nnz * sizeof(int32_t);
        if (h->budget && bytes + h->staging_bytes + h->single.bytes + h->batched.bytes > h->budget)
            return MST_ERR_BUDGET;
        cudaStreamSynchronize(s);  // the old buffer may be in use by earlier work
        if (h->csr_rows)
            cudaFree(h->csr_rows);
        h->csr_rows = nullptr;
        h->csr_cap = 0;
        if (cudaMalloc(&h->csr_rows, bytes) != cudaSuccess) {
            cudaGetLastError();
            return MST_ERR_OOM;
        }
        h->csr_cap = (size_t)nnz;
    }
    if (nnz > 0) {
        cudaError_t e = csr_rows(row_ptr, col, (uint32_t)n, (uint32_t)nnz,
                                 (flags & MST_CSR_SYMMETRIC) != 0, h->csr_rows, h->num_sms, s);
        if (e != cudaSuccess)
            return cuda_status(e);
    }
    return solve_single(h, wt, n, nnz, nnz > 0 ? h->csr_rows : nullptr, col, w, out_edge_ids,
                        out_count, s, nullptr);
}

mst_status mst_solve_host(mst_handle h, mst_weight_type wt, int32_t n, int64_t m,
                          const int32_t *src, const int32_t *dst, const void *w,
                          int32_t *out_edge_ids, int64_t *out_count, void *stream)
{
    if (!h || (wt != MST_W_U32 && wt != MST_W_F32))
        return MST_ERR_INVALID_ARG;
    mst_status st = check_graph_args(n, m, src, dst, w, out_edge_ids, out_count);
    if (st != MST_OK)
        return st;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t eb = (size_t)m * 4;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t need = 3 * al(eb) + al((size_t)(n > 1 ? n - 1 : 1) * 4) + al(8);
    if (need > h->staging_bytes) {
        if (h->budget && need + h->csr_cap * sizeof(int32_t) + h->single.bytes +
                                 h->batched.bytes > h->budget)
            return MST_ERR_BUDGET;
        cudaStreamSynchronize(s);
        if (h->staging)
            cudaFree(h->staging);
        h->staging = nullptr;
        h->staging_bytes = 0;
        if (cudaMalloc(&h->staging, need) != cudaSuccess) {
            cudaGetLastError();
            return MST_ERR_OOM;
        }
        h->staging_bytes = need;
    }
    char *p = (char *)h->staging;
    int32_t *d_src = (int32_t *)p;
    int32_t *d_dst = (int32_t *)(p + al(eb));
    void *d_w = (void *)(p + 2 * al(eb));
    int32_t *d_out = (int32_t *)(p + 3 * al(eb));
    int64_t *d_cnt = (int64_t *)(p + 3 * al(eb) + al((size_t)(n > 1 ? n - 1 : 1) * 4));
    // Pinned (page-locked, mapped) inputs are read by the fused kernel itself
    // in round 0, over the host link, while it writes the device copy: no
    // separate copy pass.  Other host memory is copied in first.
    const void *mapped[3] = {nullptr, nullptr, nullptr};
    bool zero_copy = m > 0 && h->single.schedule != 2;
    const void *hp[3] = {src, dst, w};
    for (int i = 0; i < 3 && zero_copy; i++) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, hp[i]) != cudaSuccess) {
            cudaGetLastError();
            zero_copy = false;
        } else if (a.type != cudaMemoryTypeHost || !a.devicePointer) {
            zero_copy = false;
        } else {
            mapped[i] = a.devicePointer;
        }
    }
    // pinned outputs are written by the kernel itself (no copy back)
    void *out_mapped[2] = {nullptr, nullptr};
    bool direct_out = zero_copy;
    void *op[2] = {out_edge_ids, out_count};
    for (int i = 0; i < 2 && direct_out; i++) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, op[i]) != cudaSuccess) {
            cudaGetLastError();
            direct_out = false;
        } else if (a.type != cudaMemoryTypeHost || !a.devicePointer) {
            direct_out = false;
        } else {
            out_mapped[i] = a.devicePointer;
        }
    }
    if (zero_copy) {
        const InputCopy copy{d_src, d_dst, d_w};
        int32_t *o = direct_out ? (int32_t *)out_mapped[0] : d_out;
        int64_t *oc = direct_out ? (int64_t *)out_mapped[1] : d_cnt;
        st = solve_single(h, wt, n, m, (const int32_t *)mapped[0], (const int32_t *)mapped[1],
                          mapped[2], o, oc, s, &copy);
        if (st != MST_OK)
            return st;
        if (direct_out)
            return mst_get_status(h, stream);
    } else if (m > 0) {
        // the three input arrays are copied side by side on three streams
        // (several copy engines), after the caller's stream and before the solve
        if (!h->copy_stream[0]) {
            for (cudaStream_t &cs : h->copy_stream)
                if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
                    return MST_ERR_CUDA;
            for (cudaEvent_t &ev : h->copy_event)
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                    return MST_ERR_CUDA;
        }
        cudaStream_t c1 = h->copy_stream[0], c2 = h->copy_stream[1];
        if (cudaEventRecord(h->copy_event[0], s) != cudaSuccess ||
            cudaStreamWaitEvent(c1, h->copy_event[0], 0) != cudaSuccess ||
            cudaStreamWaitEvent(c2, h->copy_event[0], 0) != cudaSuccess ||
            cudaMemcpyAsync(d_src, src, eb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_dst, dst, eb, cudaMemcpyHostToDevice, c1) != cudaSuccess ||
            cudaMemcpyAsync(d_w, w, eb, cudaMemcpyHostToDevice, c2) != cudaSuccess ||
            cudaEventRecord(h->copy_event[1], c1) != cudaSuccess ||
            cudaEventRecord(h->copy_event[2], c2) != cudaSuccess ||
            cudaStreamWaitEvent(s, h->copy_event[1], 0) != cudaSuccess ||
            cudaStreamWaitEvent(s, h->copy_event[2], 0) != cudaSuccess)
            return MST_ERR_CUDA;
    }
    if (!zero_copy) {
        st = mst_solve_ex(h, wt, n, m, d_src, d_dst, d_w, d_out, d_cnt, stream);
        if (st != MST_OK)
            return st;
    }
    if (n > 1 && cudaMemcpyAsync(out_edge_ids, d_out, (size_t)(n - 1) * 4, cudaMemcpyDeviceToHost,
                                 s) != cudaSuccess)
        return MST_ERR_CUDA;
    if (cudaMemcpyAsync(out_count, d_cnt, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MST_ERR_CUDA;
    return mst_get_status(h, stream);
}

mst_status mst_profile_last_solve(mst_handle h, void *stream, mst_kernel_profile *out,
                                  int32_t cap, int32_t *count)
{
    if (!h || !count || cap < 0 || (cap > 0 && !out))
        return MST_ERR_INVALID_ARG;
    *count = 0;
    if (!h->last_solve.valid || !h->single.base)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    const LastSolve &L = h->last_solve;
    std::vector<KernelProfile> prof;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return MST_ERR_CUDA;
    cudaError_t e = h->single.schedule == 2
                        ? single_profile(h->single, L.src, L.dst, L.w, L.wt, L.out, L.out_count,
                                         L.n, L.m, s, prof)
                        : single_phase_profile(h->single, s, prof);
    if (e != cudaSuccess)
        return cuda_status(e);
    int32_t k = 0;
    for (const auto &p : prof) {
        if (k >= cap)
            break;
        mst_kernel_profile &o = out[k++];
        snprintf(o.name, sizeof(o.name), "%s", p.name.c_str());
        o.launches = p.launches;
        o.total_ms = p.ms;
        o.alg_bytes = p.bytes;
    }
    *count = k;
    h->last = LAST_SINGLE;
    return MST_OK;
}

mst_status mst_solve(mst_handle h, int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const void *w, int32_t *out_edge_ids, int64_t *out_count, void *stream)
{
    return mst_solve_ex(h, MST_W_U32, n, m, src, dst, w, out_edge_ids, out_count, stream);
}

mst_status mst_get_status(mst_handle h, void *stream)
{
    if (!h)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return MST_ERR_CUDA;
    if (h->last == LAST_SINGLE) {
        if (!h->single.base)
            return MST_OK;
        uint32_t bits = 0;
        if (cudaMemcpy(&bits, &h->single.ws.ctl->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MST_ERR_CUDA;
        return status_from_bits(bits);
    }
    if (h->last == LAST_BATCHED) {
        cudaError_t err = cudaSuccess;
        uint32_t bits = batched_status_bits(h->batched, s, &err);
        if (err != cudaSuccess)
            return MST_ERR_CUDA;
        return status_from_bits(bits);
    }
    return MST_OK;
}

mst_status mst_get_batched_status(mst_handle h, void *stream, int32_t G, int32_t *statuses)
{
    if (!h || G < 0 || (G > 0 && !statuses))
        return MST_ERR_INVALID_ARG;
    if (G == 0)
        return MST_OK;
    if (h->last != LAST_BATCHED || G > h->batched.last_G || !h->batched.base)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    std::vector<uint32_t> bits((size_t)G);
    if (batched_graph_status(h->batched, (cudaStream_t)stream, G, bits.data()) != cudaSuccess)
        return MST_ERR_CUDA;
    for (int32_t g = 0; g < G; g++)
        statuses[g] = (int32_t)status_from_bits(bits[(size_t)g]);
    return MST_OK;
}

mst_status mst_get_round_stats(mst_handle h, void *stream, int64_t *live_edges,
                               int64_t *live_vertices, int32_t cap, int32_t *rounds)
{
    if (!h || cap < 0 || !rounds)
        return MST_ERR_INVALID_ARG;
    *rounds = 0;
    if (!h->single.base)
        return MST_OK;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return MST_ERR_CUDA;
    Ctl c;
    if (cudaMemcpy(&c, h->single.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MST_ERR_CUDA;
    int32_t r = (int32_t)c.round;
    *rounds = r;
    for (int32_t i = 0; i <= r && i < cap && i <= kMaxRounds; i++) {
        if (live_edges)
            live_edges[i] = c.stat_m[i];
        if (live_vertices)
            live_vertices[i] = c.stat_n[i];
    }
    return MST_OK;
}

mst_status mst_solve_batched(mst_handle h, mst_weight_type wt, int32_t G, const int64_t *vtx_off,
                             const int64_t *edge_off, int64_t total_n, int64_t total_m,
                             const int32_t *src, const int32_t *dst, const void *w,
                             int32_t *out_edge_ids, int64_t *out_counts, void *stream)
{
    if (!h || (wt != MST_W_U32 && wt != MST_W_F32) || G < 0 || total_n < 0 || total_m < 0)
        return MST_ERR_INVALID_ARG;
    if (G > 0 && (!vtx_off || !edge_off || !out_counts))
        return MST_ERR_INVALID_ARG;
    if (total_m > 0 && (!src || !dst || !w))
        return MST_ERR_INVALID_ARG;
    if (total_n > 0 && !out_edge_ids)
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    h->last = LAST_BATCHED;
    if (G == 0)
        return MST_OK;
    if (h->budget && batched_bytes(G, (uint64_t)total_n, (uint64_t)total_m) + h->single.bytes +
                             aux_bytes(h) > h->budget)
        return MST_ERR_BUDGET;
    cudaError_t e = batched_reserve(h->batched, G, (uint64_t)total_n, (uint64_t)total_m);
    if (e != cudaSuccess) {
        batched_release(h->batched);
        cudaGetLastError();
        return cuda_status(e);
    }
    return cuda_status(batched_launch(h->batched, h->device, (uint32_t)wt, G, vtx_off, edge_off,
                                      (uint64_t)total_n, (uint64_t)total_m, src, dst, w,
                                      out_edge_ids, out_counts, s));
}

mst_status mst_set_batched_schedule(mst_handle h, int schedule, int block_threads)
{
    if (!h || schedule < 0 || schedule > 2)
        return MST_ERR_INVALID_ARG;
    if (block_threads != 0 && block_threads != 128 && block_threads != 256 &&
        block_threads != 512 && block_threads != 1024)
        return MST_ERR_INVALID_ARG;
    h->batched.schedule = schedule;
    h->batched.block_threads = block_threads;
    return MST_OK;
}

mst_status mst_set_single_schedule(mst_handle h, int schedule, int blocks_per_sm,
                                   int block_threads)
{
    if (!h || schedule < 0 || schedule > 4 || blocks_per_sm < 0 || blocks_per_sm > 8 ||
        (block_threads != 0 && block_threads != 256 && block_threads != 512 &&
         block_threads != 768 && block_threads != 1024))
        return MST_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    cudaDeviceSynchronize();
    h->single.schedule = schedule;
    const int bps = blocks_per_sm > 0 ? blocks_per_sm : h->single.fused_blocks_per_sm;
    const int ft = block_threads > 0 ? block_threads : h->single.fused_threads;
    if (bps != h->single.fused_blocks_per_sm || ft != h->single.fused_threads) {
        h->single.fused_blocks_per_sm = bps;
        h->single.fused_threads = ft;
        single_release(h->single);  // the grid is fixed at reservation time
        h->last_solve.valid = false;
    }
    return MST_OK;
}

mst_status mst_set_wait_limit(mst_handle h, uint32_t polls)
{
    if (!h)
        return MST_ERR_INVALID_ARG;
    h->single.wait_limit = polls;
    return MST_OK;
}

mst_status mst_autotune_batched(mst_handle h, mst_weight_type wt, int32_t G,
                                const int64_t *vtx_off, const int64_t *edge_off, int64_t total_n,
                                int64_t total_m, const int32_t *src, const int32_t *dst,
                                const void *w, int32_t *out_edge_ids, int64_t *out_counts,
                                const char *cache_path, void *stream)
{
    if (!h || (wt != MST_W_U32 && wt != MST_W_F32) || G < 0 || total_n < 0 || total_m < 0)
        return MST_ERR_INVALID_ARG;
    if (G > 0 && (!vtx_off || !edge_off || !out_counts))
        return MST_ERR_INVALID_ARG;
    if (total_m > 0 && (!src || !dst || !w))
        return MST_ERR_INVALID_ARG;
    if (total_n > 0 && !out_edge_ids)
        return MST_ERR_INVALID_ARG;
    if (G == 0)
        return MST_OK;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return MST_ERR_CUDA;
    if (h->budget && batched_bytes(G, (uint64_t)total_n, (uint64_t)total_m) + h->single.bytes +
                             aux_bytes(h) > h->budget)
        return MST_ERR_BUDGET;
    cudaError_t e = batched_reserve(h->batched, G, (uint64_t)total_n, (uint64_t)total_m);
    if (e != cudaSuccess) {
        batched_release(h->batched);
        cudaGetLastError();
        return cuda_status(e);
    }
    h->last = LAST_BATCHED;
    e = batched_autotune(h->batched, h->device, (uint32_t)wt, G, vtx_off, edge_off,
                         (uint64_t)total_n, (uint64_t)total_m, src, dst, w, out_edge_ids,
                         out_counts, cache_path, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize((cudaStream_t)stream);
    return cuda_status(e);
}

mst_status mst_server_start(mst_handle h, int streams, int max_batch)
{
    if (!h || streams < 1 || streams > 64 || max_batch < 1)
        return MST_ERR_INVALID_ARG;
    return server_start(h, streams, max_batch);
}

mst_status mst_submit(mst_handle h, mst_weight_type wt, int32_t n, int64_t m, const int32_t *src,
                      const int32_t *dst, const void *w, int32_t *out_edge_ids,
                      int64_t *out_count, uint64_t *ticket)
{
    if (!h || !ticket || (wt != MST_W_U32 && wt != MST_W_F32))
        return MST_ERR_INVALID_ARG;
    mst_status st = check_graph_args(n, m, src, dst, w, out_edge_ids, out_count);
    if (st != MST_OK)
        return st;
    Request r{};
    r.wt = (uint32_t)wt;
    r.n = n;
    r.m = m;
    r.src = src;
    r.dst = dst;
    r.w = w;
    r.out = out_edge_ids;
    r.out_count = out_count;
    r.t_submit_us = now_us();
    return server_submit(h, r, ticket);
}

mst_status mst_poll(mst_handle h, uint64_t ticket, int *done, double *latency_us)
{
    if (!h || !done)
        return MST_ERR_INVALID_ARG;
    return server_poll(h, ticket, done, latency_us);
}

mst_status mst_server_drain(mst_handle h)
{
    if (!h)
        return MST_ERR_INVALID_ARG;
    return server_drain(h);
}

mst_status mst_server_stop(mst_handle h)
{
    if (!h)
        return MST_ERR_INVALID_ARG;
    return server_stop(h);
}

}  // extern "C"
