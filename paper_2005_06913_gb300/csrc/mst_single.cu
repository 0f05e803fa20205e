// mst_single.cu — data-parallel Boruvka rounds for one graph (Section 2.1),
// as hand-written sm_103a kernels captured once into a CUDA graph whose round
// loop is a device-controlled conditional WHILE node.
//
// One solve:
//   k_init            comp ids = vertex ids, minimum[] = none, M = empty
//   k_find0           round 0 find-min over the caller's COO arrays
//   round 0 body      k_hook<R0> -> k_compress [-> WHILE k_compress(jump)] -> k_compact<R0>
//   WHILE live > 0    k_hook -> k_compress [-> WHILE jump] -> k_compact
//   k_emit            M as ascending edge ids
//
// Round r works on a contracted graph: components are numbered 0..n_r-1 and
// the live edge list holds only edges between different components, with
// endpoints already renamed to component ids.  Per round:
//   find-min (Section 2.1 steps 15-28): every live edge offers its key to
//     both endpoint components with a 64-bit atomicMin (the key packs the
//     weight above the edge's list position, so ties break by edge id);
//     for round r+1 this runs fused into round r's compaction.
//   hook (steps 30-40): every component c with a minimum edge e to d points
//     at d and marks e as a tree edge, except that of two components that
//     chose the same edge the lower id stays a root.  Under a total order
//     that mutual pair is the only cycle the pointers can form, so they form
//     a forest (the lock/CAS serialisation of Sections 2.2.1-2.2.2 is not
//     needed).  Roots get new dense ids by a prefix sum.
//   compress: each component follows its pointers to its root (path halving,
//     bounded hops per pass, extra passes only if a chain is deep) and takes
//     the root's new id.
//   compact (Section 2.1 "Optimization", covered edges): edges whose two
//     renamed endpoints coincide are dropped; survivors are written, in their
//     old order, to the next list, and offer their keys for round r+1.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mst_internal.h"

namespace mst {

// -------------------------------------------------------------- kernels

__global__ void __launch_bounds__(kThreads)
k_init(Ws ws, const int32_t *src, const int32_t *dst, const void *w, int32_t *out,
       int64_t *out_count, uint32_t n, uint32_t m, uint32_t wt, uint32_t vec_ok,
       uint32_t reset_epoch)
{
    Ctl *c = ws.ctl;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    if (gtid == 0) {
        c->src = src;
        c->dst = dst;
        c->w = w;
        c->out = out;
        c->out_count = out_count;
        c->n = n;
        c->m = m;
        c->wt = wt;
        c->vec_ok = vec_ok;
        c->round = 0;
        c->n_cur = n;
        c->m_cur = m;
        c->n_next = 0;
        c->m_next = 0;
        c->ticket = 0;
        c->done = 0;
        c->deep = 0;
        c->status = 0;
        if (reset_epoch)
            c->epoch = 1;
        for (int r = 0; r <= kMaxRounds; r++) {
            c->stat_m[r] = 0;
            c->stat_n[r] = 0;
        }
        c->stat_m[0] = m;
        c->stat_n[0] = n;
    }
    unsigned long long *m0 = ws.mins[0];
    for (size_t v = gtid; v < n; v += stride)
        m0[v] = kNoEdge;
    const size_t words = ((size_t)m + 31) >> 5;
    for (size_t i = gtid; i < words; i += stride)
        ws.mst_bits[i] = 0u;
}

// Round-0 find-min: every non-loop edge offers (weight, id) to both ends.
__global__ void __launch_bounds__(kThreads) k_find0(Ws ws)
{
    Ctl *c = ws.ctl;
    const uint32_t m = c->m, n = c->n, wt = c->wt, vec = c->vec_ok;
    const int32_t *__restrict__ src = c->src;
    const int32_t *__restrict__ dst = c->dst;
    const uint32_t *__restrict__ w = (const uint32_t *)c->w;
    unsigned long long *mn = ws.mins[0];
    uint32_t *status = &c->status;
    const uint32_t groups = (m + 3u) >> 2;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += gridDim.x * blockDim.x) {
        const uint32_t e0 = g << 2;
        int32_t us[4], vs[4];
        uint32_t wr[4];
        if (vec && e0 + 3 < m) {
            const int4 a = __ldg((const int4 *)(src + e0));
            const int4 b = __ldg((const int4 *)(dst + e0));
            const uint4 x = __ldg((const uint4 *)(w + e0));
            us[0] = a.x; us[1] = a.y; us[2] = a.z; us[3] = a.w;
            vs[0] = b.x; vs[1] = b.y; vs[2] = b.z; vs[3] = b.w;
            wr[0] = x.x; wr[1] = x.y; wr[2] = x.z; wr[3] = x.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const bool in = e0 + j < m;
                us[j] = in ? __ldg(src + e0 + j) : 0;
                vs[j] = in ? __ldg(dst + e0 + j) : 0;
                wr[j] = in ? __ldg(w + e0 + j) : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (e0 + j >= m)
                continue;
            const uint32_t u = (uint32_t)us[j], v = (uint32_t)vs[j];
            if (u >= n || v >= n) {
                atomicOr(status, ST_BAD_VERTEX);
                continue;
            }
            if (u == v)
                continue;
            const unsigned long long key = make_key(weight_bits(wr[j], wt, status), e0 + j);
            atomicMin(&mn[u], key);
            atomicMin(&mn[v], key);
        }
    }
}

// Hook (Section 2.1 steps 30-40) + dense renumbering of the roots.
template <bool R0>
__global__ void __launch_bounds__(kThreads) k_hook(Ws ws)
{
    __shared__ uint32_t s32[33];
    __shared__ uint32_t s_tile, s_excl, s_flag;
    Ctl *c = ws.ctl;
    const uint32_t round = c->round, epoch = c->epoch, n_cur = c->n_cur;
    const unsigned long long *mcur = ((round & 1) ? ws.mins[1] : ws.mins[0]);
    unsigned long long *mnext = ((round & 1) ? ws.mins[0] : ws.mins[1]);
    const uint4 *ecur = ((round & 1) ? ws.E[1] : ws.E[0]);
    const int32_t *src = c->src;
    const int32_t *dst = c->dst;
    int32_t *parent = ws.parent;
    const uint32_t ntiles = (n_cur + kTile - 1) / kTile;
    for (;;) {
        const uint32_t tile = next_tile(&c->ticket, &s_tile);
        if (tile >= ntiles)
            break;
        const uint32_t base = tile * kTile;
        bool root[kItems];
        uint32_t vv[kItems];
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t v = base + j * kThreads + threadIdx.x;
            vv[j] = v;
            root[j] = false;
            if (v < n_cur) {
                const unsigned long long k = mcur[v];
                mnext[v] = kNoEdge;
                if (k == kNoEdge) {
                    root[j] = true;  // no edge leaves this component
                } else {
                    const uint32_t p = (uint32_t)k;
                    uint32_t a, b, id;
                    if (R0) {
                        a = (uint32_t)__ldg(src + p);
                        b = (uint32_t)__ldg(dst + p);
                        id = p;
                    } else {
                        const uint4 r = ecur[p];
                        a = r.x;
                        b = r.y;
                        id = r.w;
                    }
                    const uint32_t d = (a == v) ? b : a;
                    const unsigned long long kd = mcur[d];
                    if ((uint32_t)kd == p && v < d) {
                        root[j] = true;  // mutual choice: the lower id stays root
                    } else {
                        parent[v] = (int32_t)d;
                        atomicOr(&ws.mst_bits[id >> 5], 1u << (id & 31));
                    }
                }
                if (root[j])
                    parent[v] = (int32_t)v;
            }
        }
        uint32_t rank[kItems], total;
        tile_ranks_striped(root, rank, total, s32);
        if (threadIdx.x < 32) {
            const uint32_t ex = lookback_warp(ws.desc, tile, total, epoch, &c->status);
            if (threadIdx.x == 0) {
                s_excl = ex;
                if (tile == ntiles - 1)
                    c->n_next = ex + total;
            }
        }
        __syncthreads();
        const uint32_t ex = s_excl;
#pragma unroll
        for (int j = 0; j < kItems; j++)
            if (root[j])
                ws.nid[vv[j]] = (int32_t)(ex + rank[j]);
    }
    if (last_block_done(&c->done, &s_flag) && threadIdx.x == 0) {
        if (ntiles == 0)
            c->n_next = 0;
        c->epoch = epoch + 1;
        c->ticket = 0;
        c->done = 0;
    }
}

// Follows hook pointers from `start` with path halving, at most kChaseLimit
// steps.  Returns true and the root when it gets there.
__device__ __forceinline__ bool chase(int32_t *parent, uint32_t start, uint32_t &at)
{
    uint32_t x = start;
#pragma unroll 1
    for (int s = 0; s < kChaseLimit; s++) {
        const uint32_t p = (uint32_t)__ldcg(parent + x);
        if (p == x) {
            at = x;
            return true;
        }
        const uint32_t gp = (uint32_t)__ldcg(parent + p);
        if (gp == p) {
            at = p;
            return true;
        }
        __stcg(parent + x, (int32_t)gp);
        x = gp;
    }
    at = x;
    return false;
}

// Label compression: lab[v] = new id of v's root.  With first == 0 it is a
// follow-up pass over the components whose chase did not finish.  The last
// block decides whether another pass runs (conditional node `jump`).
__global__ void __launch_bounds__(kThreads)
k_compress(Ws ws, cudaGraphConditionalHandle jump, uint32_t first, uint32_t graph_mode)
{
    __shared__ uint32_t s_flag;
    Ctl *c = ws.ctl;
    const uint32_t n_cur = c->n_cur;
    int32_t *parent = ws.parent;
    bool unfinished = false;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n_cur;
         v += gridDim.x * blockDim.x) {
        uint32_t start = v;
        if (!first) {
            if (__ldcg(ws.lab + v) != -1)
                continue;
            start = (uint32_t)__ldcg(parent + v);
        }
        uint32_t at;
        if (chase(parent, start, at)) {
            ws.lab[v] = ws.nid[at];
        } else {
            ws.lab[v] = -1;
            __stcg(parent + v, (int32_t)at);
            unfinished = true;
        }
    }
    if (unfinished)
        c->deep = 1u;
    if (last_block_done(&c->done, &s_flag) && threadIdx.x == 0) {
        uint32_t deep = ld_volatile_u32(&c->deep);
        const uint32_t passes = first ? 0u : c->passes + 1u;
        if (deep && passes >= kMaxJumpPasses) {  // cannot happen for a forest: stop, flag
            atomicOr(&c->status, ST_INTERNAL);
            deep = 0;
        }
        c->passes = passes;
        if (graph_mode)
            cudaGraphSetConditional(jump, deep ? 1u : 0u);
        c->deep_seen = deep;
        c->deep = 0;
        c->done = 0;
    }
}

// Compaction of round r fused with find-min of round r+1.
template <bool R0>
__global__ void __launch_bounds__(kThreads)
k_compact(Ws ws, cudaGraphConditionalHandle loop, uint32_t graph_mode)
{
    __shared__ uint4 stage[kTile];
    __shared__ uint32_t s32[33];
    __shared__ uint32_t s_tile, s_excl, s_flag;
    Ctl *c = ws.ctl;
    const uint32_t round = c->round, epoch = c->epoch, m_cur = c->m_cur;
    const uint32_t n_in = c->n, wt = c->wt, vec = c->vec_ok, n_next = c->n_next;
    const uint4 *ecur = ((round & 1) ? ws.E[1] : ws.E[0]);
    uint4 *enext = ((round & 1) ? ws.E[0] : ws.E[1]);
    unsigned long long *mnext = ((round & 1) ? ws.mins[0] : ws.mins[1]);
    const int32_t *__restrict__ lab = ws.lab;
    const int32_t *__restrict__ src = c->src;
    const int32_t *__restrict__ dst = c->dst;
    const uint32_t *__restrict__ w = (const uint32_t *)c->w;
    uint32_t *status = &c->status;
    const uint32_t ntiles = (m_cur + kTile - 1) / kTile;
    for (;;) {
        const uint32_t tile = next_tile(&c->ticket, &s_tile);
        if (tile >= ntiles)
            break;
        const uint32_t base = tile * kTile;
        bool keep[kItems];
        uint4 rec[kItems];
        uint32_t rank[kItems], total;
        if (R0) {
            const uint32_t e0 = base + threadIdx.x * kItems;
            int32_t us[4], vs[4];
            uint32_t wr[4];
            if (vec && e0 + 3 < m_cur) {
                const int4 a = __ldg((const int4 *)(src + e0));
                const int4 b = __ldg((const int4 *)(dst + e0));
                const uint4 x = __ldg((const uint4 *)(w + e0));
                us[0] = a.x; us[1] = a.y; us[2] = a.z; us[3] = a.w;
                vs[0] = b.x; vs[1] = b.y; vs[2] = b.z; vs[3] = b.w;
                wr[0] = x.x; wr[1] = x.y; wr[2] = x.z; wr[3] = x.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const bool in = e0 + j < m_cur;
                    us[j] = in ? __ldg(src + e0 + j) : 0;
                    vs[j] = in ? __ldg(dst + e0 + j) : 0;
                    wr[j] = in ? __ldg(w + e0 + j) : 0u;
                }
            }
#pragma unroll
            for (int j = 0; j < kItems; j++) {
                keep[j] = false;
                const uint32_t u = (uint32_t)us[j], v = (uint32_t)vs[j];
                if (e0 + j < m_cur && u < n_in && v < n_in && u != v) {
                    const uint32_t nu = (uint32_t)lab[u], nv = (uint32_t)lab[v];
                    if (nu >= n_next || nv >= n_next) {
                        atomicOr(status, ST_INTERNAL);  // never for a valid forest
                    } else if (nu != nv) {
                        keep[j] = true;
                        rec[j] = make_uint4(nu, nv, weight_bits(wr[j], wt, status), e0 + j);
                    }
                }
            }
            tile_ranks_blocked(keep, rank, total, s32);
        } else {
#pragma unroll
            for (int j = 0; j < kItems; j++) {
                const uint32_t i = base + j * kThreads + threadIdx.x;
                keep[j] = false;
                if (i < m_cur) {
                    const uint4 r = ecur[i];
                    const uint32_t nu = (uint32_t)lab[r.x], nv = (uint32_t)lab[r.y];
                    if (nu >= n_next || nv >= n_next) {
                        atomicOr(status, ST_INTERNAL);  // never for a valid forest
                    } else if (nu != nv) {
                        keep[j] = true;
                        rec[j] = make_uint4(nu, nv, r.z, r.w);
                    }
                }
            }
            tile_ranks_striped(keep, rank, total, s32);
        }
        if (threadIdx.x < 32) {
            const uint32_t ex = lookback_warp(ws.desc, tile, total, epoch, status);
            if (threadIdx.x == 0) {
                s_excl = ex;
                if (tile == ntiles - 1)
                    c->m_next = ex + total;
            }
        }
#pragma unroll
        for (int j = 0; j < kItems; j++)
            if (keep[j])
                stage[rank[j]] = rec[j];
        __syncthreads();
        const uint32_t ex = s_excl;
        for (uint32_t i = threadIdx.x; i < total; i += kThreads) {
            const uint4 r = stage[i];
            const uint32_t pos = ex + i;
            enext[pos] = r;
            const unsigned long long key = make_key(r.z, pos);
            atomicMin(&mnext[r.x], key);
            atomicMin(&mnext[r.y], key);
        }
    }
    if (last_block_done(&c->done, &s_flag) && threadIdx.x == 0) {
        const uint32_t m_next = ntiles ? ld_volatile_u32(&c->m_next) : 0u;
        const uint32_t n_next = ld_volatile_u32(&c->n_next);
        const uint32_t r1 = round + 1;
        if (r1 <= (uint32_t)kMaxRounds) {
            c->stat_m[r1] = m_next;
            c->stat_n[r1] = n_next;
        }
        c->m_cur = m_next;
        c->n_cur = n_next;
        c->round = r1;
        c->epoch = epoch + 1;
        c->ticket = 0;
        c->done = 0;
        bool more = m_next > 0;
        if (more && r1 >= (uint32_t)kMaxRounds) {
            atomicOr(status, ST_INTERNAL);
            more = false;
        }
        if (graph_mode)
            cudaGraphSetConditional(loop, more ? 1u : 0u);
    }
}

// Emits M as ascending edge ids and checks |M| = n - #components.
__global__ void __launch_bounds__(kThreads) k_emit(Ws ws)
{
    __shared__ uint32_t s32[33];
    __shared__ uint32_t s_tile, s_excl, s_flag;
    Ctl *c = ws.ctl;
    const uint32_t m = c->m, epoch = c->epoch;
    const uint32_t words = (m + 31u) >> 5;
    const uint32_t ntiles = (words + kTile - 1) / kTile;
    int32_t *out = c->out;
    const uint32_t cap = c->n > 0 ? c->n - 1 : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        const uint32_t tile = next_tile(&c->ticket, &s_tile);
        if (tile >= ntiles)
            break;
        const uint32_t base = tile * kTile;
        uint32_t wv[kItems], pre[kItems];
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t i = base + j * kThreads + threadIdx.x;
            wv[j] = i < words ? ws.mst_bits[i] : 0u;
            const uint32_t cnt = __popc(wv[j]);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            pre[j] = incl - cnt;
            if (lane == 31)
                s32[j * kWarps + warp] = incl;
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = s32[lane];
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            s32[lane] = incl - v;
            if (lane == 31)
                s32[32] = incl;
        }
        __syncthreads();
        const uint32_t total = s32[32];
        if (threadIdx.x < 32) {
            const uint32_t ex = lookback_warp(ws.desc, tile, total, epoch, &c->status);
            if (threadIdx.x == 0) {
                s_excl = ex;
                if (tile == ntiles - 1)
                    c->m_next = ex + total;  // reused as the emitted count
            }
        }
        __syncthreads();
        const uint32_t ex = s_excl;
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            uint32_t bits = wv[j];
            uint32_t pos = ex + s32[j * kWarps + warp] + pre[j];
            const uint32_t i = base + j * kThreads + threadIdx.x;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                if (pos < cap)
                    out[pos] = (int32_t)(i * 32u + (uint32_t)b);
                else
                    atomicOr(&c->status, ST_INTERNAL);  // more tree edges than n-1
                pos++;
            }
        }
    }
    if (last_block_done(&c->done, &s_flag) && threadIdx.x == 0) {
        const uint32_t emitted = ntiles ? ld_volatile_u32(&c->m_next) : 0u;
        *c->out_count = (int64_t)emitted;
        const uint32_t comps = ld_volatile_u32(&c->n_cur);
        if (emitted + comps != c->n)
            atomicOr(&c->status, ST_INTERNAL);
        if (comps > 1)
            atomicOr(&c->status, ST_DISCONNECTED);
        c->m_next = 0;
        c->epoch = epoch + 1;
        c->ticket = 0;
        c->done = 0;
    }
}

// ------------------------------------------------------------------ host

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static uint32_t desc_capacity(uint32_t n_cap, uint32_t m_cap)
{
    const uint32_t words = (m_cap + 31) / 32;
    uint32_t t = (m_cap + kTile - 1) / kTile;
    t = t > (n_cap + kTile - 1) / kTile ? t : (n_cap + kTile - 1) / kTile;
    t = t > (words + kTile - 1) / kTile ? t : (words + kTile - 1) / kTile;
    return t + 1;
}

size_t single_bytes(uint32_t n_cap, uint32_t m_cap)
{
    size_t b = align_up(sizeof(Ctl));
    b += 2 * align_up((size_t)m_cap * sizeof(uint4));
    b += 2 * align_up((size_t)n_cap * 8);
    b += 3 * align_up((size_t)n_cap * 4);
    b += align_up((((size_t)m_cap + 31) / 32) * 4);
    b += align_up((size_t)desc_capacity(n_cap, m_cap) * 8);
    return b;
}

void single_release(Single &s)
{
    if (s.exec)
        cudaGraphExecDestroy(s.exec);
    if (s.graph)
        cudaGraphDestroy(s.graph);
    if (s.base)
        cudaFree(s.base);
    s = Single();
}

#define MST_TRY(x)                     \
    do {                               \
        cudaError_t e_ = (x);          \
        if (e_ != cudaSuccess)         \
            return e_;                 \
    } while (0)

static cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep,
                              size_t ndep, void *func, int grid, void **args)
{
    cudaKernelNodeParams p = {};
    p.func = func;
    p.gridDim = dim3((unsigned)grid);
    p.blockDim = dim3(kThreads);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    p.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, dep, ndep, &p);
}

static cudaError_t add_while(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep,
                             size_t ndep, cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    MST_TRY(cudaGraphAddNode(node, g, dep, nullptr, ndep, &p));
    *body = p.conditional.phGraph_out[0];
    return cudaSuccess;
}

// Appends hook -> compress -> WHILE(jump) -> compact to `g` after `dep`.
static cudaError_t add_round(cudaGraph_t g, cudaGraphNode_t dep, bool r0, Single &s,
                             cudaGraphConditionalHandle loop, cudaGraphNode_t *last)
{
    cudaGraphConditionalHandle jump;
    MST_TRY(cudaGraphConditionalHandleCreate(&jump, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t hook, comp, wj, cpt, jn;
    const cudaGraphNode_t *d0 = dep ? &dep : nullptr;
    size_t n0 = dep ? 1 : 0;
    void *ha[] = {&s.ws};
    MST_TRY(add_kernel(&hook, g, d0, n0, r0 ? (void *)k_hook<true> : (void *)k_hook<false>,
                       s.grid_tiles, ha));
    uint32_t one = 1, zero = 0;
    void *ca[] = {&s.ws, &jump, &one, &one};
    MST_TRY(add_kernel(&comp, g, &hook, 1, (void *)k_compress, s.grid_stream, ca));
    cudaGraph_t body;
    MST_TRY(add_while(&wj, g, &comp, 1, jump, &body));
    void *ja[] = {&s.ws, &jump, &zero, &one};
    MST_TRY(add_kernel(&jn, body, nullptr, 0, (void *)k_compress, s.grid_stream, ja));
    void *pa[] = {&s.ws, &loop, &one};
    MST_TRY(add_kernel(&cpt, g, &wj, 1, r0 ? (void *)k_compact<true> : (void *)k_compact<false>,
                       s.grid_tiles, pa));
    *last = cpt;
    return cudaSuccess;
}

static cudaError_t build_graph(Single &s)
{
    cudaGraph_t g;
    MST_TRY(cudaGraphCreate(&g, 0));
    s.graph = g;
    cudaGraphConditionalHandle loop;
    MST_TRY(cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t find0, r0last, wl, emit, blast;
    void *fa[] = {&s.ws};
    MST_TRY(add_kernel(&find0, g, nullptr, 0, (void *)k_find0, s.grid_stream, fa));
    MST_TRY(add_round(g, find0, true, s, loop, &r0last));
    cudaGraph_t body;
    MST_TRY(add_while(&wl, g, &r0last, 1, loop, &body));
    MST_TRY(add_round(body, nullptr, false, s, loop, &blast));
    void *ea[] = {&s.ws};
    MST_TRY(add_kernel(&emit, g, &wl, 1, (void *)k_emit, s.grid_tiles, ea));
    MST_TRY(cudaGraphInstantiate(&s.exec, g, 0));
    return cudaSuccess;
}

static int occupancy(const void *func, size_t smem)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, func, kThreads, smem) != cudaSuccess ||
        blocks < 1)
        blocks = 1;
    return blocks;
}

cudaError_t single_reserve(Single &s, int device, uint32_t n, uint32_t m)
{
    if (s.base && n <= s.ws.n_cap && m <= s.ws.m_cap)
        return cudaSuccess;
    uint32_t n_cap = n > s.ws.n_cap ? n : s.ws.n_cap;
    uint32_t m_cap = m > s.ws.m_cap ? m : s.ws.m_cap;
    n_cap = n_cap < 1024 ? 1024 : n_cap;
    m_cap = m_cap < 1024 ? 1024 : m_cap;
    single_release(s);
    const size_t bytes = single_bytes(n_cap, m_cap);
    void *base = nullptr;
    MST_TRY(cudaMalloc(&base, bytes));
    s.base = base;
    s.bytes = bytes;
    char *p = (char *)base;
    auto take = [&](size_t sz) {
        char *q = p;
        p += align_up(sz);
        return (void *)q;
    };
    s.ws.ctl = (Ctl *)take(sizeof(Ctl));
    s.ws.E[0] = (uint4 *)take((size_t)m_cap * sizeof(uint4));
    s.ws.E[1] = (uint4 *)take((size_t)m_cap * sizeof(uint4));
    s.ws.mins[0] = (unsigned long long *)take((size_t)n_cap * 8);
    s.ws.mins[1] = (unsigned long long *)take((size_t)n_cap * 8);
    s.ws.parent = (int32_t *)take((size_t)n_cap * 4);
    s.ws.nid = (int32_t *)take((size_t)n_cap * 4);
    s.ws.lab = (int32_t *)take((size_t)n_cap * 4);
    s.ws.mst_bits = (uint32_t *)take((((size_t)m_cap + 31) / 32) * 4);
    s.ws.desc_cap = desc_capacity(n_cap, m_cap);
    s.ws.desc = (unsigned long long *)take((size_t)s.ws.desc_cap * 8);
    s.ws.n_cap = n_cap;
    s.ws.m_cap = m_cap;
    MST_TRY(cudaMemset(s.ws.ctl, 0, sizeof(Ctl)));
    MST_TRY(cudaMemset(s.ws.desc, 0, (size_t)s.ws.desc_cap * 8));
    int sms = 0;
    MST_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    int occ_t = occupancy((const void *)k_compact<false>, 0);
    int occ_h = occupancy((const void *)k_hook<false>, 0);
    int occ = occ_t < occ_h ? occ_t : occ_h;
    occ = occ > 4 ? 4 : occ;
    s.grid_tiles = sms * occ;
    s.grid_stream = sms * 4;
    s.solves = 0;
    return build_graph(s);
}

cudaError_t single_launch(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                          uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n, uint32_t m,
                          cudaStream_t stream)
{
    uint32_t reset = 0;
    if (++s.solves >= (1u << 22)) {  // keep the 31-bit descriptor epoch from wrapping
        MST_TRY(cudaMemsetAsync(s.ws.desc, 0, (size_t)s.ws.desc_cap * 8, stream));
        s.solves = 1;
        reset = 1;
    }
    const uint32_t vec = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)w) & 15u) == 0 ? 1u : 0u;
    k_init<<<s.grid_stream, kThreads, 0, stream>>>(s.ws, src, dst, w, out, out_count, n, m, wt,
                                                   vec, reset);
    MST_TRY(cudaGetLastError());
    return cudaGraphLaunch(s.exec, stream);
}

// ------------------------------------------------------- per-kernel timing

// Replays a solve launching every kernel on its own between two CUDA events
// (the captured graph's conditional nodes are replaced by host decisions
// read from the control block after each kernel).  Bytes follow the DRAM
// model: edge lists and per-vertex arrays, not L2-resident gathers/atomics.
cudaError_t single_profile(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                           uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n, uint32_t m,
                           cudaStream_t stream, std::vector<KernelProfile> &prof)
{
    prof.clear();
    cudaEvent_t e0, e1;
    MST_TRY(cudaEventCreate(&e0));
    MST_TRY(cudaEventCreate(&e1));
    cudaError_t err = cudaSuccess;
    auto rec = [&](const char *name, double bytes, auto launch) {
        if (err != cudaSuccess)
            return;
        err = cudaEventRecord(e0, stream);
        if (err == cudaSuccess)
            launch();
        if (err == cudaSuccess)
            err = cudaGetLastError();
        if (err == cudaSuccess)
            err = cudaEventRecord(e1, stream);
        if (err == cudaSuccess)
            err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess)
            err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess)
            return;
        for (auto &k : prof)
            if (k.name == name) {
                k.launches++;
                k.ms += ms;
                k.bytes += bytes;
                return;
            }
        prof.push_back(KernelProfile{name, 1, (double)ms, bytes});
    };
    Ctl c;
    auto read_ctl = [&]() {
        if (err == cudaSuccess)
            err = cudaMemcpy(&c, s.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    };
    const uint32_t vec = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)w) & 15u) == 0 ? 1u : 0u;
    cudaGraphConditionalHandle none = 0;
    uint32_t zero = 0, one = 1;
    (void)zero;
    (void)one;
    const int gt = s.grid_tiles, gs = s.grid_stream;
    const double words = ((double)m + 31) / 32;
    rec("k_init", 8.0 * n + 4 * words, [&] {
        k_init<<<gs, kThreads, 0, stream>>>(s.ws, src, dst, w, out, out_count, n, m, wt, vec, 0);
    });
    rec("k_find0", 12.0 * m, [&] { k_find0<<<gs, kThreads, 0, stream>>>(s.ws); });
    read_ctl();
    for (int r = 0; err == cudaSuccess; r++) {
        const double nr = c.n_cur, mr = c.m_cur;
        if (r > 0 && c.m_cur == 0)
            break;
        // hook: read mins, reset next mins, write parent; new ids of roots
        rec(r == 0 ? "k_hook<R0>" : "k_hook<R>", 20.0 * nr, [&] {
            if (r == 0)
                k_hook<true><<<gt, kThreads, 0, stream>>>(s.ws);
            else
                k_hook<false><<<gt, kThreads, 0, stream>>>(s.ws);
        });
        read_ctl();
        const double nn = c.n_next;
        rec("k_compress", 8.0 * nr + 4.0 * nn, [&] {
            k_compress<<<gs, kThreads, 0, stream>>>(s.ws, none, 1u, 0u);
        });
        read_ctl();
        while (err == cudaSuccess && c.deep_seen) {
            rec("k_compress(jump)", 8.0 * nr, [&] {
                k_compress<<<gs, kThreads, 0, stream>>>(s.ws, none, 0u, 0u);
            });
            read_ctl();
        }
        const double in_bytes = r == 0 ? 12.0 * mr : 16.0 * mr;
        rec(r == 0 ? "k_compact<R0>" : "k_compact<R>", 0.0, [&] {
            if (r == 0)
                k_compact<true><<<gt, kThreads, 0, stream>>>(s.ws, none, 0u);
            else
                k_compact<false><<<gt, kThreads, 0, stream>>>(s.ws, none, 0u);
        });
        read_ctl();
        for (auto &k : prof)  // bytes need m_{r+1}, known only now
            if (k.name == (r == 0 ? "k_compact<R0>" : "k_compact<R>"))
                k.bytes += in_bytes + 16.0 * c.m_cur;
        if (c.m_cur == 0 || c.round >= (uint32_t)kMaxRounds)
            break;
    }
    rec("k_emit", 4 * words + 4.0 * (n > 0 ? n - 1 : 0),
        [&] { k_emit<<<gt, kThreads, 0, stream>>>(s.ws); });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

}  // namespace mst
