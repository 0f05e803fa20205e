// mst_single.cu — data-parallel Boruvka rounds for one graph (Section 2.1)
// as hand-written sm_103a kernels.
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
//     bounded hops per pass, more passes only while some chain is deep) and
//     takes the root's new id.
//   compact (Section 2.1 "Optimization", covered edges): edges whose two
//     renamed endpoints coincide are dropped; survivors are written, in their
//     old order, to the next list, and offer their keys for round r+1.
// The rounds stop when no live edge is left; the tree edges are then emitted
// in ascending id order.
//
// Two schedules run the same tile bodies:
//   fused  (default) one cooperative persistent launch, k_solve, walks every
//          phase of every round; phases are separated by a two-level grid
//          barrier instead of kernel boundaries.
//   graph  one kernel per phase, captured once into a CUDA graph whose round
//          loop and pointer-jump loop are device-controlled conditional WHILE
//          nodes (k_init, k_find0, k_hook, k_compress, k_compact, k_emit).
//          The same kernels, launched one by one between CUDA events, give
//          the per-phase timing of mst_profile_last_solve.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mst_internal.h"

namespace mst {

constexpr int kEmitWords = 128;  // bit words per emit tile: <= 4096 ids, fits the stage

struct TileSmem {
    uint4 stage[kTile];  // survivors of a compaction tile / ids of an emit tile
    uint32_t s32[33];
    uint32_t s_tile, s_excl, s_flag;
};

// ------------------------------------------------------------ tile bodies

__device__ __forceinline__ void init_range(const Ws &ws, uint32_t n, uint32_t m, size_t gtid,
                                           size_t stride)
{
    unsigned long long *m0 = ws.mins[0];
    for (size_t v = gtid; v < n; v += stride)
        m0[v] = kNoEdge;
    const size_t words = ((size_t)m + 31) >> 5;
    for (size_t i = gtid; i < words; i += stride)
        ws.mst_bits[i] = 0u;
}

__device__ __forceinline__ void load4_soa(const int32_t *__restrict__ src,
                                          const int32_t *__restrict__ dst,
                                          const uint32_t *__restrict__ w, uint32_t e0, uint32_t m,
                                          uint32_t vec, int32_t (&us)[4], int32_t (&vs)[4],
                                          uint32_t (&wr)[4])
{
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
}

// Round-0 find-min over edge groups [g0, groups) step gstep (4 edges each).
__device__ __forceinline__ void find0_range(const Ws &ws, const int32_t *src, const int32_t *dst,
                                            const uint32_t *w, uint32_t n, uint32_t m, uint32_t wt,
                                            uint32_t vec, uint32_t *status, size_t g0,
                                            size_t gstep)
{
    unsigned long long *mn = ws.mins[0];
    const size_t groups = ((size_t)m + 3) >> 2;
    for (size_t g = g0; g < groups; g += gstep) {
        const uint32_t e0 = (uint32_t)(g << 2);
        int32_t us[4], vs[4];
        uint32_t wr[4];
        load4_soa(src, dst, w, e0, m, vec, us, vs, wr);
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

// Hook one tile of components (Section 2.1 steps 30-40) and give the tile's
// roots dense new ids.  The block owning the last tile stores n_next.
template <bool R0>
__device__ __forceinline__ void hook_tile(const Ws &ws, Ctl *c, uint32_t tile, uint32_t ntiles,
                                          uint32_t round, uint32_t epoch, uint32_t n_cur,
                                          const int32_t *src, const int32_t *dst, TileSmem &sm)
{
    const unsigned long long *mcur = (round & 1) ? ws.mins[1] : ws.mins[0];
    unsigned long long *mnext = (round & 1) ? ws.mins[0] : ws.mins[1];
    const uint4 *ecur = (round & 1) ? ws.E[1] : ws.E[0];
    int32_t *parent = ws.parent;
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
    tile_ranks_striped(root, rank, total, sm.s32);
    if (threadIdx.x < 32) {
        const uint32_t ex = lookback_warp(ws.desc, tile, total, epoch, &c->status);
        if (threadIdx.x == 0) {
            sm.s_excl = ex;
            if (tile == ntiles - 1)
                c->n_next = ex + total;
        }
    }
    __syncthreads();
    const uint32_t ex = sm.s_excl;
#pragma unroll
    for (int j = 0; j < kItems; j++)
        if (root[j])
            ws.nid[vv[j]] = (int32_t)(ex + rank[j]);
    __syncthreads();  // s32/s_excl free for the next tile
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

// lab[v] = new id of v's root, for v in [v0, n_cur) step vstep.  A follow-up
// pass (first == false) only revisits components whose chase did not end.
// Returns true if some chase in this thread did not end.
__device__ __forceinline__ bool compress_range(const Ws &ws, uint32_t n_cur, bool first,
                                               size_t v0, size_t vstep)
{
    int32_t *parent = ws.parent;
    bool unfinished = false;
    for (size_t vi = v0; vi < n_cur; vi += vstep) {
        const uint32_t v = (uint32_t)vi;
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
    return unfinished;
}

// Compaction of one tile of round r's live edges fused with find-min of
// round r+1.  The block owning the last tile stores m_next.
template <bool R0>
__device__ __forceinline__ void compact_tile(const Ws &ws, Ctl *c, uint32_t tile, uint32_t ntiles,
                                             uint32_t round, uint32_t epoch, uint32_t m_cur,
                                             uint32_t n_next, uint32_t n_in, uint32_t wt,
                                             uint32_t vec, const int32_t *src, const int32_t *dst,
                                             const uint32_t *w, TileSmem &sm)
{
    const uint4 *ecur = (round & 1) ? ws.E[1] : ws.E[0];
    uint4 *enext = (round & 1) ? ws.E[0] : ws.E[1];
    unsigned long long *mnext = (round & 1) ? ws.mins[0] : ws.mins[1];
    const int32_t *__restrict__ lab = ws.lab;
    uint32_t *status = &c->status;
    const uint32_t base = tile * kTile;
    bool keep[kItems];
    uint4 rec[kItems];
    uint32_t rank[kItems], total;
    if (R0) {
        const uint32_t e0 = base + threadIdx.x * kItems;
        int32_t us[4], vs[4];
        uint32_t wr[4];
        load4_soa(src, dst, w, e0, m_cur, vec, us, vs, wr);
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            keep[j] = false;
            rec[j] = make_uint4(0, 0, 0, 0);
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
        tile_ranks_blocked(keep, rank, total, sm.s32);
    } else {
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const uint32_t i = base + j * kThreads + threadIdx.x;
            keep[j] = false;
            rec[j] = make_uint4(0, 0, 0, 0);
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
        tile_ranks_striped(keep, rank, total, sm.s32);
    }
    if (threadIdx.x < 32) {
        const uint32_t ex = lookback_warp(ws.desc, tile, total, epoch, status);
        if (threadIdx.x == 0) {
            sm.s_excl = ex;
            if (tile == ntiles - 1)
                c->m_next = ex + total;
        }
    }
#pragma unroll
    for (int j = 0; j < kItems; j++)
        if (keep[j])
            sm.stage[rank[j]] = rec[j];
    __syncthreads();
    const uint32_t ex = sm.s_excl;
    for (uint32_t i = threadIdx.x; i < total; i += kThreads) {
        const uint4 r = sm.stage[i];
        const uint32_t pos = ex + i;
        enext[pos] = r;
        const unsigned long long key = make_key(r.z, pos);
        atomicMin(&mnext[r.x], key);
        atomicMin(&mnext[r.y], key);
    }
    __syncthreads();  // stage/s32 free for the next tile
}

// Emits the tree edges of one tile of kEmitWords bit words, ascending: ids
// are staged in shared memory, then written out contiguously.  The block
// owning the last tile stores the total in c->emitted (not in m_next, which
// slower blocks of the fused kernel may still be about to read).
__device__ __forceinline__ void emit_tile(const Ws &ws, Ctl *c, uint32_t tile, uint32_t ntiles,
                                          uint32_t epoch, uint32_t words, uint32_t cap,
                                          int32_t *out, TileSmem &sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t i = tile * kEmitWords + threadIdx.x;
    const uint32_t wv = (threadIdx.x < kEmitWords && i < words) ? ws.mst_bits[i] : 0u;
    const uint32_t cnt = __popc(wv);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        sm.s32[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < kWarps ? sm.s32[lane] : 0u;
        uint32_t inc2 = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc2, o);
            if (lane >= o)
                inc2 += y;
        }
        if (lane < kWarps)
            sm.s32[lane] = inc2 - v;
        if (lane == 31)
            sm.s32[32] = inc2;
    }
    __syncthreads();
    const uint32_t total = sm.s32[32];
    uint32_t pos = sm.s32[warp] + incl - cnt;
    if (threadIdx.x < 32) {
        const uint32_t ex = lookback_warp(ws.desc, tile, total, epoch, &c->status);
        if (threadIdx.x == 0) {
            sm.s_excl = ex;
            if (tile == ntiles - 1)
                c->emitted = ex + total;
        }
    }
    uint32_t *ids = (uint32_t *)sm.stage;
    uint32_t bits = wv;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        ids[pos++] = i * 32u + (uint32_t)b;
    }
    __syncthreads();
    const uint32_t ex = sm.s_excl;
    for (uint32_t k = threadIdx.x; k < total; k += kThreads) {
        if (ex + k < cap)
            out[ex + k] = (int32_t)ids[k];
        else
            atomicOr(&c->status, ST_INTERNAL);  // more tree edges than n-1
    }
    __syncthreads();
}

// Final checks of a solve: |M| = n - #components, disconnected flag.
__device__ __forceinline__ void finish(Ctl *c, int64_t *out_count, uint32_t emitted,
                                       uint32_t n, uint32_t comps)
{
    *out_count = (int64_t)emitted;
    if (emitted + comps != n)
        atomicOr(&c->status, ST_INTERNAL);
    if (comps > 1)
        atomicOr(&c->status, ST_DISCONNECTED);
}

// ----------------------------------------------------- grid-wide barrier

// Two-level barrier for a co-resident (cooperative) grid: blocks arrive in
// groups of 16 on separate counters; the last of each group arrives at the
// top counter; the last group flips the generation word.  Waits are bounded:
// on expiry ST_TIMEOUT is set and later barriers no longer wait.
constexpr uint32_t kBarTop = 0, kBarGen = 32, kBarGroups = 64;
constexpr uint32_t kBarSpinLimit = 1u << 21;

__device__ __forceinline__ void grid_sync(uint32_t *bar, uint32_t &gen, uint32_t *status)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t g = gen;
        const uint32_t nb = gridDim.x;
        const uint32_t grp = blockIdx.x >> 4;
        const uint32_t ngrp = (nb + 15) >> 4;
        const uint32_t gsize = min(16u, nb - (grp << 4));
        uint32_t *gc = bar + kBarGroups + 32 * grp;
        __threadfence();
        if (atomicAdd(gc, 1u) == gsize - 1) {
            atomicExch(gc, 0u);
            __threadfence();
            if (atomicAdd(bar + kBarTop, 1u) == ngrp - 1) {
                atomicExch(bar + kBarTop, 0u);
                __threadfence();
                atomicExch(bar + kBarGen, g + 1);
            }
        }
        uint32_t spins = 0;
        while (ld_volatile_u32(bar + kBarGen) == g) {
            if (ld_volatile_u32(status) & ST_TIMEOUT)
                break;
            if (++spins > kBarSpinLimit) {
                atomicOr(status, ST_TIMEOUT);
                printf("mst: grid barrier gave up: block %u of %u, generation %u, top %u, "
                       "group %u count %u\n", blockIdx.x, nb, g, ld_volatile_u32(bar + kBarTop),
                       grp, ld_volatile_u32(gc));
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    gen++;
}

size_t bar_words(int max_blocks) { return kBarGroups + 32 * (size_t)((max_blocks + 15) / 16); }

// ------------------------------------------------- fused persistent kernel

// The whole solve in one cooperative launch.  Tiles are assigned statically
// (tile t to block t mod grid, in increasing order), so every look-back wait
// is on a tile whose block is resident and makes progress.
__global__ void __launch_bounds__(kThreads)
k_solve(Ws ws, const int32_t *src, const int32_t *dst, const uint32_t *w, int32_t *out,
        int64_t *out_count, uint32_t n, uint32_t m, uint32_t wt, uint32_t vec)
{
    __shared__ TileSmem sm;
    Ctl *c = ws.ctl;
    uint32_t *status = &c->status;
    const uint32_t nb = gridDim.x, bid = blockIdx.x;
    const size_t gtid = (size_t)bid * kThreads + threadIdx.x, gstride = (size_t)nb * kThreads;
    uint32_t gen = ld_volatile_u32(ws.bar + kBarGen);
    uint32_t ep = c->epoch;
    init_range(ws, n, m, gtid, gstride);
    if (gtid == 0) {
        c->n = n;
        c->m = m;
        c->flag3[0] = c->flag3[1] = c->flag3[2] = 0;
        for (int r = 0; r <= kMaxRounds; r++) {
            c->stat_m[r] = 0;
            c->stat_n[r] = 0;
        }
        c->stat_m[0] = m;
        c->stat_n[0] = n;
    }
    grid_sync(ws.bar, gen, status);
    find0_range(ws, src, dst, w, n, m, wt, vec, status, gtid, gstride);
    grid_sync(ws.bar, gen, status);
    uint32_t n_cur = n, m_cur = m, r = 0;
    for (;; r++) {
        // hook + new ids of the roots
        const uint32_t nth = (n_cur + kTile - 1) / kTile;
        if (bid == 0 && threadIdx.x == 0)
            c->flag3[0] = 0;
        for (uint32_t t = bid; t < nth; t += nb) {
            if (r == 0)
                hook_tile<true>(ws, c, t, nth, r, ep, n_cur, src, dst, sm);
            else
                hook_tile<false>(ws, c, t, nth, r, ep, n_cur, src, dst, sm);
        }
        ep++;
        grid_sync(ws.bar, gen, status);
        const uint32_t n_next = nth ? ld_volatile_u32(&c->n_next) : 0u;
        // compress, with extra pointer-jumping passes while chains are deep
        for (uint32_t pass = 0;; pass++) {
            if (bid == 0 && threadIdx.x == 0)
                c->flag3[(pass + 1) % 3] = 0;
            const bool unf = compress_range(ws, n_cur, pass == 0, gtid, gstride);
            if (__syncthreads_or(unf ? 1 : 0) && threadIdx.x == 0)
                c->flag3[pass % 3] = 1u;
            grid_sync(ws.bar, gen, status);
            if (!ld_volatile_u32(&c->flag3[pass % 3]))
                break;
            if (pass + 1 >= kMaxJumpPasses) {
                if (gtid == 0)
                    atomicOr(status, ST_INTERNAL);
                break;
            }
        }
        // compact (+ find-min of the next round)
        const uint32_t ntc = (m_cur + kTile - 1) / kTile;
        for (uint32_t t = bid; t < ntc; t += nb) {
            if (r == 0)
                compact_tile<true>(ws, c, t, ntc, r, ep, m_cur, n_next, n, wt, vec, src, dst, w, sm);
            else
                compact_tile<false>(ws, c, t, ntc, r, ep, m_cur, n_next, n, wt, vec, src, dst, w,
                                    sm);
        }
        ep++;
        grid_sync(ws.bar, gen, status);
        const uint32_t m_next = ntc ? ld_volatile_u32(&c->m_next) : 0u;
        if (gtid == 0 && r + 1 <= (uint32_t)kMaxRounds) {
            c->stat_m[r + 1] = m_next;
            c->stat_n[r + 1] = n_next;
        }
        n_cur = n_next;
        m_cur = m_next;
        if (m_cur == 0)
            break;
        if (r + 1 >= (uint32_t)kMaxRounds || (ld_volatile_u32(status) & ST_TIMEOUT)) {
            if (gtid == 0)
                atomicOr(status, ST_INTERNAL);
            break;
        }
    }
    // emit
    const uint32_t words = (m + 31u) >> 5;
    const uint32_t nte = (words + kEmitWords - 1) / kEmitWords;
    const uint32_t cap = n > 0 ? n - 1 : 0;
    for (uint32_t t = bid; t < nte; t += nb)
        emit_tile(ws, c, t, nte, ep, words, cap, out, sm);
    ep++;
    grid_sync(ws.bar, gen, status);
    if (gtid == 0) {
        finish(c, out_count, nte ? ld_volatile_u32(&c->emitted) : 0u, n, n_cur);
        c->round = r + 1;
        c->n_cur = n_cur;
        c->m_cur = 0;
        c->epoch = ep;
    }
}

// ------------------------------------------------ kernels of the graph path

__global__ void __launch_bounds__(kThreads)
k_init(Ws ws, const int32_t *src, const int32_t *dst, const void *w, int32_t *out,
       int64_t *out_count, uint32_t n, uint32_t m, uint32_t wt, uint32_t vec_ok)
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
        for (int r = 0; r <= kMaxRounds; r++) {
            c->stat_m[r] = 0;
            c->stat_n[r] = 0;
        }
        c->stat_m[0] = m;
        c->stat_n[0] = n;
    }
    init_range(ws, n, m, gtid, stride);
}

__global__ void __launch_bounds__(kThreads) k_find0(Ws ws)
{
    Ctl *c = ws.ctl;
    find0_range(ws, c->src, c->dst, (const uint32_t *)c->w, c->n, c->m, c->wt, c->vec_ok,
                &c->status, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                (size_t)gridDim.x * blockDim.x);
}

template <bool R0>
__global__ void __launch_bounds__(kThreads) k_hook(Ws ws)
{
    __shared__ TileSmem sm;
    Ctl *c = ws.ctl;
    const uint32_t round = c->round, epoch = c->epoch, n_cur = c->n_cur;
    const uint32_t ntiles = (n_cur + kTile - 1) / kTile;
    for (;;) {
        const uint32_t tile = next_tile(&c->ticket, &sm.s_tile);
        if (tile >= ntiles)
            break;
        hook_tile<R0>(ws, c, tile, ntiles, round, epoch, n_cur, c->src, c->dst, sm);
    }
    if (last_block_done(&c->done, &sm.s_flag) && threadIdx.x == 0) {
        if (ntiles == 0)
            c->n_next = 0;
        c->epoch = epoch + 1;
        c->ticket = 0;
        c->done = 0;
    }
}

// One compress pass (first != 0) or a follow-up pass; the last block
// decides whether another pass runs (conditional node `jump`).
__global__ void __launch_bounds__(kThreads)
k_compress(Ws ws, cudaGraphConditionalHandle jump, uint32_t first, uint32_t graph_mode)
{
    __shared__ uint32_t s_flag;
    Ctl *c = ws.ctl;
    const bool unfinished =
        compress_range(ws, c->n_cur, first != 0, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                       (size_t)gridDim.x * blockDim.x);
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

template <bool R0>
__global__ void __launch_bounds__(kThreads)
k_compact(Ws ws, cudaGraphConditionalHandle loop, uint32_t graph_mode)
{
    __shared__ TileSmem sm;
    Ctl *c = ws.ctl;
    const uint32_t round = c->round, epoch = c->epoch, m_cur = c->m_cur, n_next = c->n_next;
    const uint32_t ntiles = (m_cur + kTile - 1) / kTile;
    for (;;) {
        const uint32_t tile = next_tile(&c->ticket, &sm.s_tile);
        if (tile >= ntiles)
            break;
        compact_tile<R0>(ws, c, tile, ntiles, round, epoch, m_cur, n_next, c->n, c->wt, c->vec_ok,
                         c->src, c->dst, (const uint32_t *)c->w, sm);
    }
    if (last_block_done(&c->done, &sm.s_flag) && threadIdx.x == 0) {
        const uint32_t m_next = ntiles ? ld_volatile_u32(&c->m_next) : 0u;
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
            atomicOr(&c->status, ST_INTERNAL);
            more = false;
        }
        if (graph_mode)
            cudaGraphSetConditional(loop, more ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(kThreads) k_emit(Ws ws)
{
    __shared__ TileSmem sm;
    Ctl *c = ws.ctl;
    const uint32_t m = c->m, epoch = c->epoch;
    const uint32_t words = (m + 31u) >> 5;
    const uint32_t ntiles = (words + kEmitWords - 1) / kEmitWords;
    const uint32_t cap = c->n > 0 ? c->n - 1 : 0;
    for (;;) {
        const uint32_t tile = next_tile(&c->ticket, &sm.s_tile);
        if (tile >= ntiles)
            break;
        emit_tile(ws, c, tile, ntiles, epoch, words, cap, c->out, sm);
    }
    if (last_block_done(&c->done, &sm.s_flag) && threadIdx.x == 0) {
        finish(c, c->out_count, ntiles ? ld_volatile_u32(&c->emitted) : 0u, c->n,
               ld_volatile_u32(&c->n_cur));
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
    t = t > (words + kEmitWords - 1) / kEmitWords ? t : (words + kEmitWords - 1) / kEmitWords;
    return t + 1;
}

static const int kMaxGridBlocks = 152 * 8 * 2;  // bound for the barrier counters

size_t single_bytes(uint32_t n_cap, uint32_t m_cap)
{
    size_t b = align_up(sizeof(Ctl));
    b += align_up(bar_words(kMaxGridBlocks) * 4);
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
    const int schedule = s.schedule, bps = s.fused_blocks_per_sm;
    s = Single();
    s.schedule = schedule;
    s.fused_blocks_per_sm = bps;
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
    s.ws.bar = (uint32_t *)take(bar_words(kMaxGridBlocks) * 4);
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
    MST_TRY(cudaMemset(s.ws.bar, 0, bar_words(kMaxGridBlocks) * 4));
    MST_TRY(cudaMemset(s.ws.desc, 0, (size_t)s.ws.desc_cap * 8));
    int sms = 0;
    MST_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    int occ_t = occupancy((const void *)k_compact<false>, 0);
    int occ_h = occupancy((const void *)k_hook<false>, 0);
    int occ = occ_t < occ_h ? occ_t : occ_h;
    occ = occ > 4 ? 4 : occ;
    s.grid_tiles = sms * occ;
    s.grid_stream = sms * 4;
    int occ_f = occupancy((const void *)k_solve, 0);
    occ_f = occ_f > s.fused_blocks_per_sm ? s.fused_blocks_per_sm : occ_f;
    s.grid_fused = sms * occ_f;
    if (s.grid_fused > kMaxGridBlocks)
        s.grid_fused = kMaxGridBlocks;
    s.solves = 0;
    return build_graph(s);
}

// Host part of a solve shared by both schedules: keeps the descriptor
// epoch from wrapping, and clears the status word, the round statistics
// and the grid-barrier counters (one memset: they are contiguous), so a
// launch that gave up waiting cannot leave a later one out of step.
static cudaError_t begin_solve(Single &s, cudaStream_t stream)
{
    if (++s.solves >= (1u << 22)) {
        MST_TRY(cudaMemsetAsync(s.ws.desc, 0, (size_t)s.ws.desc_cap * 8, stream));
        MST_TRY(cudaMemsetAsync(&s.ws.ctl->epoch, 0, sizeof(uint32_t), stream));
        s.solves = 1;
    }
    char *from = (char *)&s.ws.ctl->status;
    char *to = (char *)(s.ws.bar + bar_words(kMaxGridBlocks));
    return cudaMemsetAsync(from, 0, (size_t)(to - from), stream);
}

cudaError_t single_launch(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                          uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n, uint32_t m,
                          cudaStream_t stream)
{
    MST_TRY(begin_solve(s, stream));
    const uint32_t vec = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)w) & 15u) == 0 ? 1u : 0u;
    if (s.schedule != 2) {
        const uint32_t *wp = (const uint32_t *)w;
        void *args[] = {(void *)&s.ws, (void *)&src, (void *)&dst, (void *)&wp, (void *)&out,
                        (void *)&out_count, (void *)&n, (void *)&m, (void *)&wt, (void *)&vec};
        return cudaLaunchCooperativeKernel((const void *)k_solve, dim3(s.grid_fused),
                                           dim3(kThreads), args, 0, stream);
    }
    k_init<<<s.grid_stream, kThreads, 0, stream>>>(s.ws, src, dst, w, out, out_count, n, m, wt,
                                                   vec);
    MST_TRY(cudaGetLastError());
    return cudaGraphLaunch(s.exec, stream);
}

// ------------------------------------------------------- per-kernel timing

// Replays a solve launching every kernel of the graph schedule on its own
// between two CUDA events (the graph's conditional nodes are replaced by
// host decisions read from the control block after each kernel).  Bytes
// follow the DRAM model: edge lists and per-vertex arrays, not the
// L2-resident label gathers and atomics.
cudaError_t single_profile(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                           uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n, uint32_t m,
                           cudaStream_t stream, std::vector<KernelProfile> &prof)
{
    prof.clear();
    MST_TRY(begin_solve(s, stream));
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
    const int gt = s.grid_tiles, gs = s.grid_stream;
    const double words = ((double)m + 31) / 32;
    rec("k_init", 8.0 * n + 4 * words, [&] {
        k_init<<<gs, kThreads, 0, stream>>>(s.ws, src, dst, w, out, out_count, n, m, wt, vec);
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
        const char *cname = r == 0 ? "k_compact<R0>" : "k_compact<R>";
        rec(cname, 0.0, [&] {
            if (r == 0)
                k_compact<true><<<gt, kThreads, 0, stream>>>(s.ws, none, 0u);
            else
                k_compact<false><<<gt, kThreads, 0, stream>>>(s.ws, none, 0u);
        });
        read_ctl();
        for (auto &k : prof)  // bytes need m_{r+1}, known only now
            if (k.name == cname)
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

// Algorithmic DRAM bytes of a whole solve from its per-round sizes: the
// caller's arrays read twice in round 0 (find-min, compaction), each later
// list read once and written once, per-vertex arrays per round, the tree
// bits and the output.
double single_alg_bytes(const Ctl &c)
{
    const double n = c.n, m = c.m;
    double b = 8.0 * n + m / 8.0;  // init: mins, bits
    b += 12.0 * m;                 // round-0 find-min
    for (uint32_t r = 0; r < c.round && r < (uint32_t)kMaxRounds; r++) {
        const double nr = c.stat_n[r], mr = c.stat_m[r], mn = c.stat_m[r + 1];
        const double nn = c.stat_n[r + 1];
        b += 20.0 * nr + 4.0 * nn;            // hook: mins in/out, parent, new ids
        b += 8.0 * nr + 4.0 * nn;             // compress: parent, labels, new ids
        b += (r == 0 ? 12.0 : 16.0) * mr;     // compaction reads the list
        b += 16.0 * mn;                        // and writes the survivors
    }
    b += m / 8.0 + 4.0 * (n > 0 ? n - 1 : 0);  // emit
    return b;
}

}  // namespace mst
