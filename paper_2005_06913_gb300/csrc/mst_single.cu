// mst_single.cu — data-parallel Boruvka rounds for one graph (Section 2.1)
// as hand-written sm_103a kernels.
//
// Round r works on a contracted graph: components are numbered 0..n_r-1 and
// the live edge list holds only edges between different components, with
// endpoints already renamed to component ids.  Per round:
//   find-min (Section 2.1, the loop over edges): every live edge offers its
//     key to both endpoint components with a 64-bit atomicMin (the key packs
//     the weight above the input edge id, so ties break by edge id); for
//     round r+1 this runs fused into round r's compaction.
//   hook (Section 2.1, the union step): every component c with a minimum
//     edge e to d points at d and marks e as a tree edge, except that of two
//     components that chose the same edge the lower id stays a root.  Under
//     a total order that mutual pair is the only cycle the pointers can
//     form, so they form a forest (the lock/CAS serialisation of Sections
//     2.2.1-2.2.2 is not needed).  Roots get new dense ids: each warp tile
//     takes a block of ids with one atomicAdd (the numbering is arbitrary;
//     the tree does not depend on it).
//   compress: each component follows its pointers to its root (path halving,
//     bounded hops per pass, more passes only while some chain is deep) and
//     takes the root's new id.
//   compact (Section 2.1 "Optimization", covered edges): edges whose two
//     renamed endpoints coincide are dropped; each warp tile writes its
//     survivors to a block of positions taken with one atomicAdd, and each
//     survivor offers its key for round r+1 (one that may win records its
//     new endpoints under its input id, for the next hook).
// The rounds stop when no live edge is left; the tree edges are then emitted
// in ascending id order.
//
// Two schedules run the same tile bodies:
//   fused  (default) one cooperative persistent launch, k_solve, walks every
//          phase of every round; phases are separated by a grid barrier
//          instead of kernel boundaries.
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
// Ablations of the fused solve (single-graph schedules 3 and 4)
constexpr uint32_t kVariantCovered = 1u;  // flag internal edges in place, no compaction
constexpr uint32_t kVariantCas = 2u;      // hook roots by compare-and-swap

struct TileSmem {
    uint4 stage[kTile];  // ids of an emit tile / per-component arrays of a one-CTA tail
    uint32_t s32[33];
    uint32_t s_tile, s_excl, s_flag;
};
static_assert(kTailLocalN * (8 + 4 + 4) <= sizeof(uint4) * kTile,
              "a one-CTA tail's minima, pointers and new ids fit the stage");

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

// Writes one group of 4 edges' fields to the device copy of the inputs
// (128-bit stores; the copy is 256-byte aligned and groups start at 4k).
__device__ __forceinline__ void store4_soa(int32_t *csrc, int32_t *cdst, uint32_t *cw, uint32_t e0,
                                           uint32_t m, const int32_t (&us)[4],
                                           const int32_t (&vs)[4], const uint32_t (&wr)[4])
{
    if (e0 + 3 < m) {
        *(int4 *)(csrc + e0) = make_int4(us[0], us[1], us[2], us[3]);
        *(int4 *)(cdst + e0) = make_int4(vs[0], vs[1], vs[2], vs[3]);
        *(uint4 *)(cw + e0) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
    } else {
        for (int j = 0; j < 4 && e0 + j < m; j++) {
            csrc[e0 + j] = us[j];
            cdst[e0 + j] = vs[j];
            cw[e0 + j] = wr[j];
        }
    }
}

// Round-0 find-min of one group of 4 edges starting at e0.  Its keys are
// (weight_bits << 32) | (edge id << 1) | side: edge ids are below 2^31, and
// the side bit (0: offered to src, 1: to dst) only rides along, since one
// edge offers once to each endpoint, so the order is still (weight, edge
// id); the hook then reads only the endpoint across from the component.
// With csrc non-null the inputs are read from mapped host memory and also
// copied to device memory (csrc, cdst, cw), which the later phases read.
__device__ __forceinline__ void find0_group(unsigned long long *mn, const int32_t *src,
                                            const int32_t *dst, const uint32_t *w, uint32_t n,
                                            uint32_t m, uint32_t wt, uint32_t vec,
                                            uint32_t *status, bool filtered, uint32_t e0,
                                            int32_t *csrc, int32_t *cdst, uint32_t *cw)
{
    int32_t us[4], vs[4];
    uint32_t wr[4];
    load4_soa(src, dst, w, e0, m, vec, us, vs, wr);
    if (csrc)
        store4_soa(csrc, cdst, cw, e0, m, us, vs, wr);
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
        const unsigned long long key = make_key(weight_bits(wr[j], wt, status), (e0 + j) << 1);
        if (filtered) {
            offer_min(&mn[u], key);
            offer_min(&mn[v], key | 1ull);
        } else {
            red_min_u64(&mn[u], key);
            red_min_u64(&mn[v], key | 1ull);
        }
    }
}

// Round-0 find-min over edge groups [g0, groups) step gstep.
__device__ __forceinline__ void find0_range(const Ws &ws, const int32_t *src, const int32_t *dst,
                                            const uint32_t *w, uint32_t n, uint32_t m, uint32_t wt,
                                            uint32_t vec, uint32_t *status, size_t g0,
                                            size_t gstep, int32_t *csrc = nullptr,
                                            int32_t *cdst = nullptr, uint32_t *cw = nullptr)
{
    const size_t groups = ((size_t)m + 3) >> 2;
    const bool filtered = use_filter(m, n);
    for (size_t g = g0; g < groups; g += gstep)
        find0_group(ws.mins[0], src, dst, w, n, m, wt, vec, status, filtered, (uint32_t)(g << 2),
                    csrc, cdst, cw);
}

// Round-0 find-min of one warp tile: kFind0Groups groups of 4 edges, lane l
// taking groups l, l + 32, ... of the tile (each load of the warp contiguous).
constexpr uint32_t kFind0Groups = 64;
constexpr uint32_t kFind0WTile = 4 * kFind0Groups;  // edges

__device__ __forceinline__ void find0_wtile(const Ws &ws, const int32_t *src, const int32_t *dst,
                                            const uint32_t *w, uint32_t n, uint32_t m, uint32_t wt,
                                            uint32_t vec, uint32_t *status, bool filtered,
                                            uint32_t tile, int32_t *csrc, int32_t *cdst,
                                            uint32_t *cw)
{
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (uint32_t j = 0; j < kFind0Groups / 32; j++) {
        const uint32_t e0 = tile * kFind0WTile + (j * 32 + lane) * 4;
        if (e0 < m)
            find0_group(ws.mins[0], src, dst, w, n, m, wt, vec, status, filtered, e0, csrc,
                        cdst, cw);
    }
}

// Runs body(t) for the warp tiles t < ntiles of a phase, balanced between
// warps.  The first kStaticShare of a warp's fair share is static (global
// warp gw takes tiles gw, gw + nw, ...); the rest of the tiles go to whichever
// warp asks next, from the phase's counter *ctr, so warps that drew slow
// tiles do not hold the phase's end.  A ticket is taken before the current
// tile's work, so its latency overlaps that work; a warp that draws a tile
// past the end leaves.  Every tile runs exactly once.  (All tiles from the
// counter made one address the bottleneck of the round-0 find-min: ~300 M
// tickets/s; with a quarter of them, the counter is no longer felt.)
constexpr uint32_t kStaticShareNum = 3, kStaticShareDen = 4, kDynMinShare = 4;

template <typename F>
__device__ __forceinline__ void for_warp_tiles(uint32_t *ctr, uint32_t ntiles, uint32_t gw,
                                               uint32_t nw, F &&body)
{
    const uint32_t lane = threadIdx.x & 31;
    // phases of fewer than kDynMinShare tiles per warp stay static: each warp
    // has too few tiles to balance, and a ticket's round trip would only
    // lengthen the phase (measured on the 1024 x 1024 grid's late rounds)
    const bool small = (unsigned long long)ntiles < (unsigned long long)kDynMinShare * nw;
    const uint32_t k_static =
        small ? (ntiles + nw - 1) / nw
              : (uint32_t)((unsigned long long)ntiles * kStaticShareNum /
                           ((unsigned long long)nw * kStaticShareDen));
    const uint32_t dyn0 = k_static * nw;  // tiles before this one are static
    // tile k of this warp: gw + k*nw while k < k_static, then dyn0 + gw (still
    // fixed), then dyn0 + nw + a ticket (one loop, so the body is inlined once)
    uint32_t k = 0, t = k_static ? gw : dyn0 + gw;
    while (t < ntiles) {
        uint32_t nx = 0;
        if (lane == 0 && k >= k_static)
            nx = atomicAdd(ctr, 1u);
        body(t);
        k++;
        if (k < k_static)
            t = gw + k * nw;
        else if (k == k_static)
            t = dyn0 + gw;
        else
            t = __shfl_sync(0xffffffffu, nx, 0) + dyn0 + nw;
    }
}

// Warp tiles: one warp owns a tile of kHookIpl*32 components or kCompIpl*32
// edges (item j of lane l is tile index j*32 + l, so every load of the warp
// is contiguous), ranks its items with ballots, takes a block of ids or
// positions with one atomicAdd on the round's counter and writes its
// results itself.  No block barrier and no wait on another warp is
// involved, so a warp waiting on memory never holds up the others.
constexpr int kHookIpl = 4, kCompIpl = 8;
constexpr int kHookWTile = 32 * kHookIpl, kCompWTile = 32 * kCompIpl;

// Hook one warp tile of components (Section 2.1, the union step) and give
// the tile's roots new ids from the round's counter.  The minimum key's tag
// is the input edge id: round 0 reads the input endpoints, later rounds the
// endpoints the edge recorded under its id when it was offered.
template <bool R0>
__device__ __forceinline__ void hook_wtile(const Ws &ws, Ctl *c, uint32_t tile, uint32_t round,
                                           uint32_t n_cur, const int32_t *src,
                                           const int32_t *dst)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long *mcur = (round & 1) ? ws.mins[1] : ws.mins[0];
    unsigned long long *mnext = (round & 1) ? ws.mins[0] : ws.mins[1];
    int32_t *parent = ws.parent;
    const uint32_t base = tile * kHookWTile;
    unsigned long long k[kHookIpl];
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        const uint32_t v = base + j * 32 + lane;
        k[j] = v < n_cur ? mcur[v] : kNoEdge;
    }
    uint32_t a[kHookIpl], b[kHookIpl], id[kHookIpl];
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        const uint32_t v = base + j * 32 + lane;
        if (v < n_cur)
            mnext[v] = kNoEdge;
        a[j] = b[j] = id[j] = 0;
        if (k[j] != kNoEdge) {
            const uint32_t p = (uint32_t)k[j];
            if (R0) {  // one gather: the endpoint across from v (side bit of the key)
                const uint32_t e = p >> 1;
                a[j] = (uint32_t)__ldg(((p & 1u) ? src : dst) + e);
                b[j] = a[j];
                id[j] = e;
            } else {
                const uint2 r = __ldcg(ws.eends + p);
                a[j] = r.x;
                b[j] = r.y;
                id[j] = p;
            }
        }
    }
    unsigned long long kd[kHookIpl];
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        const uint32_t v = base + j * 32 + lane;
        const uint32_t d = (a[j] == v) ? b[j] : a[j];
        a[j] = d;  // a now holds the other component
        kd[j] = k[j] != kNoEdge ? mcur[d] : kNoEdge;
        if (R0) {  // compare edge ids: the two sides of one edge differ in the side bit
            kd[j] >>= 1;
            k[j] = k[j] == kNoEdge ? kNoEdge : k[j] >> 1;
        }
    }
    uint32_t mask[kHookIpl], total = 0;
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        const uint32_t v = base + j * 32 + lane;
        bool root = false;
        if (v < n_cur) {
            const uint32_t d = a[j];
            if (k[j] == kNoEdge || ((uint32_t)kd[j] == (uint32_t)k[j] && v < d)) {
                root = true;  // no edge leaves it, or the lower id of a mutual pair
                parent[v] = (int32_t)v;
            } else {
                parent[v] = (int32_t)d;
                red_or_u32(&ws.mst_bits[id[j] >> 5], 1u << (id[j] & 31));
            }
        }
        mask[j] = __ballot_sync(0xffffffffu, root);
        total += __popc(mask[j]);
    }
    uint32_t ex = 0;
    if (lane == 0 && total)
        ex = atomicAdd(&c->cnt_n[round], total);
    ex = __shfl_sync(0xffffffffu, ex, 0);
    const uint32_t lt = lanemask_lt();
    uint32_t run = ex;
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        if ((mask[j] >> lane) & 1u)
            ws.nid[base + j * 32 + lane] = (int32_t)(run + __popc(mask[j] & lt));
        run += __popc(mask[j]);
    }
}

// The CAS-hook ablation (Section 2.2.2 on the GPU): each component with a
// minimum edge joins the current trees of the edge's endpoints by one
// compare-and-swap of a root's parent, while other threads do the same.
// The higher-numbered root is hooked under the lower one, not the edge's
// destination under its source: a root found first may be hooked before
// the swap, and with a fixed edge direction that stale root can already
// hang below the other one (a cycle); pointers that only ever go to lower
// ids cannot close one.  Keys are totally ordered, so the minima of a round
// are edges of the one minimum spanning forest: a failed swap only means
// the root was hooked meanwhile (the finds are retried), and endpoints
// found in one tree mean the edge was already added by the other component
// it leaves.  Whether a component stays a root is known only after every
// swap, so the roots are numbered in a phase of their own.
constexpr uint32_t kCasRetryLimit = 1u << 16;
constexpr uint32_t kNoRoot = 0xffffffffu;

// Root of x while other threads hook roots: path halving.  Only a root's
// pointer is swapped, and a non-root's pointer only moves to an ancestor, so
// every pointer read stays an ancestor, ids fall along a path and a path has
// fewer than n_cur hops (more would mean a broken forest: the status is set
// and the find gives up).  Reads bypass L1: pointers change during the phase.
__device__ __forceinline__ uint32_t cas_find(int32_t *parent, uint32_t x, uint32_t n_cur,
                                             uint32_t *status)
{
    for (uint32_t s = 0; s <= n_cur; s++) {
        const uint32_t p = (uint32_t)__ldcg(parent + x);
        if (p == x)
            return x;
        const uint32_t gp = (uint32_t)__ldcg(parent + p);
        if (gp != p)
            __stcg(parent + x, (int32_t)gp);
        x = gp;
    }
    atomicOr(status, ST_INTERNAL);
    return kNoRoot;
}

template <bool R0>
__device__ __forceinline__ void hook_cas_wtile(const Ws &ws, Ctl *c, uint32_t tile,
                                               uint32_t round, uint32_t n_cur,
                                               const int32_t *src, const int32_t *dst)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long *mcur = (round & 1) ? ws.mins[1] : ws.mins[0];
    unsigned long long *mnext = (round & 1) ? ws.mins[0] : ws.mins[1];
    int32_t *parent = ws.parent;
    uint32_t *status = &c->status;
    const uint32_t base = tile * kHookWTile;
#pragma unroll 1
    for (int j = 0; j < kHookIpl; j++) {
        const uint32_t v = base + j * 32 + lane;
        if (v >= n_cur)
            continue;
        const unsigned long long k = mcur[v];
        mnext[v] = kNoEdge;
        if (k == kNoEdge)
            continue;
        uint32_t p = (uint32_t)k;
        uint32_t a, b;
        if (R0) {  // the round-0 key carries a side bit below the edge id
            p >>= 1;
            a = v;
            b = (uint32_t)__ldg((((uint32_t)k & 1u) ? src : dst) + p);
        } else {
            const uint2 e = __ldcg(ws.eends + p);
            a = e.x;
            b = e.y;
        }
        bool joined = false;
        for (uint32_t t = 0; t < kCasRetryLimit && !joined; t++) {
            const uint32_t c1 = cas_find(parent, a, n_cur, status);
            const uint32_t c2 = cas_find(parent, b, n_cur, status);
            const uint32_t lo = c1 < c2 ? c1 : c2, hi = c1 < c2 ? c2 : c1;
            if (c1 == kNoRoot || c2 == kNoRoot || c1 == c2)
                joined = true;  // (or given up, with the status set)
            else if ((uint32_t)atomicCAS(parent + hi, (int32_t)hi, (int32_t)lo) == hi) {
                red_or_u32(&ws.mst_bits[p >> 5], 1u << (p & 31));
                joined = true;
            }
        }
        if (!joined)
            atomicOr(status, ST_INTERNAL);
    }
}

// New ids of the roots left after the CAS hooks (one warp tile).
__device__ __forceinline__ void number_roots_wtile(const Ws &ws, Ctl *c, uint32_t tile,
                                                   uint32_t round, uint32_t n_cur)
{
    const int lane = threadIdx.x & 31;
    const uint32_t base = tile * kHookWTile;
    uint32_t mask[kHookIpl], total = 0;
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        const uint32_t v = base + j * 32 + lane;
        const bool root = v < n_cur && (uint32_t)__ldcg(ws.parent + v) == v;
        mask[j] = __ballot_sync(0xffffffffu, root);
        total += __popc(mask[j]);
    }
    uint32_t ex = 0;
    if (lane == 0 && total)
        ex = atomicAdd(&c->cnt_n[round], total);
    ex = __shfl_sync(0xffffffffu, ex, 0);
    const uint32_t lt = lanemask_lt();
    uint32_t run = ex;
#pragma unroll
    for (int j = 0; j < kHookIpl; j++) {
        if ((mask[j] >> lane) & 1u)
            ws.nid[base + j * 32 + lane] = (int32_t)(run + __popc(mask[j] & lt));
        run += __popc(mask[j]);
    }
}

// One compress pass over components [v0, n_cur) step vstep: each thread
// follows the hook pointers of kCompressU components in lock step (path
// halving, at most kChaseLimit steps), so their loads overlap, and gives
// each the new id of its root; a component whose chase did not end keeps
// lab = -1 and its pointer moved up the chain for the next pass.  Pointer
// loads may come from L1: every value a pointer has held in this pass is an
// ancestor, so an older one only shortens the step.
constexpr int kCompressU = 2;

__device__ __forceinline__ bool compress_range(const Ws &ws, uint32_t n_cur, bool first,
                                               size_t v0, size_t vstep)
{
    int32_t *parent = ws.parent;
    bool unfinished = false;
    for (size_t b0 = v0; b0 < n_cur; b0 += kCompressU * vstep) {
        uint32_t x[kCompressU];
        bool act[kCompressU];
#pragma unroll
        for (int i = 0; i < kCompressU; i++) {
            const size_t v = b0 + i * vstep;
            act[i] = v < n_cur;
            x[i] = (uint32_t)v;
        }
        if (!first) {  // follow-up pass: only components left unfinished
#pragma unroll
            for (int i = 0; i < kCompressU; i++)
                act[i] = act[i] && __ldcg(ws.lab + x[i]) == -1;
#pragma unroll
            for (int i = 0; i < kCompressU; i++)
                x[i] = act[i] ? (uint32_t)__ldcg(parent + x[i]) : x[i];
        }
        uint32_t root[kCompressU];
        bool done[kCompressU];
#pragma unroll
        for (int i = 0; i < kCompressU; i++) {
            done[i] = !act[i];
            root[i] = 0;
        }
#pragma unroll 1
        for (int s = 0; s < kChaseLimit; s++) {
            uint32_t p[kCompressU], gp[kCompressU];
#pragma unroll
            for (int i = 0; i < kCompressU; i++)
                p[i] = done[i] ? 0u : (uint32_t)__ldca(parent + x[i]);
#pragma unroll
            for (int i = 0; i < kCompressU; i++) {
                if (!done[i] && p[i] == x[i]) {
                    root[i] = x[i];
                    done[i] = true;
                }
            }
#pragma unroll
            for (int i = 0; i < kCompressU; i++)
                gp[i] = done[i] ? 0u : (uint32_t)__ldca(parent + p[i]);
            bool more = false;
#pragma unroll
            for (int i = 0; i < kCompressU; i++) {
                if (done[i])
                    continue;
                if (gp[i] == p[i]) {
                    root[i] = p[i];
                    done[i] = true;
                } else {
                    __stcg(parent + x[i], (int32_t)gp[i]);
                    x[i] = gp[i];
                    more = true;
                }
            }
            if (!more)
                break;
        }
        int32_t nl[kCompressU];
#pragma unroll
        for (int i = 0; i < kCompressU; i++)
            nl[i] = act[i] && done[i] ? __ldca(ws.nid + root[i]) : -1;
#pragma unroll
        for (int i = 0; i < kCompressU; i++) {
            if (!act[i])
                continue;
            const uint32_t v = (uint32_t)(b0 + i * vstep);
            ws.lab[v] = nl[i];
            if (!done[i]) {
                __stcg(parent + v, (int32_t)x[i]);
                unfinished = true;
            }
        }
    }
    return unfinished;
}

// The "covered" ablation (the sequential optimisation of Section 2.1 kept
// on the GPU as a flag): the list keeps all m slots in E[1] and a slot whose
// edge has become internal is overwritten by this marker, whose first
// endpoint is never a component id; later rounds read and skip it.
constexpr uint32_t kDeadEdge = 0xffffffffu;

__device__ __forceinline__ uint4 *edge_list(const Ws &ws, uint32_t round, bool covered, bool next)
{
    if (covered)
        return ws.E[1];
    return ((round & 1) != 0) != next ? ws.E[1] : ws.E[0];
}

// Compaction of one warp tile of round r's live edges fused with find-min
// of round r+1: survivors are written from registers to a block of
// positions taken from the round's counter (one contiguous run per row of
// the tile), possible minima record their new endpoints by input id, and
// they offer their (weight, id) keys with fire-and-forget reductions.  In
// the covered ablation survivors are rewritten in their own slot and newly
// internal edges are flagged there instead.
template <bool R0, bool covered = false>
__device__ __forceinline__ void compact_wtile(const Ws &ws, Ctl *c, uint32_t tile,
                                              uint32_t round, uint32_t m_cur, uint32_t n_next,
                                              uint32_t n_in,
                                              uint32_t wt, const int32_t *src, const int32_t *dst,
                                              const uint32_t *w, uint32_t m_live = 0)
{
    const int lane = threadIdx.x & 31;
    const uint4 *ecur = edge_list(ws, round, covered, false);
    uint4 *enext = edge_list(ws, round, covered, true);
    unsigned long long *mnext = (round & 1) ? ws.mins[0] : ws.mins[1];
    const int32_t *__restrict__ lab = ws.lab;
    uint32_t *status = &c->status;
    const uint32_t base = tile * kCompWTile;
    uint4 rec[kCompIpl];
    bool ok[kCompIpl];
#pragma unroll
    for (int j = 0; j < kCompIpl; j++) {
        const uint32_t i = base + j * 32 + lane;
        const bool in = i < m_cur;
        if (R0) {
            const uint32_t u = in ? (uint32_t)__ldg(src + i) : 0u;
            const uint32_t v = in ? (uint32_t)__ldg(dst + i) : 0u;
            const uint32_t x = in ? __ldg(w + i) : 0u;
            ok[j] = in && u < n_in && v < n_in && u != v;
            rec[j] = make_uint4(u, v, x, i);
        } else {
            rec[j] = in ? ecur[i] : make_uint4(0, 0, 0, 0);
            ok[j] = in && rec[j].x != kDeadEdge;
        }
    }
    uint32_t mask[kCompIpl], total = 0;
#pragma unroll
    for (int j = 0; j < kCompIpl; j++) {
        bool keep = false;
        if (ok[j]) {
            const uint32_t nu = (uint32_t)lab[rec[j].x], nv = (uint32_t)lab[rec[j].y];
            if (nu >= n_next || nv >= n_next) {
                atomicOr(status, ST_INTERNAL);  // never for a valid forest
            } else if (nu != nv) {
                keep = true;
                rec[j].x = nu;
                rec[j].y = nv;
                if (R0)
                    rec[j].z = weight_bits(rec[j].z, wt, status);
            }
        }
        mask[j] = __ballot_sync(0xffffffffu, keep);
        total += __popc(mask[j]);
    }
    uint32_t ex = 0;
    if (lane == 0 && total)
        ex = atomicAdd(&c->cnt_m[round], total);
    ex = __shfl_sync(0xffffffffu, ex, 0);
    const uint32_t lt = lanemask_lt();
    const bool filtered = use_filter(covered ? m_live : m_cur, n_next);
    uint32_t run = ex;
#pragma unroll
    for (int j = 0; j < kCompIpl; j++) {
        const uint32_t i = base + j * 32 + lane;
        // flagged, not removed: every slot of round 0, later only new ones
        if (covered && !((mask[j] >> lane) & 1u) && (R0 ? i < m_cur : ok[j]))
            enext[i] = make_uint4(kDeadEdge, kDeadEdge, 0u, 0u);
        if ((mask[j] >> lane) & 1u) {
            const uint32_t pos = covered ? i : run + __popc(mask[j] & lt);
            enext[pos] = rec[j];
            const unsigned long long key = make_key(rec[j].z, rec[j].w);
            // Only an edge that passes a filter can end up as a minimum (the
            // minimum only decreases), so only those record their endpoints
            // for the next hook.
            bool may_win = true;
            if (filtered) {
                may_win = offer_min(&mnext[rec[j].x], key);
                may_win |= offer_min(&mnext[rec[j].y], key);
            } else {
                red_min_u64(&mnext[rec[j].x], key);
                red_min_u64(&mnext[rec[j].y], key);
            }
            if (may_win)
                __stcg(ws.eends + rec[j].w, make_uint2(rec[j].x, rec[j].y));
        }
        run += __popc(mask[j]);
    }
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
    const int nwarps = (int)(blockDim.x >> 5);
    if (warp == 0) {
        const uint32_t v = lane < nwarps ? sm.s32[lane] : 0u;
        uint32_t inc2 = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc2, o);
            if (lane >= o)
                inc2 += y;
        }
        if (lane < nwarps)
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
    for (uint32_t k = threadIdx.x; k < total; k += blockDim.x) {
        if (ex + k < cap)
            out[ex + k] = (int32_t)ids[k];
        else
            atomicOr(&c->status, ST_INTERNAL);  // more tree edges than n-1
    }
    __syncthreads();
}

// Emit of the fused schedule, in two passes with a grid barrier between
// them instead of a look-back.  Each CTA owns a contiguous range of groups
// of 32 bit words.  First every group counts its tree edges (one warp a
// group) and each CTA stores its range's total; then each CTA sums the
// totals of the CTAs before it (one load per thread), and its warps write
// the ids of its groups in order.  (Summing the groups' own counts instead
// took one dependent L2 load per 1,024 groups per thread: 23 us on R-MAT 22.)
template <int kFT>
__device__ __forceinline__ void emit_count(const Ws &ws, uint32_t words, uint32_t ngroups,
                                           TileSmem &sm)
{
    constexpr int kFW = kFT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (ngroups + gridDim.x - 1) / gridDim.x;
    const uint32_t t0 = blockIdx.x * per;
    const uint32_t t1 = t0 + per < ngroups ? t0 + per : ngroups;
    uint32_t sum = 0;
    for (uint32_t t = t0 + warp; t < t1; t += kFW) {
        const uint32_t i = t * 32 + lane;
        uint32_t cnt = i < words ? __popc(__ldcg(ws.mst_bits + i)) : 0u;
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0)
            ws.emit_cnt[t] = cnt;
        sum += cnt;
    }
    if (lane == 0)
        sm.s32[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t total = 0;
        for (int k = 0; k < kFW; k++)
            total += sm.s32[k];
        ws.emit_cta[blockIdx.x] = total;
    }
}

// Position of the set bit of rank r (0-based) in w (w has more than r set
// bits): the smallest p with more than r set bits in w[0..p].
__device__ __forceinline__ uint32_t select_bit(uint32_t w, uint32_t r)
{
    uint32_t lo = 0, hi = 31;
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint32_t)__popc(w & ((2u << mid) - 1u)) > r)  // 2u << 31 wraps to 0: all bits
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Writes the ids of groups [t0, t1) (this CTA's contiguous range) in
// ascending order.  The CTA sums the counts of all groups before t0, then
// takes its range in windows that fit the stage: warp 0 scans a window's
// counts into shared memory and the warps expand its groups on their own,
// one group of 32 words each: lane k of an output step finds the word
// holding the k-th id by a binary search over the warp's scanned counts and
// the bit by select_bit, so the writes are coalesced.
template <int kFT>
__device__ __forceinline__ void emit_range(const Ws &ws, Ctl *c, uint32_t ngroups, uint32_t words,
                                           uint32_t cap, int32_t *out, TileSmem &sm)
{
    constexpr int kFW = kFT / 32;
    constexpr uint32_t kWindow = sizeof(sm.stage) / 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (ngroups + gridDim.x - 1) / gridDim.x;
    const uint32_t t0 = blockIdx.x * per;
    const uint32_t t1 = t0 + per < ngroups ? t0 + per : ngroups;
    if (t0 >= t1)
        return;
    uint32_t part = 0;
    for (uint32_t b = threadIdx.x; b < blockIdx.x; b += kFT)
        part += __ldcg(ws.emit_cta + b);
    part = __reduce_add_sync(0xffffffffu, part);
    if (lane == 0)
        sm.s32[warp] = part;
    __syncthreads();
    uint32_t run = 0;  // ids before the current window (kept by every thread)
#pragma unroll
    for (int k = 0; k < kFW; k++)
        run += sm.s32[k];
    uint32_t *offs = (uint32_t *)sm.stage;  // exclusive offset of each group of the window
    for (uint32_t w0 = t0; w0 < t1; w0 += kWindow) {
        const uint32_t w1 = w0 + kWindow < t1 ? w0 + kWindow : t1;
        __syncthreads();  // the previous window's offsets are no longer read
        if (warp == 0) {
            uint32_t r = run;
            for (uint32_t b = w0; b < w1; b += 32) {
                const uint32_t t = b + lane;
                const uint32_t v = t < w1 ? __ldcg(ws.emit_cnt + t) : 0u;
                uint32_t incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                if (t < w1)
                    offs[t - w0] = r + incl - v;
                r += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0)
                sm.s32[32] = r;
        }
        __syncthreads();
        for (uint32_t t = w0 + warp; t < w1; t += kFW) {
            const uint32_t base = offs[t - w0];
            const uint32_t wi = t * 32 + lane;
            const uint32_t wv = wi < words ? __ldcg(ws.mst_bits + wi) : 0u;
            const uint32_t cnt = __popc(wv);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            const uint32_t excl = incl - cnt;
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            for (uint32_t k0 = 0; k0 < total; k0 += 32) {
                const uint32_t k = k0 + lane;
                // the word j holding the id of rank k: the last with excl_j <= k
                uint32_t j = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t e = __shfl_sync(0xffffffffu, excl, (int)(j + step));
                    if (e <= k)
                        j += step;
                }
                const uint32_t wj = __shfl_sync(0xffffffffu, wv, (int)j);
                const uint32_t ej = __shfl_sync(0xffffffffu, excl, (int)j);
                if (k < total) {
                    const uint32_t id = (t * 32 + j) * 32u + select_bit(wj, k - ej);
                    if (base + k < cap)
                        out[base + k] = (int32_t)id;
                    else
                        atomicOr(&c->status, ST_INTERNAL);  // more tree edges than n-1
                }
            }
        }
        run = sm.s32[32];
    }
    if (threadIdx.x == 0 && t1 == ngroups)
        c->emitted = run;
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

// Grid barrier for a co-resident (cooperative) grid.  One counter: block 0
// adds 2^31 - (grid - 1) and every other block adds 1, so the counter's top
// bit flips exactly when the last block arrives and its low bits return to
// where they were; each block spins until the top bit differs from the
// value it saw when it arrived.  One atomic per block, nothing to reset.
// Thread 0 arrives with a gpu-scope release atomic and polls with
// gpu-scope acquire loads; the block barriers before and after make the
// pattern cover every thread of the CTA (the PTX model's release is
// cumulative over what bar.sync ordered before it).  Measured against full
// fences around a relaxed atomic: grid 1024^2 0.340 -> 0.323 ms, random
// 4,096 / 32,768 0.116 -> 0.109 ms.
// Waits are bounded (spin_limit polls; 0 means kBarSpinLimit): on expiry
// ST_TIMEOUT is set, later barriers no longer wait, and the barrier tells
// every thread of the CTA to abandon the solve.
constexpr uint32_t kBarCount = 0;
constexpr uint32_t kBarSpinLimit = 1u << 22;

// Barrier among CTAs [0, nb) (all co-resident).  Returns true in every
// thread of the CTA when the solve has timed out (this CTA's wait ran out,
// or another CTA's did before): the data of the phase just ended may then
// be incomplete, so the caller must not start the next phase.  The outcome
// is read once by thread 0 and broadcast, so a CTA never splits on it.
__device__ __forceinline__ bool team_sync(uint32_t *counter, uint32_t nb, uint32_t *status,
                                          uint32_t spin_limit)
{
    __shared__ uint32_t s_abort;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t limit = spin_limit ? spin_limit : kBarSpinLimit;
        const uint32_t inc = blockIdx.x == 0 ? 0x80000000u - (nb - 1) : 1u;
        uint32_t old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;"
                     : "=r"(old)
                     : "l"(counter), "r"(inc)
                     : "memory");
        uint32_t spins = 0;
        for (;;) {
            uint32_t now;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(counter) : "memory");
            if (((old ^ now) & 0x80000000u) != 0)
                break;
            if (++spins > limit) {
                atomicOr(status, ST_TIMEOUT);
                if (!spin_limit)  // a real give-up, not an injected short limit
                    printf("mst: grid barrier gave up: block %u of %u, arrival value %u, now %u\n",
                           blockIdx.x, nb, old, now);
                break;
            }
            if ((spins & 15) == 0 && (ld_volatile_u32(status) & ST_TIMEOUT))
                break;  // another CTA gave up: stop waiting
            if (spins > 64)
                __nanosleep(32);
        }
        s_abort = (ld_volatile_u32(status) & ST_TIMEOUT) ? 1u : 0u;
    }
    __syncthreads();
    return s_abort != 0u;
}

__device__ __forceinline__ bool grid_sync(uint32_t *bar, uint32_t &gen, uint32_t *status,
                                          uint32_t spin_limit)
{
    gen++;
    return team_sync(bar + kBarCount, gridDim.x, status, spin_limit);
}

constexpr uint32_t kBarTeam = 32;  // counter of the tail's sub-grid team (own 128-B line)

size_t bar_words(int) { return 64; }

// CTA 0 stamps when its own work of a phase is done (before the barrier)
// and when the phase ends (everyone has passed the barrier).
__device__ __forceinline__ void mark_work(Ctl *c)
{
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t i = c->nphase;
        if (i < (uint32_t)kMaxPhaseLog)
            c->work_ns[i] = global_timer_ns();
    }
}

__device__ __forceinline__ void log_phase(Ctl *c, uint8_t kind, uint32_t round = 0)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t i = c->nphase;
        if (i < (uint32_t)kMaxPhaseLog) {
            c->phase_kind[i] = kind;
            c->phase_round[i] = (uint8_t)(round < 255 ? round : 255);
            c->phase_ns[i] = global_timer_ns();
            c->nphase = i + 1;
        }
    }
}

// ----------------------------------------------------------------- the tail
//
// Once a round leaves at most kTailMaxN components, that round's compaction
// does not write a next edge list: every surviving edge offers its key
// (weight_bits, input id) to a dense table with one slot per component pair
// (a < b).  Of parallel edges between the same two components only the
// lightest can be in the tree (a heavier one closes a cycle with it), so the
// table's non-empty slots are the whole remaining problem.  They become a
// short list, and each tail round then runs on it:
//   hook by edge: an edge that is the minimum of an endpoint hooks it (the
//     list needs no order: the key names the edge);
//   roots: every component finds its root; roots take dense new ids;
//   merge: each edge between two different new components offers its key to
//     the slot of that pair (fire-and-forget);
//   next list: the non-empty slots of the new components' table, read and
//     reset, are the next round's list and offer their keys to their
//     components (the next find-min).
// So parallel edges are merged every round, and a round costs O(list) plus
// a scan of the (shrinking) table of the new components' pairs.  The rounds
// run on a team of CTAs sized to the list (one CTA per
// kTailEdgesPerThread edges a thread, never growing): a team of one keeps
// the per-component arrays in shared memory once at most kTailLocalN
// components are left, and syncs with block barriers,
// a larger team keeps them in global memory and syncs with a barrier among
// its own CTAs.

// Appends the lanes' kept records to `list` (one atomic per warp).
__device__ __forceinline__ void warp_append(uint4 *list, uint32_t *counter, bool keep,
                                            const uint4 &rec)
{
    const uint32_t mask = __ballot_sync(0xffffffffu, keep);
    if (!mask)
        return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader)
        base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep)
        list[base + __popc(mask & lanemask_lt())] = rec;
}

// Appends the lanes' kept words to `list` (one atomic per warp).
__device__ __forceinline__ void warp_append_u32(uint32_t *list, uint32_t *counter, bool keep,
                                                uint32_t x)
{
    const uint32_t mask = __ballot_sync(0xffffffffu, keep);
    if (!mask)
        return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader)
        base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep)
        list[base + __popc(mask & lanemask_lt())] = x;
}

// Tail-mode compaction of one warp tile: edges between different components
// of round r+1 offer (weight_bits, input id) to their pair's slot.
template <bool R0>
__device__ __forceinline__ void compact_pairs_wtile(const Ws &ws, Ctl *c, uint32_t tile,
                                                    uint32_t round, uint32_t m_cur,
                                                    uint32_t n_next, uint32_t n_in, uint32_t wt,
                                                    const int32_t *src, const int32_t *dst,
                                                    const uint32_t *w, bool covered)
{
    const int lane = threadIdx.x & 31;
    const uint4 *ecur = edge_list(ws, round, covered, false);
    const int32_t *lab = ws.lab;
    uint32_t *status = &c->status;
    const uint32_t base = tile * kCompWTile;
#pragma unroll
    for (int j = 0; j < kCompIpl; j++) {
        const uint32_t i = base + j * 32 + lane;
        if (i >= m_cur)
            continue;
        uint4 rec;
        bool ok;
        if (R0) {
            rec = make_uint4((uint32_t)__ldg(src + i), (uint32_t)__ldg(dst + i), __ldg(w + i), i);
            ok = rec.x < n_in && rec.y < n_in && rec.x != rec.y;
        } else {
            rec = ecur[i];
            ok = rec.x != kDeadEdge;
        }
        if (!ok)
            continue;
        const uint32_t nu = (uint32_t)lab[rec.x], nv = (uint32_t)lab[rec.y];
        if (nu >= n_next || nv >= n_next) {
            atomicOr(status, ST_INTERNAL);
            continue;
        }
        if (nu == nv)
            continue;
        const uint32_t wb = R0 ? weight_bits(rec.z, wt, status) : rec.z;
        const uint32_t a = nu < nv ? nu : nv, b = nu < nv ? nv : nu;
        offer_min(&ws.pair_tab[(size_t)a * n_next + b], make_key(wb, rec.w));
    }
}

// Gathers the non-empty pair slots into tail list 0 (grid-stride), resets
// them, and offers each pair's key to both of its components (find-min of
// the first tail round).
__device__ __forceinline__ void extract_pairs(const Ws &ws, Ctl *c, uint32_t n_t, size_t i0,
                                              size_t step)
{
    const size_t total = (size_t)n_t * n_t;
    const size_t rounds = (total + step - 1) / step;  // every lane runs the same trip count
    for (size_t k = 0; k < rounds; k++) {
        const size_t i = i0 + k * step;
        bool keep = false;
        uint4 rec = make_uint4(0, 0, 0, 0);
        if (i < total) {
            const uint32_t a = (uint32_t)(i / n_t), b = (uint32_t)(i % n_t);
            if (a < b) {
                const unsigned long long key = __ldcg(ws.pair_tab + i);
                if (key != kNoEdge) {
                    keep = true;
                    rec = make_uint4(a, b, (uint32_t)(key >> 32), (uint32_t)key);
                    ws.pair_tab[i] = kNoEdge;
                    offer_min(&ws.tmin[a], key);
                    offer_min(&ws.tmin[b], key);
                }
            }
        }
        warp_append(ws.tl[0], &c->tail_cnt[0], keep, rec);
    }
}

// The tail rounds on list 0 (m_r pairs among n_r components, whose minimum
// keys are already in ws.tmin and whose hook pointers are the identity).
// Every CTA of the grid enters; CTAs outside a round's team leave.  CTA 0
// always stays and records the components left in c->tail_added.
constexpr int kTailU = 4;
constexpr uint32_t kTailEdgesPerThread = 4;  // swept 2..64: 4 is fastest on small graphs

template <int kFT>
__device__ void tail_rounds(const Ws &ws, Ctl *c, uint32_t n_r, uint32_t m_r, uint32_t r_base,
                            TileSmem &sm, uint32_t spin_limit)
{
    const uint32_t bid = blockIdx.x;
    const uint32_t n_t = n_r;
    uint32_t team_prev = gridDim.x;
    volatile unsigned long long *tmin = ws.tmin;
    volatile int32_t *tpar = ws.tpar;
    volatile int32_t *tnid = ws.tnid;
    bool local = false;  // per-component arrays in shared memory (team of one)
    uint32_t cur = 0;
    uint32_t rounds = 0;
    for (uint32_t tr = 0; m_r > 0; tr++, rounds++) {
        if (tr + 1 >= (uint32_t)kMaxRounds) {
            if (bid == 0 && threadIdx.x == 0)
                atomicOr(&c->status, ST_INTERNAL);
            break;
        }
        constexpr uint32_t kPer = kTailEdgesPerThread * kFT;
        uint32_t team = (m_r + kPer - 1) / kPer;
        team = team < 1 ? 1 : (team > team_prev ? team_prev : team);
        if (bid >= team)
            return;
        if (team == 1 && !local && n_r <= kTailLocalN) {  // CTA 0 alone: arrays into smem
            unsigned long long *smin = (unsigned long long *)sm.stage;
            int32_t *spar = (int32_t *)(smin + kTailLocalN);
            int32_t *snid = spar + kTailLocalN;
            for (uint32_t v = threadIdx.x; v < n_r; v += kFT) {
                smin[v] = __ldcg(ws.tmin + v);
                spar[v] = (int32_t)v;
            }
            __syncthreads();
            tmin = smin;
            tpar = spar;
            tnid = snid;
            local = true;
        }
        team_prev = team;
        bool aborted = false;  // a team barrier ran out: leave (the grid barrier after
                               // the tail then sees the timeout and ends the solve)
        auto sync = [&]() {
            if (team > 1)
                aborted = aborted || team_sync(ws.bar + kBarTeam, team, &c->status, spin_limit);
            else
                __syncthreads();
        };
        const size_t tid = (size_t)bid * kFT + threadIdx.x;
        const size_t nthr = (size_t)team * kFT;
        const uint4 *L = ws.tl[cur];
        uint4 *Ln = ws.tl[cur ^ 1];
        // hook by edge
        for (size_t e0 = tid; e0 < m_r; e0 += kTailU * nthr) {
            uint4 r[kTailU];
#pragma unroll
            for (int k = 0; k < kTailU; k++) {
                const size_t e = e0 + k * nthr;
                r[k] = e < m_r ? __ldcg(L + e) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < kTailU; k++) {
                if (e0 + k * nthr >= m_r)
                    continue;
                const unsigned long long key = make_key(r[k].z, r[k].w);
                const uint32_t a = r[k].x, b = r[k].y;
                const bool ha = tmin[a] == key, hb = tmin[b] == key;
                if (!ha && !hb)
                    continue;
                if (ha && hb)  // mutual: the lower id stays root
                    tpar[a > b ? a : b] = (int32_t)(a < b ? a : b);
                else if (ha)
                    tpar[a] = (int32_t)b;
                else
                    tpar[b] = (int32_t)a;
                red_or_u32(&ws.mst_bits[r[k].w >> 5], 1u << (r[k].w & 31));
            }
        }
        sync();
        if (aborted)
            return;
        // roots: full path compression (any pointer value read is an
        // ancestor); roots take dense new ids
        uint32_t *nn = &c->tail_nn[tr];
        for (size_t v = tid; v < n_r; v += nthr) {
            uint32_t x = (uint32_t)v;
            for (uint32_t hop = 0; hop < n_r; hop++) {  // a forest: depth < n_r
                const uint32_t p = (uint32_t)tpar[x];
                if (p == x)
                    break;
                x = p;
            }
            if (x == (uint32_t)v)
                tnid[v] = (int32_t)atomicAdd(nn, 1u);
            else
                tpar[v] = (int32_t)x;
        }
        sync();
        if (aborted)
            return;
        const uint32_t n_next = ld_volatile_u32(nn);
        // merge: relabel, offer each key to its pair's slot (fire-and-forget:
        // no thread waits on the table here)
        for (size_t e = tid; e < m_r; e += nthr) {
            const uint4 r = __ldcg(L + e);
            const uint32_t A = (uint32_t)tnid[tpar[r.x]], B = (uint32_t)tnid[tpar[r.y]];
            if (A != B)
                red_min_u64(ws.pair_tab + (A < B ? A : B) * n_next + (A < B ? B : A),
                            make_key(r.z, r.w));
        }
        for (size_t v = tid; v < n_next; v += nthr)
            tmin[v] = kNoEdge;
        sync();
        if (aborted)
            return;
        // next list: the non-empty slots of the n_next x n_next table, reset;
        // find-min of the next round.  (A scan of the table replaced recording
        // first writers, which cost each merge offer a returning atomic: on
        // the 4,096 / 32,768 random graph the first tail round took 20 us.)
        uint32_t *touched = &c->tail_cnt[tr + 1];
        const size_t slots = (size_t)n_next * n_next;
        const size_t steps = (slots + nthr - 1) / nthr;  // every lane runs the same trip count
        for (size_t k = 0; k < steps; k++) {
            const size_t i = tid + k * nthr;
            bool keep = false;
            uint4 rec = make_uint4(0, 0, 0, 0);
            if (i < slots) {
                const uint32_t a = (uint32_t)(i / n_next), b = (uint32_t)(i % n_next);
                if (a < b) {
                    const unsigned long long key = __ldcg(ws.pair_tab + i);
                    if (key != kNoEdge) {
                        keep = true;
                        ws.pair_tab[i] = kNoEdge;
                        rec = make_uint4(a, b, (uint32_t)(key >> 32), (uint32_t)key);
                        if (local) {
                            atomicMin((unsigned long long *)&tmin[a], key);
                            atomicMin((unsigned long long *)&tmin[b], key);
                        } else {
                            offer_min(ws.tmin + a, key);
                            offer_min(ws.tmin + b, key);
                        }
                    }
                }
            }
            warp_append(Ln, touched, keep, rec);
        }
        for (size_t v = tid; v < n_next; v += nthr)
            tpar[v] = (int32_t)v;
        sync();
        if (aborted)
            return;
        const uint32_t m_next = ld_volatile_u32(touched);
        if (bid == 0 && threadIdx.x == 0 && r_base + tr + 1 <= (uint32_t)kMaxRounds) {
            c->stat_m[r_base + tr + 1] = m_next;
            c->stat_n[r_base + tr + 1] = n_next;
        }
        m_r = m_next;
        n_r = n_next;
        cur ^= 1;
    }
    if (bid == 0 && threadIdx.x == 0) {
        c->tail_added = n_t - n_r;
        c->tail_rounds = rounds;
    }
}

// ------------------------------------------------- fused persistent kernel

// The whole solve in one cooperative launch of kFT-thread CTAs (64
// registers a thread at any size: 256 x 4, 512 x 2 or 1024 x 1 per SM).
// Warp tiles are assigned statically (tile t to global warp t mod warps);
// no phase waits on another CTA except at the grid barriers.
template <int kFT>
__global__ void __launch_bounds__(kFT, 1024 / kFT)
k_solve(Ws ws, const int32_t *src, const int32_t *dst, const uint32_t *w, int32_t *out,
        int64_t *out_count, uint32_t n, uint32_t m, uint32_t wt, uint32_t vec, int32_t *csrc,
        int32_t *cdst, uint32_t *cw, uint32_t variant, uint32_t spin_limit)
{
    const bool covered = (variant & kVariantCovered) != 0, cas = (variant & kVariantCas) != 0;
    constexpr int kFW = kFT / 32;
    __shared__ TileSmem sm;
    Ctl *c = ws.ctl;
    uint32_t *status = &c->status;
    const uint32_t nb = gridDim.x, bid = blockIdx.x;
    const size_t gtid = (size_t)bid * kFT + threadIdx.x, gstride = (size_t)nb * kFT;
    const uint32_t gw = bid * kFW + (threadIdx.x >> 5), nw = nb * kFW;  // global warp
    uint32_t gen = 0;  // barrier count (the barrier itself keeps no generation)
// Every grid barrier of the solve: when a bounded wait has run out (here or
// in another CTA), the phase just ended may be incomplete, so the CTA stops
// before reading its results; no later index can then leave its buffer.
// The status word keeps ST_TIMEOUT and the count of written ids is 0.
#define MST_SYNC_OR_ABORT()                               \
    do {                                                  \
        if (grid_sync(ws.bar, gen, status, spin_limit)) { \
            if (gtid == 0)                                \
                *out_count = 0;                           \
            return;                                       \
        }                                                 \
    } while (0)
    log_phase(c, PH_START);
    init_range(ws, n, m, gtid, gstride);
    if (cas)  // the CAS hook swaps roots' pointers: every component starts as one
        for (size_t v = gtid; v < n; v += gstride)
            ws.parent[v] = (int32_t)v;
    mark_work(c);
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
    MST_SYNC_OR_ABORT();
    log_phase(c, PH_INIT);
    {
        const bool filtered = use_filter(m, n);
        for_warp_tiles(&c->tick_find0, (m + kFind0WTile - 1) / kFind0WTile, gw, nw,
                       [&](uint32_t t) {
                           find0_wtile(ws, src, dst, w, n, m, wt, vec, status, filtered, t, csrc,
                                       cdst, cw);
                       });
    }
    mark_work(c);
    MST_SYNC_OR_ABORT();
    log_phase(c, PH_FIND0);
    if (csrc) {  // host inputs: the later phases read the device copy
        src = csrc;
        dst = cdst;
        w = cw;
    }
    // m_cur: slots of the current list; m_live: its live edges (equal, except
    // in the "covered" ablation, where the list keeps all m slots)
    uint32_t n_cur = n, m_cur = m, m_live = m, r = 0;
    for (;; r++) {
        // hook + new ids of the roots
        const uint32_t nth = (n_cur + kHookWTile - 1) / kHookWTile;
        if (bid == 0 && threadIdx.x == 0)
            c->flag3[0] = 0;
        if (cas) {
            for (uint32_t t = gw; t < nth; t += nw) {
                if (r == 0)
                    hook_cas_wtile<true>(ws, c, t, r, n_cur, src, dst);
                else
                    hook_cas_wtile<false>(ws, c, t, r, n_cur, src, dst);
            }
        } else if (r == 0) {
            for_warp_tiles(&c->tick_hook[r], nth, gw, nw, [&](uint32_t t) {
                hook_wtile<true>(ws, c, t, r, n_cur, src, dst);
            });
        } else {
            for_warp_tiles(&c->tick_hook[r], nth, gw, nw, [&](uint32_t t) {
                hook_wtile<false>(ws, c, t, r, n_cur, src, dst);
            });
        }
        mark_work(c);
        MST_SYNC_OR_ABORT();
        log_phase(c, PH_HOOK, r);
        if (cas) {
            for (uint32_t t = gw; t < nth; t += nw)
                number_roots_wtile(ws, c, t, r, n_cur);
            mark_work(c);
            MST_SYNC_OR_ABORT();
            log_phase(c, PH_ROOTS, r);
        }
        const uint32_t n_next = ld_volatile_u32(&c->cnt_n[r]);
        // few components left: this round's compaction feeds the tail instead
        const bool tail = n_next >= 2 && n_next <= kTailMaxN && m_cur > 0;
        if (tail) {
            for (size_t i = gtid; i < (size_t)n_next * n_next; i += gstride)
                ws.pair_tab[i] = kNoEdge;
            for (size_t v = gtid; v < n_next; v += gstride) {
                ws.tmin[v] = kNoEdge;
                ws.tpar[v] = (int32_t)v;
            }
        }
        // compress, with extra pointer-jumping passes while chains are deep
        for (uint32_t pass = 0;; pass++) {
            if (bid == 0 && threadIdx.x == 0)
                c->flag3[(pass + 1) % 3] = 0;
            const bool unf = compress_range(ws, n_cur, pass == 0, gtid, gstride);
            if (__syncthreads_or(unf ? 1 : 0) && threadIdx.x == 0)
                c->flag3[pass % 3] = 1u;
            mark_work(c);
            MST_SYNC_OR_ABORT();
            log_phase(c, PH_COMPRESS, r);
            if (!ld_volatile_u32(&c->flag3[pass % 3]))
                break;
            if (pass + 1 >= kMaxJumpPasses) {
                if (gtid == 0)
                    atomicOr(status, ST_INTERNAL);
                break;
            }
        }
        if (tail) {
            const uint32_t ntp = (m_cur + kCompWTile - 1) / kCompWTile;
            for_warp_tiles(&c->tick_comp[r], ntp, gw, nw, [&](uint32_t t) {
                if (r == 0)
                    compact_pairs_wtile<true>(ws, c, t, r, m_cur, n_next, n, wt, src, dst, w,
                                              covered);
                else
                    compact_pairs_wtile<false>(ws, c, t, r, m_cur, n_next, n, wt, src, dst, w,
                                               covered);
            });
            mark_work(c);
            MST_SYNC_OR_ABORT();
            log_phase(c, PH_COMPACT, r);
            extract_pairs(ws, c, n_next, gtid, gstride);
            mark_work(c);
            MST_SYNC_OR_ABORT();
            const uint32_t m_t = ld_volatile_u32(&c->tail_cnt[0]);
            if (gtid == 0 && r + 1 <= (uint32_t)kMaxRounds) {
                c->stat_m[r + 1] = m_t;
                c->stat_n[r + 1] = n_next;
            }
            tail_rounds<kFT>(ws, c, n_next, m_t, r + 1, sm, spin_limit);
            mark_work(c);
            MST_SYNC_OR_ABORT();
            log_phase(c, PH_TAIL, r + 1);
            // components left and rounds run, as CTA 0 recorded them
            n_cur = n_next - ld_volatile_u32(&c->tail_added);
            const uint32_t tr = ld_volatile_u32(&c->tail_rounds);
            r = r + tr;  // rounds finished by the tail
            break;
        }
        // compact (+ find-min of the next round)
        if (cas)  // the next round's components start as roots
            for (size_t v = gtid; v < n_next; v += gstride)
                ws.parent[v] = (int32_t)v;
        const uint32_t ntc = (m_cur + kCompWTile - 1) / kCompWTile;
        for_warp_tiles(&c->tick_comp[r], ntc, gw, nw, [&](uint32_t t) {
            if (covered) {
                if (r == 0)
                    compact_wtile<true, true>(ws, c, t, r, m_cur, n_next, n, wt, src, dst, w,
                                              m_live);
                else
                    compact_wtile<false, true>(ws, c, t, r, m_cur, n_next, n, wt, src, dst, w,
                                               m_live);
            } else if (r == 0) {
                compact_wtile<true>(ws, c, t, r, m_cur, n_next, n, wt, src, dst, w);
            } else {
                compact_wtile<false>(ws, c, t, r, m_cur, n_next, n, wt, src, dst, w);
            }
        });
        mark_work(c);
        MST_SYNC_OR_ABORT();
        log_phase(c, PH_COMPACT, r);
        const uint32_t m_next = ld_volatile_u32(&c->cnt_m[r]);
        if (gtid == 0 && r + 1 <= (uint32_t)kMaxRounds) {
            c->stat_m[r + 1] = m_next;
            c->stat_n[r + 1] = n_next;
        }
        n_cur = n_next;
        m_live = m_next;
        m_cur = covered ? m : m_next;
        if (m_live == 0)
            break;
        if (r + 1 >= (uint32_t)kMaxRounds) {
            if (gtid == 0)
                atomicOr(status, ST_INTERNAL);
            break;
        }
    }
    // emit: count per group of 32 words, barrier, write
    const uint32_t words = (m + 31u) >> 5;
    const uint32_t nte = (words + 31u) >> 5;
    const uint32_t cap = n > 0 ? n - 1 : 0;
    emit_count<kFT>(ws, words, nte, sm);
    MST_SYNC_OR_ABORT();
    emit_range<kFT>(ws, c, nte, words, cap, out, sm);
    mark_work(c);
    MST_SYNC_OR_ABORT();
    log_phase(c, PH_EMIT, r);
    if (gtid == 0) {
        finish(c, out_count, nte ? ld_volatile_u32(&c->emitted) : 0u, n, n_cur);
        c->round = r + 1;
        c->n_cur = n_cur;
        c->m_cur = 0;
    }
}

#undef MST_SYNC_OR_ABORT

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

// Takes the next tile index for the calling warp from *ticket.
__device__ __forceinline__ uint32_t next_warp_tile(uint32_t *ticket)
{
    uint32_t t = 0;
    if ((threadIdx.x & 31) == 0)
        t = atomicAdd(ticket, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
}

template <bool R0>
__global__ void __launch_bounds__(kThreads) k_hook(Ws ws)
{
    __shared__ uint32_t s_flag;
    Ctl *c = ws.ctl;
    const uint32_t round = c->round, n_cur = c->n_cur;
    const uint32_t ntiles = (n_cur + kHookWTile - 1) / kHookWTile;
    for (;;) {
        const uint32_t tile = next_warp_tile(&c->ticket);
        if (tile >= ntiles)
            break;
        hook_wtile<R0>(ws, c, tile, round, n_cur, c->src, c->dst);
    }
    if (last_block_done(&c->done, &s_flag) && threadIdx.x == 0) {
        c->n_next = ld_volatile_u32(&c->cnt_n[round]);
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
    __shared__ uint32_t s_flag;
    Ctl *c = ws.ctl;
    const uint32_t round = c->round, m_cur = c->m_cur, n_next = c->n_next;
    const uint32_t ntiles = (m_cur + kCompWTile - 1) / kCompWTile;
    for (;;) {
        const uint32_t tile = next_warp_tile(&c->ticket);
        if (tile >= ntiles)
            break;
        compact_wtile<R0>(ws, c, tile, round, m_cur, n_next, c->n, c->wt, c->src, c->dst,
                          (const uint32_t *)c->w);
    }
    if (last_block_done(&c->done, &s_flag) && threadIdx.x == 0) {
        const uint32_t m_next = ld_volatile_u32(&c->cnt_m[round]);
        c->m_next = m_next;
        const uint32_t r1 = round + 1;
        if (r1 <= (uint32_t)kMaxRounds) {
            c->stat_m[r1] = m_next;
            c->stat_n[r1] = n_next;
        }
        c->m_cur = m_next;
        c->n_cur = n_next;
        c->round = r1;
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
    (void)n_cap;  // only the graph schedule's emit scans with look-back
    const uint32_t words = (m_cap + 31) / 32;
    return (words + kEmitWords - 1) / kEmitWords + 1;
}

static const int kMaxGridBlocks = 152 * 8 * 2;  // bound for the barrier counters

// Groups of 32 tree-bit words counted by the fused emit.
static size_t emit_groups(uint32_t m_cap)
{
    const size_t words = ((size_t)m_cap + 31) / 32;
    return (words + 31) / 32 + 1;
}

// Tail capacities: the pair table covers up to min(kTailMaxN, n) components,
// and no pair list is longer than the edge list (a pair needs an edge).
static size_t tail_n_cap(uint32_t n_cap)
{
    return n_cap < kTailMaxN ? n_cap : kTailMaxN;
}

static size_t tail_pairs_cap(uint32_t n_cap, uint32_t m_cap)
{
    const size_t tn = tail_n_cap(n_cap);
    const size_t pairs = tn * (tn - 1) / 2;
    return pairs < m_cap ? pairs : m_cap;
}

size_t single_bytes(uint32_t n_cap, uint32_t m_cap)
{
    size_t b = align_up(sizeof(Ctl));
    b += align_up(bar_words(kMaxGridBlocks) * 4);
    b += 2 * align_up((size_t)m_cap * sizeof(uint4));
    b += 2 * align_up((size_t)n_cap * 8);
    b += 3 * align_up((size_t)n_cap * 4);
    b += align_up((((size_t)m_cap + 31) / 32) * 4);
    b += align_up((size_t)m_cap * 8);  // endpoints of possible minima, by id
    b += align_up((size_t)desc_capacity(n_cap, m_cap) * 8);
    b += align_up(emit_groups(m_cap) * 4);  // emit group counts
    b += align_up((size_t)kMaxGridBlocks * 4);  // emit totals per CTA
    const size_t tn = tail_n_cap(n_cap), tp = tail_pairs_cap(n_cap, m_cap);
    b += align_up(tn * tn * 8);                  // pair table
    b += 2 * align_up(tp * 16);                  // tail lists
    b += align_up((size_t)kTailMaxN * 8) + 2 * align_up((size_t)kTailMaxN * 4);
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
    const int schedule = s.schedule, bps = s.fused_blocks_per_sm, ft = s.fused_threads;
    const uint32_t wait_limit = s.wait_limit;
    s = Single();
    s.schedule = schedule;
    s.fused_blocks_per_sm = bps;
    s.fused_threads = ft;
    s.wait_limit = wait_limit;
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

static int occupancy(const void *func, size_t smem, int threads = kThreads)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, func, threads, smem) != cudaSuccess ||
        blocks < 1)
        blocks = 1;
    return blocks;
}

// Edge count above which the automatic shape (schedule 0) takes 1024-thread
// CTAs instead of 256-thread ones, one CTA per SM either way.  Measured on
// GB300 (random graphs of 4K..4.5M edges, the grid and R-MAT workloads):
// below ~0.6M edges one 256-thread CTA per SM is 12-20% faster than four
// (fewer arrivals at each barrier, enough parallelism for the work); above,
// one 1024-thread CTA per SM is fastest (R-MAT 22: 1.71 ms against 1.77 ms).
constexpr uint32_t kAutoWideM = 600000;

// The fused kernel for a CTA size (256, 512, 768 or 1024 threads).
static const void *fused_kernel(int threads)
{
    switch (threads) {
    case 256: return (const void *)k_solve<256>;
    case 512: return (const void *)k_solve<512>;
    case 768: return (const void *)k_solve<768>;
    default: return (const void *)k_solve<1024>;
    }
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
    s.ws.eends = (uint2 *)take((size_t)m_cap * 8);
    s.ws.desc_cap = desc_capacity(n_cap, m_cap);
    s.ws.desc = (unsigned long long *)take((size_t)s.ws.desc_cap * 8);
    s.ws.emit_cnt = (uint32_t *)take(emit_groups(m_cap) * 4);
    s.ws.emit_cta = (uint32_t *)take((size_t)kMaxGridBlocks * 4);
    const size_t tn = tail_n_cap(n_cap), tp = tail_pairs_cap(n_cap, m_cap);
    s.ws.pair_tab = (unsigned long long *)take(tn * tn * 8);
    s.ws.tl[0] = (uint4 *)take(tp * 16);
    s.ws.tl[1] = (uint4 *)take(tp * 16);
    s.ws.tmin = (unsigned long long *)take((size_t)kTailMaxN * 8);
    s.ws.tpar = (int32_t *)take((size_t)kTailMaxN * 4);
    s.ws.tnid = (int32_t *)take((size_t)kTailMaxN * 4);
    s.ws.n_cap = n_cap;
    s.ws.m_cap = m_cap;
    MST_TRY(cudaMemset(s.ws.ctl, 0, sizeof(Ctl)));
    MST_TRY(cudaMemset(s.ws.bar, 0, bar_words(kMaxGridBlocks) * 4));
    MST_TRY(cudaMemset(s.ws.desc, 0, (size_t)s.ws.desc_cap * 8));
    int sms = 0;
    MST_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    s.sms = sms;
    int occ_t = occupancy((const void *)k_compact<false>, 0);
    int occ_h = occupancy((const void *)k_hook<false>, 0);
    int occ = occ_t < occ_h ? occ_t : occ_h;
    occ = occ > 4 ? 4 : occ;
    s.grid_tiles = sms * occ;
    s.grid_stream = sms * 4;
    int occ_f = occupancy(fused_kernel(s.fused_threads), 0, s.fused_threads);
    occ_f = occ_f > s.fused_blocks_per_sm ? s.fused_blocks_per_sm : occ_f;
    s.grid_fused = sms * occ_f;
    if (s.grid_fused > kMaxGridBlocks)
        s.grid_fused = kMaxGridBlocks;
    s.solves = 0;
    return cudaSuccess;  // the graph schedule's CUDA graph is built on first use
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

// Fused solves on one device are ordered among themselves.  A fused grid
// waits on itself at grid barriers, so all its CTAs must be resident at
// once; two fused grids launched at the same time (other streams, other
// handles, the server's lane) could each be left partly resident and wait
// until their barriers give up.  So every fused launch on a device first
// waits (on its own stream) for the previous fused launch on that device
// to finish, through one event per device recorded after each launch.  The
// chain holds across handles and streams of the process; other kernels
// (batched solves, copies) still run beside a fused solve.  A stream that
// is being captured into a CUDA graph is left out of the chain: the caller
// orders what it replays.
struct FusedChain {
    std::mutex mu;
    cudaEvent_t last = nullptr;
};
static FusedChain g_fused_chain[64];

template <typename F>
static cudaError_t ordered_fused_launch(cudaStream_t stream, F &&launch)
{
    int dev = 0;
    MST_TRY(cudaGetDevice(&dev));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MST_TRY(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusNone || dev < 0 || dev >= 64)
        return launch();
    FusedChain &ch = g_fused_chain[dev];
    std::lock_guard<std::mutex> lk(ch.mu);
    if (!ch.last)
        MST_TRY(cudaEventCreateWithFlags(&ch.last, cudaEventDisableTiming));
    else
        MST_TRY(cudaStreamWaitEvent(stream, ch.last, 0));
    MST_TRY(launch());
    return cudaEventRecord(ch.last, stream);
}

cudaError_t single_launch(Single &s, const int32_t *src, const int32_t *dst, const void *w,
                          uint32_t wt, int32_t *out, int64_t *out_count, uint32_t n, uint32_t m,
                          cudaStream_t stream, int grid, const InputCopy *copy)
{
    // the fused kernel runs on any grid up to the co-resident one
    int g = grid > 0 && grid < s.grid_fused ? grid : s.grid_fused;
    int threads = s.fused_threads;
    const uint32_t variant =
        s.schedule == 3 ? kVariantCovered : s.schedule == 4 ? kVariantCas : 0u;
    if (s.schedule == 0 || s.schedule >= 3) {  // shape per solve: one CTA per SM, wider for large graphs
        threads = m > kAutoWideM ? 1024 : 256;
        g = s.sms;
    }
    MST_TRY(begin_solve(s, stream));
    const uint32_t vec = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)w) & 15u) == 0 ? 1u : 0u;
    if (s.schedule != 2) {
        const uint32_t *wp = (const uint32_t *)w;
        int32_t *csrc = copy ? copy->src : nullptr, *cdst = copy ? copy->dst : nullptr;
        uint32_t *cw = copy ? (uint32_t *)copy->w : nullptr;
        void *args[] = {(void *)&s.ws, (void *)&src, (void *)&dst, (void *)&wp, (void *)&out,
                        (void *)&out_count, (void *)&n, (void *)&m, (void *)&wt, (void *)&vec,
                        (void *)&csrc, (void *)&cdst, (void *)&cw, (void *)&variant,
                        (void *)&s.wait_limit};
        return ordered_fused_launch(stream, [&] {
            return cudaLaunchCooperativeKernel(fused_kernel(threads), dim3(g), dim3(threads),
                                               args, 0, stream);
        });
    }
    if (!s.exec)
        MST_TRY(build_graph(s));
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

// Per-phase times of the last fused solve, from its phase log (measured
// inside the timed kernel: %globaltimer at each grid barrier), with the
// algorithmic bytes of each phase kind from the per-round sizes.
cudaError_t single_phase_profile(Single &s, cudaStream_t stream, std::vector<KernelProfile> &prof)
{
    prof.clear();
    MST_TRY(cudaStreamSynchronize(stream));
    Ctl c;
    MST_TRY(cudaMemcpy(&c, s.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    static const char *names[] = {"start", "init", "find0", "hook",
                                  "compress", "compact", "emit", "tail", "roots"};
    const double n = c.n, m = c.m;
    auto bytes_of = [&](int kind, uint32_t r) -> double {
        switch (kind) {
        case PH_INIT: return 8.0 * n + m / 8.0;
        case PH_FIND0: return 12.0 * m;
        case PH_HOOK: return 20.0 * c.stat_n[r] + 4.0 * c.stat_n[r + 1];
        case PH_COMPRESS: return 0.0;  // attributed once per round below
        case PH_COMPACT: return (r == 0 ? 12.0 : 16.0) * c.stat_m[r] + 16.0 * c.stat_m[r + 1];
        case PH_EMIT: return m / 8.0 + 4.0 * (n > 0 ? n - 1 : 0);
        }
        return 0.0;
    };
    const uint32_t np = c.nphase < (uint32_t)kMaxPhaseLog ? c.nphase : (uint32_t)kMaxPhaseLog;
    auto add = [&](const std::string &name, double ms, double bytes) {
        for (auto &k : prof)
            if (k.name == name) {
                k.launches++;
                k.ms += ms;
                k.bytes += bytes;
                return;
            }
        prof.push_back(KernelProfile{name, 1, ms, bytes});
    };
    uint32_t last_compress_round = 0xffffffffu;
    double wait_ms = 0.0;
    int waits = 0;
    for (uint32_t i = 1; i < np; i++) {
        const int k = c.phase_kind[i] <= PH_ROOTS ? c.phase_kind[i] : 0;
        const uint32_t r = c.phase_round[i];
        const double ms = (double)(c.phase_ns[i] - c.phase_ns[i - 1]) * 1e-6;
        double b = bytes_of(k, r < (uint32_t)kMaxRounds ? r : 0);
        if (k == PH_COMPRESS && r != last_compress_round) {
            b = 8.0 * c.stat_n[r] + 4.0 * c.stat_n[r + 1];
            last_compress_round = r;
        }
        std::string name = std::string("k_solve:") + names[k];
        if (k == PH_HOOK || k == PH_COMPRESS || k == PH_COMPACT || k == PH_ROOTS)
            name += r < 3 ? "@r" + std::to_string(r) : std::string("@r3+");
        add(name, ms, b);
        if (c.work_ns[i] > c.phase_ns[i - 1] && c.work_ns[i] <= c.phase_ns[i]) {
            wait_ms += (double)(c.phase_ns[i] - c.work_ns[i]) * 1e-6;
            waits++;
        }
    }
    if (waits)
        prof.push_back(KernelProfile{"(of which CTA 0 waits at barriers)", waits, wait_ms, 0.0});
    return cudaSuccess;
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
