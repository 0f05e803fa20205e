// mst_batched.cu — many independent graphs in one persistent launch.
//
// Each graph runs the same Boruvka rounds as the single-graph path (Section
// 2.1: find-min, hook, compress, compact/"covered" removal, repeat), but all
// rounds of one graph are walked by one team of threads — a whole CTA, or a
// single warp for small graphs — synchronised with __syncthreads/__syncwarp
// instead of kernel boundaries, so a batch costs one launch however many
// rounds its graphs need.
//
//   k_b_prep    validates the offset tables and counts graphs per size bin
//   k_b_order   orders graph ids largest bin first (longest-job-first)
//   k_b_solve   persistent CTAs take big graphs from a queue; when that
//               queue is empty each warp takes small graphs from a second one
//
// Per graph, the vertex arrays (minimum keys, parents, new ids, labels, tree
// bits) and, when they fit, the live edge list are placed in the CTA's (or
// warp's) shared memory; otherwise in its slice of global workspace.  The
// solver is one function over generic pointers, so both placements run the
// same code.  Compaction is in place: tiles are read before any survivor of
// the tile is written, and survivors move only to lower positions.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "mst_internal.h"

namespace mst {

struct BCtl {
    uint32_t status;
    uint32_t big_queue;
    uint32_t small_queue;
    uint32_t pad;
    uint32_t bin_count[64];
    uint32_t bin_cursor[64];
};

struct BWs {
    BCtl *ctl;
    uint4 *E;                   // total_m live edge records
    unsigned long long *mins;   // 2 * total_n
    int32_t *parent, *nid, *lab;
    uint32_t *bits;             // total_m/32 + G + 1 words
    int32_t *order;             // G
    uint32_t *gstat;            // G: status bits of each graph's own solve
    uint64_t total_n, total_m;
};

struct BJob {
    const int64_t *vtx_off, *edge_off;
    const int32_t *src, *dst;
    const uint32_t *w;
    int32_t *out;
    int64_t *out_counts;
    uint32_t wt;
    int32_t G;
    uint32_t warp_max_m;  // graphs with m <= this go to warps; 0 = no warp mode
    uint32_t smem_bytes;  // dynamic shared memory per CTA
    const GraphDesc *descs;  // when set, graphs come from this list instead
};

// One graph of a batch: its inputs, outputs and workspace slice.
struct GraphView {
    const int32_t *src, *dst;
    const uint32_t *w;
    int32_t *out;
    int64_t *out_count;
    uint32_t n, m, wt;
    uint64_t vo, eo;  // workspace offsets
    bool bad;
};

__device__ __forceinline__ GraphView graph_at(const BJob &job, int g)
{
    GraphView v;
    if (job.descs) {
        const GraphDesc d = job.descs[g];
        v.src = d.src;
        v.dst = d.dst;
        v.w = (const uint32_t *)d.w;
        v.out = d.out;
        v.out_count = d.out_count;
        v.n = d.n;
        v.m = d.m;
        v.wt = d.wt;
        v.vo = d.ws_vo;
        v.eo = d.ws_eo;
        v.bad = false;
        return v;
    }
    const int64_t v0 = job.vtx_off[g], v1 = job.vtx_off[g + 1];
    const int64_t e0 = job.edge_off[g], e1 = job.edge_off[g + 1];
    v.bad = v0 < 0 || e0 < 0 || v1 < v0 || e1 < e0 || v1 - v0 > INT32_MAX || e1 - e0 > INT32_MAX;
    v.n = v.bad ? 0u : (uint32_t)(v1 - v0);
    v.m = v.bad ? 0u : (uint32_t)(e1 - e0);
    v.vo = (uint64_t)v0;
    v.eo = (uint64_t)e0;
    v.src = job.src + e0;
    v.dst = job.dst + e0;
    v.w = job.w + e0;
    v.out = job.out + v0;
    v.out_count = job.out_counts + g;
    v.wt = job.wt;
    return v;
}

// ------------------------------------------------------------- thread teams

// A whole CTA of T threads.
template <int T>
struct BlockTeam {
    static constexpr int kSize = T;
    static constexpr int kW = T / 32;
    static constexpr int kWarps = T / 32;
    uint32_t *scratch;             // 4*kW + 2 words of shared memory
    unsigned long long *ring;      // kRing look-back slots in shared memory
    uint32_t *total;               // one shared word: a phase's total
    __device__ __forceinline__ int warp() const { return threadIdx.x >> 5; }
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool any(bool x) const { return __syncthreads_or(x ? 1 : 0) != 0; }

    // Exclusive scan of the 4*kW per-(row, warp) counts in scratch; total
    // into scratch[4*kW].  Called after a sync, followed by a sync.
    __device__ __forceinline__ void scan_counts() const
    {
        constexpr int K = 4 * kW;
        constexpr int per = (K + 31) / 32;
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            uint32_t loc[per], sum = 0;
#pragma unroll
            for (int i = 0; i < per; i++) {
                const int idx = lane * per + i;
                loc[i] = idx < K ? scratch[idx] : 0u;
                sum += loc[i];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            uint32_t run = incl - sum;
#pragma unroll
            for (int i = 0; i < per; i++) {
                const int idx = lane * per + i;
                if (idx < K)
                    scratch[idx] = run;
                run += loc[i];
            }
            if (lane == 31)
                scratch[K] = incl;
        }
    }

    // Stable ranks of kept items of a striped tile (item j of thread t is
    // tile index j*T + t) and the tile total.
    __device__ __forceinline__ void tile_ranks(const bool (&keep)[4], uint32_t (&rank)[4],
                                               uint32_t &total) const
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t mask[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            mask[j] = __ballot_sync(0xffffffffu, keep[j]);
        __syncthreads();  // previous users of scratch are done
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                scratch[j * kW + warp] = __popc(mask[j]);
        }
        __syncthreads();
        scan_counts();
        __syncthreads();
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int j = 0; j < 4; j++)
            rank[j] = scratch[j * kW + warp] + __popc(mask[j] & lt);
        total = scratch[4 * kW];
    }

    // Exclusive offsets of per-item counts of a striped tile.
    __device__ __forceinline__ void tile_offsets(const uint32_t (&cnt)[4], uint32_t (&off)[4],
                                                 uint32_t &total) const
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t incl[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            incl[j] = cnt[j];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl[j], o);
                if (lane >= o)
                    incl[j] += y;
            }
        }
        __syncthreads();
        if (lane == 31) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                scratch[j * kW + warp] = incl[j];
        }
        __syncthreads();
        scan_counts();
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; j++)
            off[j] = scratch[j * kW + warp] + incl[j] - cnt[j];
        total = scratch[4 * kW];
    }
};

// One warp.
struct WarpTeam {
    static constexpr int kSize = 32;
    static constexpr int kWarps = 1;
    __device__ __forceinline__ int warp() const { return 0; }
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ bool any(bool x) const { return __any_sync(0xffffffffu, x) != 0; }
    __device__ __forceinline__ void tile_ranks(const bool (&keep)[4], uint32_t (&rank)[4],
                                               uint32_t &total) const
    {
        const uint32_t lt = lanemask_lt();
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t mk = __ballot_sync(0xffffffffu, keep[j]);
            rank[j] = run + __popc(mk & lt);
            run += __popc(mk);
        }
        total = run;
    }
    __device__ __forceinline__ void tile_offsets(const uint32_t (&cnt)[4], uint32_t (&off)[4],
                                                 uint32_t &total) const
    {
        const int lane = threadIdx.x & 31;
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint32_t incl = cnt[j];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            off[j] = run + incl - cnt[j];
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        total = run;
    }
};

// ------------------------------------------------------------ graph solver

struct GraphArrays {
    uint4 *E;
    unsigned long long *mA, *mB;
    int32_t *parent, *nid, *lab;
    uint32_t *bits;
    // the pair table of the merging tail (shared memory left over by the
    // graph's own arrays): once a round leaves at most tail_n components,
    // parallel edges are merged (0: never)
    unsigned long long *ptab = nullptr;
    uint32_t tail_n = 0;
    // a team whose vertex arrays start in global memory moves them into
    // this shared memory at the first round whose arrays fit it (0: never)
    char *mig_sm = nullptr;
    size_t mig_budget = 0;
};

// Slot of component pair (a, b), a < b < n, in a triangular table.
__device__ __forceinline__ uint32_t tri_slot(uint32_t a, uint32_t b, uint32_t n)
{
    return a * (2 * n - a - 1) / 2 + (b - a - 1);
}

__host__ __device__ __forceinline__ uint32_t tri_size(uint32_t n) { return n * (n - 1) / 2; }

constexpr uint32_t kBTailMaxN = 128;  // components at which a graph's tail may start

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Bytes of the five per-vertex arrays (two minimum-key arrays, parents, new
// ids, labels) for n vertices.
__host__ __device__ __forceinline__ size_t vert_bytes(uint32_t n)
{
    return 2 * al16((size_t)n * 8) + 3 * al16((size_t)n * 4);
}

// Lays the per-vertex arrays for up to n vertices out at the start of `sm`,
// the second minimum array last, and gives the merging tail's pair table the
// shared memory from that array on (tail_n = 0 when too little is left).
// The second minimum array is dead whenever the pair table is in use: the
// tail starts after a round's hook, that round's compaction (the only writer
// of the next minima) does not run, and the tail's own minima are in mA.
__device__ __forceinline__ void carve_vertex(GraphArrays &A, char *sm, size_t budget, uint32_t n)
{
    char *p = sm;
    A.mA = (unsigned long long *)p;
    p += al16((size_t)n * 8);
    A.parent = (int32_t *)p;
    p += al16((size_t)n * 4);
    A.nid = (int32_t *)p;
    p += al16((size_t)n * 4);
    A.lab = (int32_t *)p;
    p += al16((size_t)n * 4);
    A.mB = (unsigned long long *)p;
    const size_t left = budget - (size_t)(p - sm);
    uint32_t tn = kBTailMaxN;
    while (tn >= 8 && (size_t)tri_size(tn) * 8 > left)
        tn--;
    A.ptab = tn >= 8 ? (unsigned long long *)p : nullptr;
    A.tail_n = tn >= 8 ? tn : 0u;
}

// Offers a key to a running minimum that may live in shared or global
// memory (generic pointer): a filtered min (values only decrease, so a key
// not below the current value cannot win), as a fire-and-forget reduction
// in global memory and an atomic in shared memory.  In global memory the
// filter reads through L1: an older value only lets a key through, and the
// phases that use the minima read them after the team's barrier (measured:
// the 4,096-graph batch 3% faster than with volatile filter loads).
__device__ __forceinline__ void offer_any(unsigned long long *p, unsigned long long key)
{
    if (__isGlobal(p)) {
        if (key < __ldca(p))
            red_min_u64(p, key);  // fire-and-forget in L2
    } else if (key < *(volatile unsigned long long *)p) {
        atomicMin(p, key);
    }
}

// Pointer chase with path halving through a volatile view (the array may
// live in shared or global memory; one team owns it).
__device__ __forceinline__ bool chase_v(volatile int32_t *parent, uint32_t start, uint32_t &at)
{
    uint32_t x = start;
#pragma unroll 1
    for (int s = 0; s < kChaseLimit; s++) {
        const uint32_t p = (uint32_t)parent[x];
        if (p == x) {
            at = x;
            return true;
        }
        const uint32_t gp = (uint32_t)parent[p];
        if (gp == p) {
            at = p;
            return true;
        }
        parent[x] = (int32_t)gp;
        x = gp;
    }
    at = x;
    return false;
}

// ---------------------------------------------------- warp tiles in a team
//
// Inside a CTA team each warp owns tiles w, w + W, w + 2W, ... of a phase
// and takes its output offset from a decoupled look-back over a ring of
// kRing descriptors in shared memory (tagged with the tile number).  Tiles
// cannot run more than about W ahead of the slowest unfinished one (each
// waits on its predecessors' aggregates, and a warp's previous tile is W
// back), and the nearest inclusive prefix is at most W back, so a ring of
// 4W slots is never overwritten while still needed.  A one-warp team needs
// no look-back: it keeps a running offset.
constexpr uint32_t kRing = 128;
constexpr int kTeamHookIpl = 4, kTeamCompIpl = 8;

__device__ __forceinline__ unsigned long long ring_word(uint32_t tile, uint32_t flag, uint32_t v)
{
    return ((unsigned long long)(tile + 1) << 32) | ((unsigned long long)flag << 30) |
           (v & 0x3fffffffu);
}

__device__ __forceinline__ uint32_t lookback_ring(unsigned long long *ring, uint32_t tile,
                                                  uint32_t aggregate, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    volatile unsigned long long *rv = ring;
    if (tile == 0) {
        if (lane == 0)
            rv[0] = ring_word(0, 2u, aggregate);
        __syncwarp();
        return 0;
    }
    if (lane == 0)
        rv[tile % kRing] = ring_word(tile, 1u, aggregate);
    uint32_t excl = 0;
    uint32_t spins = 0;
    for (;;) {
        const int64_t idx = (int64_t)tile - 1 - lane;
        uint32_t flag = 2u, val = 0u;
        if (idx >= 0) {
            const unsigned long long d = rv[(uint32_t)idx % kRing];
            const bool mine = (uint32_t)(d >> 32) == (uint32_t)idx + 1u;
            flag = mine ? (uint32_t)((d >> 30) & 3u) : 0u;
            val = (uint32_t)(d & 0x3fffffffu);
        }
        const uint32_t pmask = __ballot_sync(0xffffffffu, flag == 2u);
        const uint32_t zmask = __ballot_sync(0xffffffffu, flag == 0u);
        const uint32_t stop = pmask ? (uint32_t)(__ffs(pmask) - 1) : 32u;
        const uint32_t need = stop == 32u ? 0xffffffffu : ((2u << stop) - 1u);
        if (stop == 32u || (zmask & need)) {  // wait (a prefix is always within 32 back)
            if (++spins > kSpinLimit) {
                if (lane == 0)
                    atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(20);
            continue;
        }
        uint32_t part = ((uint32_t)lane <= stop) ? val : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            part += __shfl_xor_sync(0xffffffffu, part, o);
        excl = part;
        break;
    }
    if (lane == 0)
        rv[tile % kRing] = ring_word(tile, 2u, excl + aggregate);
    __syncwarp();
    return excl;
}

// A phase's exclusive offset for one warp tile: running offset for a
// one-warp team, ring look-back otherwise.
template <class Team>
__device__ __forceinline__ uint32_t tile_offset(const Team &tm, uint32_t tile, uint32_t total,
                                                uint32_t &run, uint32_t *status);

template <int T>
__device__ __forceinline__ uint32_t tile_offset(const BlockTeam<T> &tm, uint32_t tile,
                                                uint32_t total, uint32_t &run, uint32_t *status)
{
    (void)run;
    return lookback_ring(tm.ring, tile, total, status);
}

template <>
__device__ __forceinline__ uint32_t tile_offset<WarpTeam>(const WarpTeam &, uint32_t, uint32_t total,
                                                          uint32_t &run, uint32_t *)
{
    const uint32_t ex = run;
    run += total;
    return ex;
}

// Empties the look-back ring before a phase that uses it (after the barrier
// that ended the previous phase), then waits for the whole team.
template <int T>
__device__ __forceinline__ void ring_reset(const BlockTeam<T> &tm)
{
    for (uint32_t i = threadIdx.x; i < kRing; i += T)
        ((volatile unsigned long long *)tm.ring)[i] = 0ull;
    __syncthreads();
}
__device__ __forceinline__ void ring_reset(const WarpTeam &) {}

// Stores a phase total (the owner of the last tile) and reads it after the
// team barrier.
template <int T>
__device__ __forceinline__ void put_total(const BlockTeam<T> &tm, uint32_t v) { *(volatile uint32_t *)tm.total = v; }
__device__ __forceinline__ void put_total(const WarpTeam &, uint32_t) {}
template <int T>
__device__ __forceinline__ uint32_t get_total(const BlockTeam<T> &tm, uint32_t) { return *(volatile uint32_t *)tm.total; }
__device__ __forceinline__ uint32_t get_total(const WarpTeam &, uint32_t run) { return run; }


// ------------------------------------------------------- the merging tail
//
// Once a round leaves at most A.tail_n components, a block team stops
// carrying every live edge from round to round.  Of the parallel edges
// between two components only the lightest can be in the tree (a heavier one
// closes a cycle with it), so the round's compaction keeps one record per
// component pair in a triangular table in shared memory, and the remaining
// Boruvka rounds run on those records: hook by edge (a record whose key is
// the minimum of an endpoint hooks that endpoint), roots numbered, records
// relabelled and merged again.  Records carry (a, b, weight bits, input id)
// and keys are (weight, input id), so the order is the same as before.

// Gathers the non-empty slots of the pair table into E (any order: keys
// name their edges); returns their number.  After a team sync.
template <int T>
__device__ __forceinline__ uint32_t pairs_to_list(const BlockTeam<T> &tm, const GraphArrays &A,
                                                  uint32_t n2)
{
    volatile uint32_t *cnt = tm.total;
    if (threadIdx.x == 0)
        *cnt = 0u;
    tm.sync();
    for (uint32_t i = threadIdx.x; i < n2 * n2; i += T) {
        const uint32_t a = i / n2, b = i % n2;
        if (a >= b)
            continue;
        const unsigned long long key = A.ptab[tri_slot(a, b, n2)];
        if (key == kNoEdge)
            continue;
        const uint32_t pos = atomicAdd((uint32_t *)cnt, 1u);
        A.E[pos] = make_uint4(a, b, (uint32_t)(key >> 32), (uint32_t)key);
    }
    tm.sync();
    const uint32_t m2 = *cnt;
    tm.sync();  // every thread has read the count before it is reused
    return m2;
}

// The tail rounds on the m_t records of E among n_t components; returns the
// components left.
template <int T>
__device__ uint32_t merge_tail(const BlockTeam<T> &tm, const GraphArrays &A, uint32_t n_t,
                               uint32_t m_t, uint32_t *status)
{
    volatile uint32_t *cnt = tm.total;
    volatile unsigned long long *tmin = A.mA;
    volatile int32_t *par = A.parent;
    volatile int32_t *nid = A.nid, *lab = A.lab;
    const uint32_t t = threadIdx.x;
    for (uint32_t tr = 0; m_t > 0; tr++) {
        if (tr >= (uint32_t)kMaxRounds) {
            if (t == 0)
                atomicOr(status, ST_INTERNAL);
            break;
        }
        for (uint32_t v = t; v < n_t; v += T) {
            tmin[v] = kNoEdge;
            par[v] = (int32_t)v;
        }
        tm.sync();
        // find-min (Section 2.1, the loop over edges)
        for (uint32_t e = t; e < m_t; e += T) {
            const uint4 q = A.E[e];
            const unsigned long long key = make_key(q.z, q.w);
            offer_any((unsigned long long *)&tmin[q.x], key);
            offer_any((unsigned long long *)&tmin[q.y], key);
        }
        tm.sync();
        // hook by edge (Section 2.1, the union step); a mutual pair keeps the lower id
        for (uint32_t e = t; e < m_t; e += T) {
            const uint4 q = A.E[e];
            const unsigned long long key = make_key(q.z, q.w);
            const bool ha = tmin[q.x] == key, hb = tmin[q.y] == key;
            if (ha && hb)
                par[q.x > q.y ? q.x : q.y] = (int32_t)(q.x < q.y ? q.x : q.y);
            else if (ha)
                par[q.x] = (int32_t)q.y;
            else if (hb)
                par[q.y] = (int32_t)q.x;
            if (ha || hb)
                atomicOr(&A.bits[q.w >> 5], 1u << (q.w & 31));
        }
        if (t == 0)
            *cnt = 0u;
        tm.sync();
        for (uint32_t v = t; v < n_t; v += T)  // roots take new ids
            if ((uint32_t)par[v] == v)
                nid[v] = (int32_t)atomicAdd((uint32_t *)cnt, 1u);
        tm.sync();
        const uint32_t n2 = *cnt;
        for (uint32_t v = t; v < n_t; v += T) {  // a forest: depth < n_t
            uint32_t x = v;
            for (uint32_t hop = 0; hop < n_t; hop++) {
                const uint32_t p = (uint32_t)par[x];
                if (p == x)
                    break;
                x = p;
            }
            lab[v] = nid[x];
        }
        for (uint32_t i = t; i < tri_size(n2); i += T)
            A.ptab[i] = kNoEdge;
        tm.sync();
        // merge: relabel, keep the lightest record per pair
        for (uint32_t e = t; e < m_t; e += T) {
            const uint4 q = A.E[e];
            const uint32_t a = (uint32_t)lab[q.x], b = (uint32_t)lab[q.y];
            if (a == b)
                continue;
            offer_any(&A.ptab[tri_slot(a < b ? a : b, a < b ? b : a, n2)], make_key(q.z, q.w));
        }
        tm.sync();
        m_t = pairs_to_list(tm, A, n2);
        n_t = n2;
    }
    return n_t;
}

// Entry into the merging tail from round r, after its compress: when the
// round leaves 2..A.tail_n components, its compaction keeps the lightest
// record per component pair instead of every edge, and the tail finishes
// the graph.  Returns false (nothing done) otherwise; a warp team never
// merges (its graphs are small).
template <int T>
__device__ bool merge_entry(const BlockTeam<T> &tm, const GraphArrays &A, uint32_t r, uint32_t n,
                            uint32_t m_r, uint32_t n_next, const int32_t *src, const int32_t *dst,
                            const uint32_t *w, uint32_t wt, uint32_t *status, uint32_t *n_left)
{
    if (!A.ptab || n_next < 2 || n_next > A.tail_n || m_r == 0)
        return false;
    for (uint32_t i = threadIdx.x; i < tri_size(n_next); i += T)
        A.ptab[i] = kNoEdge;
    tm.sync();
    for (uint32_t i = threadIdx.x; i < m_r; i += T) {
        uint32_t u, v, wb, id;
        if (r == 0) {
            u = (uint32_t)__ldg(src + i);
            v = (uint32_t)__ldg(dst + i);
            if (u >= n || v >= n || u == v)
                continue;
            wb = weight_bits(__ldg(w + i), wt, status);
            id = i;
        } else {
            const uint4 q = A.E[i];
            u = q.x;
            v = q.y;
            wb = q.z;
            id = q.w;
        }
        const uint32_t a = (uint32_t)((volatile int32_t *)A.lab)[u];
        const uint32_t b = (uint32_t)((volatile int32_t *)A.lab)[v];
        if (a >= n_next || b >= n_next) {
            atomicOr(status, ST_INTERNAL);
            continue;
        }
        if (a != b)
            offer_any(&A.ptab[tri_slot(a < b ? a : b, a < b ? b : a, n_next)], make_key(wb, id));
    }
    tm.sync();
    const uint32_t m_t = pairs_to_list(tm, A, n_next);
    *n_left = merge_tail(tm, A, n_next, m_t, status);
    return true;
}

__device__ __forceinline__ bool merge_entry(const WarpTeam &, const GraphArrays &, uint32_t,
                                            uint32_t, uint32_t, uint32_t, const int32_t *,
                                            const int32_t *, const uint32_t *, uint32_t,
                                            uint32_t *, uint32_t *)
{
    return false;
}

// All Boruvka rounds of one graph by one team.  Inputs are the graph's slice
// of the caller's arrays (local ids); A the graph's working arrays.
template <class Team>
__device__ void solve_graph(const Team &tm, uint32_t n, uint32_t m, const int32_t *src,
                            const int32_t *dst, const uint32_t *w, uint32_t wt,
                            GraphArrays A, int32_t *out, int64_t *out_count,
                            uint32_t *status)
{
    constexpr int T = Team::kSize;
    constexpr int TILE = 4 * T;
    const int t = tm.rank();
    const uint32_t words = (m + 31u) >> 5;
    for (uint32_t v = t; v < n; v += T)
        A.mA[v] = kNoEdge;
    for (uint32_t i = t; i < words; i += T)
        A.bits[i] = 0u;
    tm.sync();
    // round-0 find-min (Section 2.1, the loop over edges), four edges a
    // thread per step so that their loads overlap
    for (uint32_t e0 = t; e0 < m; e0 += 4 * T) {
        uint32_t us[4], vs[4], xs[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t e = e0 + j * T;
            const bool in = e < m;
            us[j] = in ? (uint32_t)__ldg(src + e) : 0u;
            vs[j] = in ? (uint32_t)__ldg(dst + e) : 0u;
            xs[j] = in ? __ldg(w + e) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t e = e0 + j * T;
            if (e >= m)
                continue;
            const uint32_t u = us[j], v = vs[j];
            if (u >= n || v >= n) {
                atomicOr(status, ST_BAD_VERTEX);
                continue;
            }
            if (u == v)
                continue;
            const unsigned long long key = make_key(weight_bits(xs[j], wt, status), e);
            offer_any(&A.mA[u], key);
            offer_any(&A.mA[v], key);
        }
    }
    tm.sync();
    uint32_t n_r = n, m_r = m;
    unsigned long long *mc = A.mA, *mx = A.mB;
    for (uint32_t r = 0;; r++) {
        // hook (Section 2.1, the union step) and dense renumbering of roots, warp tiles
        const int lane = threadIdx.x & 31;
        const uint32_t lt = lanemask_lt();
        uint32_t run = 0;
        ring_reset(tm);
        {
            constexpr uint32_t WT = 32 * kTeamHookIpl;
            const uint32_t ntiles = (n_r + WT - 1) / WT;
            for (uint32_t tile = tm.warp(); tile < ntiles; tile += Team::kWarps) {
                const uint32_t base = tile * WT;
                unsigned long long k[kTeamHookIpl];
#pragma unroll
                for (int j = 0; j < kTeamHookIpl; j++) {
                    const uint32_t v = base + j * 32 + lane;
                    k[j] = v < n_r ? mc[v] : kNoEdge;
                }
                uint32_t dd[kTeamHookIpl], id[kTeamHookIpl];
#pragma unroll
                for (int j = 0; j < kTeamHookIpl; j++) {
                    const uint32_t v = base + j * 32 + lane;
                    if (v < n_r)
                        mx[v] = kNoEdge;
                    dd[j] = id[j] = 0;
                    if (k[j] != kNoEdge) {
                        const uint32_t p = (uint32_t)k[j];
                        uint32_t a, b;
                        if (r == 0) {
                            a = (uint32_t)__ldg(src + p);
                            b = (uint32_t)__ldg(dst + p);
                            id[j] = p;
                        } else {
                            const uint4 q = A.E[p];
                            a = q.x;
                            b = q.y;
                            id[j] = q.w;
                        }
                        dd[j] = (a == v) ? b : a;
                    }
                }
                uint32_t mask[kTeamHookIpl], total = 0;
#pragma unroll
                for (int j = 0; j < kTeamHookIpl; j++) {
                    const uint32_t v = base + j * 32 + lane;
                    bool root = false;
                    if (v < n_r) {
                        const uint32_t d = dd[j];
                        const unsigned long long kd = k[j] != kNoEdge ? mc[d] : kNoEdge;
                        if (k[j] == kNoEdge || ((uint32_t)kd == (uint32_t)k[j] && v < d)) {
                            root = true;
                            A.parent[v] = (int32_t)v;
                        } else {
                            A.parent[v] = (int32_t)d;
                            atomicOr(&A.bits[id[j] >> 5], 1u << (id[j] & 31));
                        }
                    }
                    mask[j] = __ballot_sync(0xffffffffu, root);
                    total += __popc(mask[j]);
                }
                const uint32_t ex = tile_offset(tm, tile, total, run, status);
                if (lane == 0 && tile == ntiles - 1)
                    put_total(tm, ex + total);
                uint32_t pos = ex;
#pragma unroll
                for (int j = 0; j < kTeamHookIpl; j++) {
                    if ((mask[j] >> lane) & 1u)
                        A.nid[base + j * 32 + lane] = (int32_t)(pos + __popc(mask[j] & lt));
                    pos += __popc(mask[j]);
                }
            }
            if (ntiles == 0)
                put_total(tm, 0u);
        }
        tm.sync();
        run = get_total(tm, run);
        const uint32_t n_next = run;
        tm.sync();
        // Vertex arrays in global memory move into shared memory as soon as
        // the next round's fit: this round's compaction already offers into
        // the shared minima (cleared here; the compress loop's barrier
        // orders the clearing before them), and the next round runs on the
        // new arrays.  This round's own arrays stay where they are.
        const bool mig = A.mig_sm && n_next > 1 && vert_bytes(n_next) <= A.mig_budget;
        if (mig) {
            mx = (unsigned long long *)A.mig_sm;  // the new layout's first array
            for (uint32_t v = t; v < n_next; v += T)
                mx[v] = kNoEdge;
        }
        // compress: every component takes its root's new id
        for (uint32_t pass = 0;; pass++) {
            bool unfinished = false;
            for (uint32_t v = t; v < n_r; v += T) {
                uint32_t start = v;
                if (pass > 0) {
                    if (((volatile int32_t *)A.lab)[v] != -1)
                        continue;
                    start = (uint32_t)((volatile int32_t *)A.parent)[v];
                }
                uint32_t at;
                if (chase_v(A.parent, start, at)) {
                    A.lab[v] = A.nid[at];
                } else {
                    A.lab[v] = -1;
                    ((volatile int32_t *)A.parent)[v] = (int32_t)at;
                    unfinished = true;
                }
            }
            if (!tm.any(unfinished))
                break;
            if (pass + 1 >= kMaxJumpPasses) {
                atomicOr(status, ST_INTERNAL);
                break;
            }
        }
        tm.sync();
        {
            uint32_t n_left = 0;
            if (merge_entry(tm, A, r, n, m_r, n_next, src, dst, w, wt, status, &n_left)) {
                n_r = n_left;  // the tail finished the graph
                break;
            }
        }
        // compact in place + find-min of the next round, warp tiles: a tile's
        // survivors move only to positions of tiles whose loads are done
        // (their aggregates were published after their loads)
        run = 0;
        ring_reset(tm);
        {
            constexpr uint32_t WT = 32 * kTeamCompIpl;
            const uint32_t ntiles = (m_r + WT - 1) / WT;
            const bool filt = 2ull * m_r >= 8ull * (unsigned long long)(n_next ? n_next : 1);
            for (uint32_t tile = tm.warp(); tile < ntiles; tile += Team::kWarps) {
                const uint32_t base = tile * WT;
                uint4 rec[kTeamCompIpl];
                bool ok[kTeamCompIpl];
#pragma unroll
                for (int j = 0; j < kTeamCompIpl; j++) {
                    const uint32_t i = base + j * 32 + lane;
                    const bool in = i < m_r;
                    if (r == 0) {
                        const uint32_t u = in ? (uint32_t)__ldg(src + i) : 0u;
                        const uint32_t v = in ? (uint32_t)__ldg(dst + i) : 0u;
                        const uint32_t x = in ? __ldg(w + i) : 0u;
                        ok[j] = in && u < n && v < n && u != v;
                        rec[j] = make_uint4(u, v, x, i);
                    } else {
                        rec[j] = in ? A.E[i] : make_uint4(0, 0, 0, 0);
                        ok[j] = in;
                    }
                }
                uint32_t mask[kTeamCompIpl], total = 0;
#pragma unroll
                for (int j = 0; j < kTeamCompIpl; j++) {
                    bool keep = false;
                    if (ok[j]) {
                        const uint32_t nu = (uint32_t)A.lab[rec[j].x], nv = (uint32_t)A.lab[rec[j].y];
                        if (nu >= n_next || nv >= n_next) {
                            atomicOr(status, ST_INTERNAL);
                        } else if (nu != nv) {
                            keep = true;
                            rec[j].x = nu;
                            rec[j].y = nv;
                            if (r == 0)
                                rec[j].z = weight_bits(rec[j].z, wt, status);
                        }
                    }
                    mask[j] = __ballot_sync(0xffffffffu, keep);
                    total += __popc(mask[j]);
                }
                const uint32_t ex = tile_offset(tm, tile, total, run, status);
                if (lane == 0 && tile == ntiles - 1)
                    put_total(tm, ex + total);
                uint32_t pos = ex;
#pragma unroll
                for (int j = 0; j < kTeamCompIpl; j++) {
                    if ((mask[j] >> lane) & 1u) {
                        const uint32_t at = pos + __popc(mask[j] & lt);
                        A.E[at] = rec[j];
                        const unsigned long long key = make_key(rec[j].z, at);
                        if (filt) {
                            offer_any(&mx[rec[j].x], key);
                            offer_any(&mx[rec[j].y], key);
                        } else {
                            atomicMin(&mx[rec[j].x], key);
                            atomicMin(&mx[rec[j].y], key);
                        }
                    }
                    pos += __popc(mask[j]);
                }
            }
            if (ntiles == 0)
                put_total(tm, 0u);
        }
        tm.sync();
        run = get_total(tm, run);
        tm.sync();
        m_r = run;
        n_r = n_next;
        if (mig) {  // once per graph; carve_vertex only sets pointers (the minima
                    // were cleared above)
            carve_vertex(A, A.mig_sm, A.mig_budget, n_r);
            A.mig_sm = nullptr;
            mc = A.mA;
            mx = A.mB;
        } else {
            unsigned long long *tmp = mc;
            mc = mx;
            mx = tmp;
        }
        if (m_r == 0)
            break;
        if (r + 1 >= (uint32_t)kMaxRounds) {
            atomicOr(status, ST_INTERNAL);
            break;
        }
    }
    // emit ascending edge ids
    const uint32_t cap = n > 0 ? n - 1 : 0;
    uint32_t run = 0;
    for (uint32_t base = 0; base < words; base += TILE) {
        uint32_t wv[4], cnt[4], off[4], total;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t i = base + j * T + t;
            wv[j] = i < words ? A.bits[i] : 0u;
            cnt[j] = __popc(wv[j]);
        }
        tm.tile_offsets(cnt, off, total);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint32_t bits = wv[j], pos = run + off[j];
            const uint32_t i = base + j * T + t;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                if (pos < cap)
                    out[pos] = (int32_t)(i * 32u + (uint32_t)b);
                else
                    atomicOr(status, ST_INTERNAL);
                pos++;
            }
        }
        run += total;
    }
    if (t == 0) {
        *out_count = (int64_t)run;
        if (run + n_r != n)
            atomicOr(status, ST_INTERNAL);
        if (n_r > 1)
            atomicOr(status, ST_DISCONNECTED);
    }
    tm.sync();
}

// Shared-memory bytes of a graph's vertex arrays and of its edge list.
__host__ __device__ __forceinline__ size_t vbytes_of(uint32_t n, uint32_t m)
{
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    return 2 * al((size_t)n * 8) + 3 * al((size_t)n * 4) + al((((size_t)m + 31) / 32) * 4);
}

__host__ __device__ __forceinline__ size_t ebytes_of(uint32_t m) { return (size_t)m * 16; }

// Places a graph's arrays in `sm` (shared, `budget` bytes) where they fit.
__device__ __forceinline__ GraphArrays place(const BWs &ws, char *sm, size_t budget, int g,
                                            uint64_t vo, uint64_t eo, uint32_t n, uint32_t m)
{
    GraphArrays A;
    const size_t vb = vbytes_of(n, m), eb = ebytes_of(m);
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    if (vb <= budget) {
        char *p = sm;
        A.mA = (unsigned long long *)p;
        p += al((size_t)n * 8);
        A.mB = (unsigned long long *)p;
        p += al((size_t)n * 8);
        A.parent = (int32_t *)p;
        p += al((size_t)n * 4);
        A.nid = (int32_t *)p;
        p += al((size_t)n * 4);
        A.lab = (int32_t *)p;
        p += al((size_t)n * 4);
        A.bits = (uint32_t *)p;
        p += al((((size_t)m + 31) / 32) * 4);
        A.E = (vb + eb <= budget) ? (uint4 *)p : ws.E + eo;
    } else {
        A.mA = ws.mins + vo;
        A.mB = ws.mins + ws.total_n + vo;
        A.parent = ws.parent + vo;
        A.nid = ws.nid + vo;
        A.lab = ws.lab + vo;
        A.bits = ws.bits + (eo >> 5) + (uint64_t)g;
        A.E = ws.E + eo;
        A.mig_sm = sm;
        A.mig_budget = budget;
    }
    // the merging tail's pair table takes the shared memory left over
    const size_t used = vb > budget ? 0 : (vb + eb <= budget ? vb + eb : vb);
    const size_t left = budget - used;
    uint32_t tn = kBTailMaxN;
    while (tn >= 8 && (size_t)tri_size(tn) * 8 > left)
        tn--;
    if (tn >= 8) {
        A.ptab = (unsigned long long *)(sm + used);
        A.tail_n = tn;
    }
    return A;
}

// ---------------------------------------------------------------- kernels

__global__ void k_b_prep(BWs ws, BJob job, uint64_t total_n, uint64_t total_m)
{
    BCtl *c = ws.ctl;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < job.G; g += gridDim.x * blockDim.x) {
        const GraphView gv = graph_at(job, g);
        bool bad = gv.bad || gv.vo + gv.n > total_n || gv.eo + gv.m > total_m;
        if (!job.descs) {
            if (g == 0 && (gv.vo != 0 || gv.eo != 0))
                bad = true;
            if (g == job.G - 1 && (gv.vo + gv.n != total_n || gv.eo + gv.m != total_m))
                bad = true;
        }
        if (bad)
            atomicOr(&c->status, ST_BAD_OFFSETS);
        ws.gstat[g] = bad ? ST_BAD_OFFSETS : 0u;
        const uint32_t m = bad ? 0u : gv.m;
        const uint32_t bin = m ? 31u - __clz(m) : 0u;
        const bool big = job.warp_max_m == 0 || m > job.warp_max_m;
        atomicAdd(&c->bin_count[bin + (big ? 32 : 0)], 1u);
    }
}

__global__ void k_b_order(BWs ws, BJob job)
{
    __shared__ uint32_t base[64];
    BCtl *c = ws.ctl;
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 63; b >= 0; b--) {  // big bins first, larger bins first
            base[b] = run;
            run += c->bin_count[b];
        }
    }
    __syncthreads();
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < job.G; g += gridDim.x * blockDim.x) {
        const GraphView gv = graph_at(job, g);
        const uint32_t m = gv.bad ? 0u : gv.m;
        const uint32_t bin = m ? 31u - __clz(m) : 0u;
        const bool big = job.warp_max_m == 0 || m > job.warp_max_m;
        const uint32_t b = bin + (big ? 32 : 0);
        if (gv.out_count)
            *gv.out_count = 0;
        if (c->status & ST_BAD_OFFSETS)  // nothing of this batch is solved
            ws.gstat[g] = ST_BAD_OFFSETS;
        ws.order[base[b] + atomicAdd(&c->bin_cursor[b], 1u)] = g;
    }
}

// Records the status bits of graph g's solve (kept in the team's shared
// memory while it runs, so a graph's outcome never reaches its batch-mates)
// and adds them to the batch's combined status word.
__device__ __forceinline__ void publish_status(const BWs &ws, int g, uint32_t bits)
{
    ws.gstat[g] = bits;
    if (bits)
        atomicOr(&ws.ctl->status, bits);
}

template <int T>
__global__ void __launch_bounds__(T) k_b_solve(BWs ws, BJob job)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ uint32_t scratch[4 * (T / 32) + 2];
    __shared__ unsigned long long ring[kRing];
    __shared__ uint32_t s_claim, s_total, s_gstat, s_wstat[T / 32];
    BCtl *c = ws.ctl;
    if (c->status & ST_BAD_OFFSETS)
        return;
    uint32_t n_big = 0;
    for (int b = 32; b < 64; b++)
        n_big += c->bin_count[b];
    BlockTeam<T> team{scratch, ring, &s_total};
    // big graphs: one CTA each, largest first
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_claim = atomicAdd(&c->big_queue, 1u);
        __syncthreads();
        const uint32_t q = s_claim;
        if (q >= n_big)
            break;
        const int g = ws.order[q];
        const GraphView gv = graph_at(job, g);
        const GraphArrays A = place(ws, smem, job.smem_bytes, g, gv.vo, gv.eo, gv.n, gv.m);
        if (threadIdx.x == 0)
            s_gstat = 0u;  // ordered before any use by the solver's first team barrier
        solve_graph(team, gv.n, gv.m, gv.src, gv.dst, gv.w, gv.wt, A, gv.out, gv.out_count,
                    &s_gstat);
        if (threadIdx.x == 0)
            publish_status(ws, g, *(volatile uint32_t *)&s_gstat);
    }
    if (job.warp_max_m == 0)
        return;
    // small graphs: one warp each
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t share = (job.smem_bytes / (T / 32)) & ~(size_t)15;
    char *mine = smem + (size_t)warp * share;
    WarpTeam wt_team;
    const uint32_t G = (uint32_t)job.G;
    for (;;) {
        uint32_t q = 0;
        if (lane == 0)
            q = atomicAdd(&c->small_queue, 1u);
        q = __shfl_sync(0xffffffffu, q, 0) + n_big;
        if (q >= G)
            break;
        const int g = ws.order[q];
        const GraphView gv = graph_at(job, g);
        const GraphArrays A = place(ws, mine, share, g, gv.vo, gv.eo, gv.n, gv.m);
        if (lane == 0)
            s_wstat[warp] = 0u;
        __syncwarp();
        solve_graph(wt_team, gv.n, gv.m, gv.src, gv.dst, gv.w, gv.wt, A, gv.out, gv.out_count,
                    &s_wstat[warp]);
        if (lane == 0)
            publish_status(ws, g, *(volatile uint32_t *)&s_wstat[warp]);
    }
}

// ------------------------------------------------------------------- host

#define MST_TRY(x)                     \
    do {                               \
        cudaError_t e_ = (x);          \
        if (e_ != cudaSuccess)         \
            return e_;                 \
    } while (0)

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t batched_bytes(int32_t G, uint64_t n, uint64_t m)
{
    size_t b = al256(sizeof(BCtl));
    b += al256(m * 16);
    b += al256(n * 16);
    b += 3 * al256(n * 4);
    b += al256((m / 32 + (uint64_t)G + 1) * 4);
    b += 2 * al256((size_t)G * 4);  // order, per-graph status
    return b;
}

void batched_release(Batched &b)
{
    if (b.base)
        cudaFree(b.base);
    std::map<int, BatchedConfig> tuned;
    tuned.swap(b.tuned);
    const int schedule = b.schedule, threads = b.block_threads;
    const bool loaded = b.tuned_loaded;
    b = Batched();
    b.tuned.swap(tuned);
    b.schedule = schedule;
    b.block_threads = threads;
    b.tuned_loaded = loaded;
}

cudaError_t batched_reserve(Batched &b, int32_t G, uint64_t n, uint64_t m)
{
    if (b.base && G <= b.g_cap && n <= b.n_cap && m <= b.m_cap)
        return cudaSuccess;
    const int32_t gc = std::max(G, b.g_cap);
    const uint64_t nc = std::max(n, b.n_cap), mc = std::max(m, b.m_cap);
    if (b.base)
        cudaFree(b.base);
    b.base = nullptr;
    b.bytes = batched_bytes(gc, nc, mc);
    MST_TRY(cudaMalloc(&b.base, b.bytes));
    b.g_cap = gc;
    b.n_cap = nc;
    b.m_cap = mc;
    return cudaSuccess;
}

static BWs carve_at(void *base, int32_t g_cap, uint64_t n_cap, uint64_t m_cap, uint64_t total_n,
                    uint64_t total_m)
{
    BWs ws;
    char *p = (char *)base;
    auto take = [&](size_t sz) {
        char *q = p;
        p += al256(sz);
        return (void *)q;
    };
    ws.ctl = (BCtl *)take(sizeof(BCtl));
    ws.E = (uint4 *)take(m_cap * 16);
    ws.mins = (unsigned long long *)take(n_cap * 16);
    ws.parent = (int32_t *)take(n_cap * 4);
    ws.nid = (int32_t *)take(n_cap * 4);
    ws.lab = (int32_t *)take(n_cap * 4);
    ws.bits = (uint32_t *)take((m_cap / 32 + (uint64_t)g_cap + 1) * 4);
    ws.order = (int32_t *)take((size_t)g_cap * 4);
    ws.gstat = (uint32_t *)take((size_t)g_cap * 4);
    ws.total_n = total_n;
    ws.total_m = total_m;
    return ws;
}

static BWs carve(Batched &b, uint64_t total_n, uint64_t total_m)
{
    BWs ws;
    char *p = (char *)b.base;
    auto take = [&](size_t sz) {
        char *q = p;
        p += al256(sz);
        return (void *)q;
    };
    ws.ctl = (BCtl *)take(sizeof(BCtl));
    ws.E = (uint4 *)take(b.m_cap * 16);
    ws.mins = (unsigned long long *)take(b.n_cap * 16);
    ws.parent = (int32_t *)take(b.n_cap * 4);
    ws.nid = (int32_t *)take(b.n_cap * 4);
    ws.lab = (int32_t *)take(b.n_cap * 4);
    ws.bits = (uint32_t *)take((b.m_cap / 32 + (uint64_t)b.g_cap + 1) * 4);
    ws.order = (int32_t *)take((size_t)b.g_cap * 4);
    ws.gstat = (uint32_t *)take((size_t)b.g_cap * 4);
    ws.total_n = total_n;  // mins B half starts after the batch's vertices
    ws.total_m = total_m;
    return ws;
}

struct Choice {
    int threads;
    int blocks_per_sm;
    uint32_t warp_max_m;
};

static uint32_t smem_for(int device, int bps, size_t static_bytes);

// The persistent grid: min(blocks_per_sm, what registers and threads allow)
// CTAs per SM, each with 1/blocks_per_sm of the SM's shared memory.  The
// share stays 1/blocks_per_sm even where registers let fewer CTAs run: the
// rest of the SM's 256 KB of on-chip memory is then L1 cache, which the
// random gathers and minimum filters of graphs held in global memory need
// (one 1024-thread CTA per SM with all of it as shared memory, leaving about
// 26 KB of L1, ran the 4,096-graph batch at 16.2 ms against 8.2 ms with half).
template <int T>
static cudaError_t launch_solve(const BWs &ws, BJob job, int device, int blocks_per_sm,
                                cudaStream_t s)
{
    int sms = 0;
    MST_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    int fit = 0;
    MST_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_b_solve<T>, T, 0));
    if (fit < 1)
        return cudaErrorInvalidConfiguration;
    const int want = std::max(1, std::min(fit, blocks_per_sm));
    cudaFuncAttributes fa;
    MST_TRY(cudaFuncGetAttributes(&fa, k_b_solve<T>));
    job.smem_bytes = smem_for(device, std::max(1, blocks_per_sm), fa.sharedSizeBytes);
    MST_TRY(cudaFuncSetAttribute(k_b_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)job.smem_bytes));
    int occ = 0;
    MST_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_b_solve<T>, T, job.smem_bytes));
    if (occ < 1)
        return cudaErrorInvalidConfiguration;
    const int bps = std::min(occ, want);
    k_b_solve<T><<<sms * bps, T, job.smem_bytes, s>>>(ws, job);
    return cudaGetLastError();
}

// Dynamic shared memory per CTA for `bps` CTAs on one SM: an equal share of
// the SM's shared memory less each CTA's 1 KB system reserve and the
// kernel's static shared memory, within the per-CTA opt-in limit.
static uint32_t smem_for(int device, int bps, size_t static_bytes)
{
    int per_sm = 0, per_block = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t share = (size_t)per_sm / (size_t)bps;
    size_t s = share > 1024 + static_bytes ? share - 1024 - static_bytes : 0;
    s = std::min(s, (size_t)per_block > static_bytes ? (size_t)per_block - static_bytes : 0);
    return (uint32_t)(s & ~(size_t)255);
}

static cudaError_t run_batched(Batched &b, int device, const BWs &ws, BJob job, const Choice &ch,
                               cudaStream_t s)
{
    job.warp_max_m = ch.warp_max_m;
    b.last_G = job.G;
    MST_TRY(cudaMemsetAsync(ws.ctl, 0, sizeof(BCtl), s));
    const int pg = (int)std::min<int64_t>((job.G + 255) / 256, 1024);
    k_b_prep<<<std::max(pg, 1), 256, 0, s>>>(ws, job, ws.total_n, ws.total_m);
    MST_TRY(cudaGetLastError());
    k_b_order<<<std::max(pg, 1), 256, 0, s>>>(ws, job);
    MST_TRY(cudaGetLastError());
    switch (ch.threads) {
    case 128: return launch_solve<128>(ws, job, device, ch.blocks_per_sm, s);
    case 256: return launch_solve<256>(ws, job, device, ch.blocks_per_sm, s);
    case 512: return launch_solve<512>(ws, job, device, ch.blocks_per_sm, s);
    default: return launch_solve<1024>(ws, job, device, ch.blocks_per_sm, s);
    }
}

// Size bucket of a batch for the autotune cache: log2 of its mean edges.
static int bucket_of(int32_t G, uint64_t total_m)
{
    const double mean = G > 0 ? (double)total_m / G : 0.0;
    return mean < 1 ? 0 : (int)std::floor(std::log2(mean));
}

static Choice default_choice(int32_t G, uint64_t total_m)
{
    const double mean = G > 0 ? (double)total_m / G : 0.0;
    if (mean < 4096)
        return Choice{256, 4, 512};
    return Choice{1024, 2, 1024};
}

static Choice choice_from_config(const BatchedConfig &c)
{
    Choice ch{c.block_threads, c.blocks_per_sm, (uint32_t)c.warp_max_m};
    return ch;
}

static bool json_load(Batched &b, const char *path)
{
    std::ifstream f(path);
    if (!f)
        return false;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t pos = 0;
    int loaded = 0;
    // entries: {"bucket": B, "threads": T, "blocks_per_sm": K, "warp_max_m": W}
    while ((pos = s.find("\"bucket\"", pos)) != std::string::npos) {
        BatchedConfig c;
        int bucket = 0;
        if (sscanf(s.c_str() + pos, "\"bucket\": %d, \"threads\": %d, \"blocks_per_sm\": %d, "
                                    "\"warp_max_m\": %d",
                   &bucket, &c.block_threads, &c.blocks_per_sm, &c.warp_max_m) == 4) {
            c.schedule = c.warp_max_m > 0 ? 2 : 1;
            b.tuned[bucket] = c;
            loaded++;
        }
        pos += 8;
    }
    return loaded > 0;
}

static void json_store(const Batched &b, const char *path)
{
    FILE *f = fopen(path, "w");
    if (!f)
        return;
    fprintf(f, "{\"mst_batched_autotune\": [\n");
    size_t i = 0;
    for (const auto &kv : b.tuned) {
        fprintf(f, "  {\"bucket\": %d, \"threads\": %d, \"blocks_per_sm\": %d, \"warp_max_m\": %d}%s\n",
                kv.first, kv.second.block_threads, kv.second.blocks_per_sm, kv.second.warp_max_m,
                ++i < b.tuned.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    fclose(f);
}

cudaError_t batched_launch(Batched &b, int device, uint32_t wt, int32_t G, const int64_t *vtx_off,
                           const int64_t *edge_off, uint64_t total_n, uint64_t total_m,
                           const int32_t *src, const int32_t *dst, const void *w, int32_t *out,
                           int64_t *out_counts, cudaStream_t stream)
{
    const BWs ws = carve(b, total_n, total_m);
    BJob job{vtx_off, edge_off, src, dst, (const uint32_t *)w, out, out_counts, wt, G, 0, 0,
             nullptr};
    Choice ch = default_choice(G, total_m);
    auto it = b.tuned.find(bucket_of(G, total_m));
    if (it != b.tuned.end())
        ch = choice_from_config(it->second);
    if (b.schedule == 1)
        ch.warp_max_m = 0;
    else if (b.schedule == 2 && ch.warp_max_m == 0)
        ch.warp_max_m = 512;
    if (b.block_threads)
        ch.threads = b.block_threads;
    return run_batched(b, device, ws, job, ch, stream);
}

size_t desc_batch_bytes(int32_t G, uint64_t total_n, uint64_t total_m)
{
    return batched_bytes(G, total_n, total_m);
}

cudaError_t batched_launch_desc(const Batched &tuning, int device, void *ws_base, int32_t G,
                                const GraphDesc *descs, uint64_t total_n, uint64_t total_m,
                                cudaStream_t stream)
{
    const BWs ws = carve_at(ws_base, G, total_n, total_m, total_n, total_m);
    BJob job{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, G, 0, 0, descs};
    Choice ch = default_choice(G, total_m);
    auto it = tuning.tuned.find(bucket_of(G, total_m));
    if (it != tuning.tuned.end())
        ch = choice_from_config(it->second);
    Batched scratch;  // run_batched only reads its caller's shapes
    scratch.m_cap = total_m;
    return run_batched(scratch, device, ws, job, ch, stream);
}

cudaError_t desc_batch_status(void *ws_base, uint32_t *bits, cudaStream_t stream)
{
    MST_TRY(cudaMemcpyAsync(bits, ws_base, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    return cudaStreamSynchronize(stream);
}

cudaError_t desc_batch_graph_status(void *ws_base, int32_t G, uint64_t total_n, uint64_t total_m,
                                    uint32_t *bits)
{
    const BWs ws = carve_at(ws_base, G, total_n, total_m, total_n, total_m);
    return cudaMemcpy(bits, ws.gstat, (size_t)G * 4, cudaMemcpyDeviceToHost);
}

cudaError_t batched_graph_status(Batched &b, cudaStream_t stream, int32_t G, uint32_t *bits)
{
    if (!b.base || G > b.last_G)
        return cudaErrorInvalidValue;
    const BWs ws = carve(b, 0, 0);
    MST_TRY(cudaStreamSynchronize(stream));
    return cudaMemcpy(bits, ws.gstat, (size_t)G * 4, cudaMemcpyDeviceToHost);
}

uint32_t batched_status_bits(Batched &b, cudaStream_t stream, cudaError_t *err)
{
    *err = cudaSuccess;
    if (!b.base)
        return 0;
    uint32_t bits = 0;
    *err = cudaStreamSynchronize(stream);
    if (*err == cudaSuccess)
        *err = cudaMemcpy(&bits, b.base, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    return bits;
}

constexpr int kTuneRuns = 5;  // timed launches per autotune candidate (median)

cudaError_t batched_autotune(Batched &b, int device, uint32_t wt, int32_t G,
                             const int64_t *vtx_off, const int64_t *edge_off, uint64_t total_n,
                             uint64_t total_m, const int32_t *src, const int32_t *dst,
                             const void *w, int32_t *out, int64_t *out_counts, const char *path,
                             cudaStream_t stream)
{
    const int bucket = bucket_of(G, total_m);
    if (path && !b.tuned_loaded) {
        json_load(b, path);
        b.tuned_loaded = true;
    }
    if (b.tuned.count(bucket))
        return cudaSuccess;
    const BWs ws = carve(b, total_n, total_m);
    BJob job{vtx_off, edge_off, src, dst, (const uint32_t *)w, out, out_counts, wt, G, 0, 0,
             nullptr};
    // CTA size, the SM's shared memory split (1/blocks_per_sm a CTA; what
    // is not shared memory is L1) and the warp-per-graph split size
    const Choice cands[] = {
        {1024, 2, 1024}, {1024, 2, 0},   {1024, 2, 2048}, {1024, 1, 1024},
        {1024, 3, 1024}, {1024, 4, 1024}, {512, 2, 1024}, {512, 2, 0},
        {512, 4, 512},   {256, 4, 512},  {256, 4, 0},    {256, 2, 1024},
    };
    cudaEvent_t e0, e1;
    MST_TRY(cudaEventCreate(&e0));
    MST_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    Choice bestc = default_choice(G, total_m);
    for (const Choice &c : cands) {
        if (run_batched(b, device, ws, job, c, stream) != cudaSuccess) {  // warm-up
            cudaGetLastError();
            continue;
        }
        // the median of kTuneRuns timed launches decides, not one sample
        float runs[kTuneRuns];
        for (int k = 0; k < kTuneRuns; k++) {
            MST_TRY(cudaEventRecord(e0, stream));
            MST_TRY(run_batched(b, device, ws, job, c, stream));
            MST_TRY(cudaEventRecord(e1, stream));
            MST_TRY(cudaEventSynchronize(e1));
            MST_TRY(cudaEventElapsedTime(&runs[k], e0, e1));
        }
        std::sort(runs, runs + kTuneRuns);
        const float ms = runs[kTuneRuns / 2];
        if (ms < best) {
            best = ms;
            bestc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BatchedConfig bc;
    bc.block_threads = bestc.threads;
    bc.blocks_per_sm = bestc.blocks_per_sm;
    bc.warp_max_m = (int)bestc.warp_max_m;
    bc.schedule = bestc.warp_max_m ? 2 : 1;
    b.tuned[bucket] = bc;
    if (path)
        json_store(b, path);
    return cudaSuccess;
}

// ------------------------------------------------- allocation-free solve

// Some callers cannot allocate device memory at solve time: a real-time or
// plugin host whose device memory is handed out once at start-up (the
// allocator may synchronise the device and take unbounded time), or a
// process whose device memory a framework's caching allocator already
// holds.  mst_solve_noalloc serves them: one CTA runs every Boruvka round of one graph (the batched solver's
// per-graph team), with its working arrays in this file-scope device array
// instead of a handle's workspace.  Every GPU that loads the library holds
// the array until the process exits; every call shares it and it keeps the
// last call's contents, so the kernel clears what must start empty, and
// calls that overlap on the GPU (different streams, or different host
// threads) race on it.
constexpr uint32_t kNoAllocMaxN = 65536;
constexpr uint32_t kNoAllocMaxM = 262144;
constexpr size_t kNoAllocEdgeBytes = (size_t)kNoAllocMaxM * 16;
constexpr size_t kNoAllocVtxBytes = 2 * (size_t)kNoAllocMaxN * 8 + 3 * (size_t)kNoAllocMaxN * 4;
constexpr size_t kNoAllocBitsBytes = ((size_t)kNoAllocMaxM / 32 + 1) * 4;
constexpr size_t kNoAllocBytes = 256 + kNoAllocEdgeBytes + kNoAllocVtxBytes + kNoAllocBitsBytes;
static_assert(kNoAllocBytes == 6062340, "the byte count documented in mst.h");
constexpr int kNoAllocThreads = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Lays a graph's working arrays out: in shared memory when they fit (as
// the batched solver does), else in the scratch array.  The first 256
// bytes of the scratch hold the status word.
__device__ __forceinline__ GraphArrays place_noalloc(unsigned char *scratch, char *sm,
                                                     size_t budget, uint32_t n, uint32_t m)
{
    GraphArrays A;
    const size_t vb = vbytes_of(n, m), eb = ebytes_of(m);
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    char *p = (vb <= budget) ? sm : (char *)scratch + 256 + kNoAllocEdgeBytes;
    A.mA = (unsigned long long *)p;
    p += al((size_t)n * 8);
    A.mB = (unsigned long long *)p;
    p += al((size_t)n * 8);
    A.parent = (int32_t *)p;
    p += al((size_t)n * 4);
    A.nid = (int32_t *)p;
    p += al((size_t)n * 4);
    A.lab = (int32_t *)p;
    p += al((size_t)n * 4);
    A.bits = (uint32_t *)p;
    p += al((((size_t)m + 31) / 32) * 4);
    A.E = (vb + eb <= budget) ? (uint4 *)p : (uint4 *)(scratch + 256);
    return A;
}

__global__ void __launch_bounds__(kNoAllocThreads)
k_noalloc(unsigned char *scratch, uint32_t smem_bytes, const int32_t *src, const int32_t *dst,
          const uint32_t *w, uint32_t wt, uint32_t n, uint32_t m, int32_t *out,
          int64_t *out_count, int32_t *out_status)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ uint32_t scratch_words[4 * (kNoAllocThreads / 32) + 2];
    __shared__ unsigned long long ring[kRing];
    __shared__ uint32_t s_total;
    uint32_t *status = (uint32_t *)scratch;
    if (threadIdx.x == 0)
        *status = 0u;  // the previous call's outcome must not leak into this one
    __syncthreads();
    BlockTeam<kNoAllocThreads> team{scratch_words, ring, &s_total};
    const GraphArrays A = place_noalloc(scratch, smem, smem_bytes, n, m);
    solve_graph(team, n, m, src, dst, w, wt, A, out, out_count, status);
    if (threadIdx.x == 0 && out_status)
        *out_status = (int32_t)status_code(*(volatile uint32_t *)status);
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host stand-in).
static std::mutex g_noalloc_mu;
static std::map<int, unsigned char *> g_noalloc_ptr;
static std::map<int, uint32_t> g_noalloc_smem;

static cudaError_t noalloc_setup(int device, unsigned char **ptr, uint32_t *smem)
{
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_ptr.find(device);
    if (it != g_noalloc_ptr.end()) {
        *ptr = it->second;
        *smem = g_noalloc_smem[device];
        return cudaSuccess;
    }
    void *p = nullptr;
    MST_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    int optin = 0;
    MST_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    const uint32_t bytes = (uint32_t)((optin - 2048) & ~255);
    MST_TRY(cudaFuncSetAttribute(k_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    g_noalloc_ptr[device] = (unsigned char *)p;
    g_noalloc_smem[device] = bytes;
    *ptr = (unsigned char *)p;
    *smem = bytes;
    return cudaSuccess;
}

}  // namespace mst

extern "C" mst_status mst_solve_noalloc(mst_weight_type wt, int32_t n, int64_t m,
                                        const int32_t *src, const int32_t *dst, const void *w,
                                        int32_t *out_edge_ids, int64_t *out_count,
                                        int32_t *out_status, void *stream)
{
    using namespace mst;
    if ((wt != MST_W_U32 && wt != MST_W_F32) || n < 0 || m < 0 || !out_count)
        return MST_ERR_INVALID_ARG;
    if (m > 0 && (!src || !dst || !w))
        return MST_ERR_INVALID_ARG;
    if (n > 1 && !out_edge_ids)
        return MST_ERR_INVALID_ARG;
    if (n == 0 && m > 0)
        return MST_ERR_INVALID_ARG;
    if ((uint64_t)n > kNoAllocMaxN || (uint64_t)m > kNoAllocMaxM)
        return MST_ERR_BUDGET;  // beyond the fixed scratch
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess)
        return MST_ERR_CUDA;
    unsigned char *scratch = nullptr;
    uint32_t smem = 0;
    if (noalloc_setup(device, &scratch, &smem) != cudaSuccess) {
        cudaGetLastError();
        return MST_ERR_CUDA;
    }
    k_noalloc<<<1, kNoAllocThreads, smem, (cudaStream_t)stream>>>(
        scratch, smem, src, dst, (const uint32_t *)w, (uint32_t)wt, (uint32_t)n, (uint32_t)m,
        out_edge_ids, out_count, out_status);
    return cudaGetLastError() == cudaSuccess ? MST_OK : MST_ERR_CUDA;
}

namespace mst {

}  // namespace mst
