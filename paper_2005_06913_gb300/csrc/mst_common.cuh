// mst_common.cuh — device-side building blocks shared by the single-graph
// and batched Boruvka solvers: the control block, the workspace layout, the
// edge key, ballot-based tile ranking and the decoupled look-back scan.
//
// Edge key (Section 2.1: the find-min loop compares weights; ties are
// broken by edge id): key = (weight_bits << 32) | tag.  weight_bits is the
// uint32 weight, or for float32 an order-preserving remap of the IEEE bits.
// The single-graph solver tags with the input edge id itself and finds the
// edge's endpoints in an endpoints-by-id array.  The batched solver tags with
// the edge's index in its live list; its compaction is stable, so position
// order equals edge-id order among the edges still alive.  Either way the
// minimum over keys is the minimum over (weight, edge id).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

namespace mst {

constexpr int kThreads = 256;                 // threads per block, streaming kernels
constexpr int kWarps = kThreads / 32;         // 8
constexpr int kTile = 1024;                   // 16-byte slots of a CTA's shared stage
constexpr int kMaxRounds = 64;                // > log2(2^31) + 1: never reached
constexpr uint64_t kNoEdge = ~0ull;           // minimum[] = -1 of Section 2.1
constexpr int kChaseLimit = 64;               // pointer hops per thread per pass
constexpr uint32_t kMaxJumpPasses = 64;       // > log2(2^31): pointer jumping ends sooner
constexpr uint32_t kSpinLimit = 1u << 22;     // iterations of any device wait
constexpr int kMaxPhaseLog = 256;             // phase-log entries kept per fused solve
constexpr uint32_t kTailMaxN = 1024;          // components at which the tail takes over (2048
                                              // measured slower: multi-CTA tail rounds cost
                                              // more than the grid round they save)
constexpr uint32_t kTailMaxPairs = kTailMaxN * (kTailMaxN - 1) / 2;
constexpr uint32_t kTailLocalN = 1024;        // a one-CTA tail keeps arrays in shared memory

// Phase kinds of the fused solve's phase log.
enum : uint8_t { PH_START = 0, PH_INIT, PH_FIND0, PH_HOOK, PH_COMPRESS, PH_COMPACT, PH_EMIT,
                 PH_TAIL, PH_ROOTS };

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device status bits (mapped to mst_status on the host).
enum : uint32_t {
    ST_BAD_VERTEX = 1u,
    ST_NAN = 2u,
    ST_TIMEOUT = 4u,
    ST_INTERNAL = 8u,
    ST_DISCONNECTED = 16u,
    ST_BAD_OFFSETS = 32u,
};

// Control block of one single-graph solve, in device memory.  Kernels of a
// captured round read it at block start; only the last block of a kernel
// (see last_block_done) advances it, after every other block has finished.
struct Ctl {
    const int32_t *src;
    const int32_t *dst;
    const void *w;
    int32_t *out;
    int64_t *out_count;
    uint32_t n, m, wt, vec_ok;
    uint32_t round;   // current round r
    uint32_t n_cur;   // components entering round r (ids 0..n_cur-1)
    uint32_t m_cur;   // live edges entering round r
    uint32_t n_next;  // components after round r (written by hook)
    uint32_t m_next;  // live edges after round r (written by compaction)
    uint32_t epoch;   // look-back descriptor epoch, +1 per scanning kernel
    uint32_t ticket;  // tile ticket of the running kernel
    uint32_t done;    // finished-block counter of the running kernel
    uint32_t deep;    // some pointer chase did not reach its root
    uint32_t deep_seen;  // value of deep at the end of the last compress pass
    uint32_t passes;     // follow-up compress passes in the current round
    uint32_t flag3[3];   // per-pass "chase unfinished" flags of the fused kernel
    uint32_t emitted;    // tree edges written by emit (own field: m_next may still be read)
    uint32_t status;  // ST_* bits
    uint32_t cnt_n[kMaxRounds + 2];  // roots numbered so far in round r (hook)
    uint32_t cnt_m[kMaxRounds + 2];  // edges kept so far in round r (compaction)
    uint32_t tail_cnt[kMaxRounds + 2];  // tail edge-list lengths (fused schedule)
    uint32_t tail_nn[kMaxRounds + 2];   // components after each tail round
    uint32_t tail_added;                // tree edges the tail added
    uint32_t tail_rounds;               // rounds the tail ran
    uint32_t tick_find0;                // tile tickets of the fused kernel's balanced phases
    uint32_t tick_hook[kMaxRounds + 2];
    uint32_t tick_comp[kMaxRounds + 2];
    uint32_t nphase;  // entries used in the phase log (fused schedule)
    uint8_t phase_kind[kMaxPhaseLog];
    uint8_t phase_round[kMaxPhaseLog];
    unsigned long long phase_ns[kMaxPhaseLog];  // %globaltimer at each phase end
    unsigned long long work_ns[kMaxPhaseLog];   // when CTA 0 finished its own work
    uint32_t stat_m[kMaxRounds + 1];
    uint32_t stat_n[kMaxRounds + 1];
};

// Workspace of the single-graph solver.  E[] holds live edge records
// (u, v, weight_bits, input edge id); mins[] the per-component minimum key,
// double-buffered by round parity.
struct Ws {
    Ctl *ctl;
    uint4 *E[2];
    unsigned long long *mins[2];
    int32_t *parent;   // hook pointer of each component (itself for a root)
    int32_t *nid;      // new dense id of each root
    int32_t *lab;      // new id of each component after compression
    uint32_t *mst_bits;
    uint2 *eends;              // current endpoints of a possible minimum edge, by input id
    unsigned long long *desc;  // look-back descriptors (emit of the graph schedule)
    uint32_t *emit_cnt;        // tree edges per emit chunk (fused schedule)
    uint32_t *emit_cta;        // tree edges in each CTA's range of emit chunks
    uint32_t *bar;             // grid-barrier counters of the fused kernel
    unsigned long long *pair_tab;  // lightest key per component pair (tail)
    uint4 *tl[2];                  // tail edge lists (a, b, weight_bits, input id)
    unsigned long long *tmin;      // tail: minimum key per component
    int32_t *tpar;                 // tail: hook pointers, then roots
    int32_t *tnid;                 // tail: new ids of the roots
    uint32_t n_cap, m_cap, desc_cap;
};

// ---------------------------------------------------------------- weights

__device__ __forceinline__ uint32_t weight_bits_f32(uint32_t b, uint32_t *status)
{
    if ((b & 0x7fffffffu) > 0x7f800000u) {  // NaN
        atomicOr(status, ST_NAN);
        return 0xffffffffu;
    }
    if (b == 0x80000000u)
        b = 0;  // -0 -> +0
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ uint32_t weight_bits(uint32_t raw, uint32_t wt, uint32_t *status)
{
    return wt ? weight_bits_f32(raw, status) : raw;
}

__device__ __forceinline__ unsigned long long make_key(uint32_t wbits, uint32_t pos)
{
    return ((unsigned long long)wbits << 32) | pos;
}

// ------------------------------------------------------------ memory helpers

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Fire-and-forget reductions (no returned value, so the issuing warp never
// waits on them).
__device__ __forceinline__ void red_min_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_or_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Offers `key` to the running minimum at p.  The load first filters keys
// that cannot win: values at p only decrease, so a cached (possibly older)
// value is never below the true one, and skipping key >= cached is exact.
// On hot components this turns most same-address atomics into cache hits.
__device__ __forceinline__ bool offer_min(unsigned long long *p, unsigned long long key)
{
    if (key < __ldca(p)) {
        red_min_u64(p, key);
        return true;
    }
    return false;
}

// Whether offers go through the filtering load: measured on GB300, a plain
// red.min.u64 sustains ~157 G/s on distinct addresses but ~1.5 G/s on one
// hot address, while the filtered offer costs ~15-65% on distinct addresses
// and is 25x faster on a hot one.  Filter when a target receives many
// offers on average (hot spots likely): at least 16 per target (swept over
// 2..32 on the grid and R-MAT workloads: 16 is fastest on both; at 32 the
// R-MAT round-0 find-min runs unfiltered into its hubs and takes twice as
// long).
__device__ __forceinline__ bool use_filter(uint32_t m_cur, uint32_t targets)
{
    return 2ull * m_cur >= 16ull * (unsigned long long)(targets > 0 ? targets : 1);
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p)
{
    return *(const volatile uint32_t *)p;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------- decoupled look-back scan
//
// Single-pass prefix sum over tiles (Merrill & Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", 2016).  Tiles are taken in order
// from an atomic ticket, so every predecessor of a waiting tile has already
// started and the wait ends.  A descriptor is one 64-bit word:
//   bits 0..30 value, bits 31..32 flag (1 aggregate, 2 inclusive prefix),
//   bits 33..63 epoch (a descriptor from another epoch reads as empty).
// Every wait is bounded by kSpinLimit; on expiry ST_TIMEOUT is set and the
// scan continues with a wrong value rather than hanging.

constexpr unsigned long long kDescAgg = 1ull << 31;
constexpr unsigned long long kDescPrefix = 2ull << 31;

__device__ __forceinline__ unsigned long long desc_word(uint32_t epoch, unsigned long long flag,
                                                        uint32_t value)
{
    return ((unsigned long long)(epoch & 0x7fffffffu) << 33) | flag | (value & 0x7fffffffu);
}

// Called by all 32 lanes of one warp.  Publishes the tile's aggregate, looks
// back over predecessors 32*kLookPerLane at a time (lane l reads distances
// l*kLookPerLane .. +kLookPerLane-1), publishes the inclusive prefix and
// returns the exclusive prefix (same value in every lane).  Measured on
// GB300: reading 4 per lane was slower than 1 (the extra loads cost more
// than the shorter walks save), so one per lane it is.
constexpr int kLookPerLane = 1;

__device__ __forceinline__ uint32_t lookback_warp(unsigned long long *desc, uint32_t tile,
                                                  uint32_t aggregate, uint32_t epoch,
                                                  uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long ep = (unsigned long long)(epoch & 0x7fffffffu);
    if (tile == 0) {
        if (lane == 0)
            st_relaxed_u64(&desc[0], desc_word(epoch, kDescPrefix, aggregate));
        return 0;
    }
    if (lane == 0)
        st_relaxed_u64(&desc[tile], desc_word(epoch, kDescAgg, aggregate));
    uint32_t excl = 0;
    int64_t hi = (int64_t)tile - 1;  // nearest predecessor not yet summed
    uint32_t spins = 0;
    for (;;) {
        // this lane's 4 predecessors, nearest first: flag, value
        uint32_t flag[kLookPerLane], val[kLookPerLane];
#pragma unroll
        for (int k = 0; k < kLookPerLane; k++) {
            const int64_t idx = hi - (lane * kLookPerLane + k);
            if (idx >= 0) {
                const unsigned long long d = ld_relaxed_u64(&desc[idx]);
                flag[k] = (d >> 33) == ep ? (uint32_t)((d >> 31) & 3u) : 0u;
                val[k] = (uint32_t)(d & 0x7fffffffu);
            } else {
                flag[k] = 2u;  // before tile 0: prefix 0
                val[k] = 0u;
            }
        }
        // within the lane: first prefix, any gap before it, sum up to it
        int first = kLookPerLane;
        bool gap = false;
        uint32_t part = 0;
#pragma unroll
        for (int k = kLookPerLane - 1; k >= 0; k--)
            if (flag[k] == 2u)
                first = k;
#pragma unroll
        for (int k = 0; k < kLookPerLane; k++)
            if (k <= first && k < kLookPerLane) {
                gap |= flag[k] == 0u;
                part += val[k];
            }
        const uint32_t pmask = __ballot_sync(0xffffffffu, first < kLookPerLane);
        const uint32_t zmask = __ballot_sync(0xffffffffu, gap);
        const uint32_t stop = pmask ? (uint32_t)(__ffs(pmask) - 1) : 32u;
        const uint32_t need = stop == 32u ? 0xffffffffu : ((2u << stop) - 1u);
        if (zmask & need) {  // an unpublished tile before the nearest prefix: wait
            if (++spins > kSpinLimit) {
                if (lane == 0) {
                    atomicOr(status, ST_TIMEOUT);
                    printf("mst: look-back gave up: tile %u epoch %u (block %u of %u)\n", tile,
                           epoch, blockIdx.x, gridDim.x);
                }
                break;
            }
            __nanosleep(20);
            continue;
        }
        uint32_t sum = ((uint32_t)lane <= stop) ? part : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        excl += sum;
        if (stop != 32u)
            break;
        hi -= 32 * kLookPerLane;
    }
    if (lane == 0)
        st_relaxed_u64(&desc[tile], desc_word(epoch, kDescPrefix, excl + aggregate));
    return excl;
}

// ------------------------------------------------------- block coordination

// Takes the next tile index from *ticket (thread 0) and broadcasts it.
__device__ __forceinline__ uint32_t next_tile(uint32_t *ticket, uint32_t *s_tile)
{
    __syncthreads();  // everyone has read the previous value
    if (threadIdx.x == 0)
        *s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    return *s_tile;
}

// Returns true in exactly one block: the last one to reach this point.  All
// writes of all other blocks are visible to it afterwards.
__device__ __forceinline__ bool last_block_done(uint32_t *done, uint32_t *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(done, 1u);
        *s_flag = (prev == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    const bool last = *s_flag != 0u;
    if (last)
        __threadfence();
    return last;
}

}  // namespace mst
