/*
 * mst.h — C ABI of libmst: minimum spanning trees by data-parallel Boruvka
 * rounds on one NVIDIA GB300 (sm_103a).
 *
 * The method (Boruvka; "Parallel Minimum Spanning Tree Algorithms and
 * Evaluation", Section 2.1) repeats rounds until no edge joins two
 * components: every component picks its lightest outgoing edge, those edges
 * are added to the tree M and the components they join are merged.  The
 * paper's "Optimization" (Section 2.1) drops edges that have become internal
 * to a component; here they are removed physically every round.
 *
 * Problem (Section 1 defines the tree, Section 2.1 "Inputs" the graph): an
 * undirected graph with n vertices 0..n-1 and m edges given as COO arrays
 * src[m], dst[m] and weights w[m]; edge id e is the index into these arrays.
 * The result is the minimum spanning tree, or the minimum spanning forest
 * when the graph is not connected.  The paper assumes distinct weights; this
 * library accepts ties and breaks them by edge id (the lighter of two edges
 * with equal weight is the one with the smaller id), which makes the result
 * unique for every input.  Self-loops and parallel edges are allowed.
 *
 * Conventions for every entry point:
 *   - Pointers named src, dst, w, out_*, *_off are DEVICE pointers, owned by
 *     the caller, and must stay valid until the work queued on `stream`
 *     completes.  `stream` is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream).  Calls are asynchronous: they return after
 *     queueing work; results are ready when the stream reaches that point.
 *   - Argument errors are detected on the host, before any work is queued,
 *     and returned synchronously.  Conditions found on the device (a vertex
 *     id out of range, a NaN weight, a disconnected graph, a bounded wait
 *     that ran out) are recorded in a device status word that
 *     mst_get_status() returns; an out-of-range edge is ignored and a NaN
 *     weight sorts after every other weight.
 *   - A handle owns device workspace sized for the largest problem it has
 *     solved; it grows on demand (cudaMalloc) and is freed by mst_destroy.
 *     A handle is not thread-safe and its workspace is shared by all calls
 *     on it: use one handle per host thread and per stream.
 *   - Limits: 0 <= n <= 2^31-1, 0 <= m <= 2^31-1.
 */
#ifndef MST_H
#define MST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mst_handle_s *mst_handle;

typedef enum {
    MST_OK = 0,
    MST_ERR_INVALID_ARG = 1,  /* bad argument (host) or bad vertex id / NaN (device) */
    MST_ERR_OOM = 2,          /* device allocation failed */
    MST_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    MST_ERR_DISCONNECTED = 4, /* informational: the result is a spanning forest */
    MST_ERR_TIMEOUT = 5,      /* a bounded device wait gave up; results invalid */
    MST_ERR_BUDGET = 6,       /* the request does not fit the memory budget */
    MST_ERR_INTERNAL = 7      /* an internal consistency check failed */
} mst_status;

typedef enum {
    MST_W_U32 = 0, /* uint32 weights, compared as unsigned integers */
    MST_W_F32 = 1  /* float32 weights, compared as floats; -0 equals +0 */
} mst_weight_type;

/* Human-readable name of a status code (static string). */
const char *mst_status_string(mst_status s);

/*
 * Creates a handle on CUDA device `device`.  mem_budget_bytes caps the
 * device memory this handle may allocate (0 = no cap): the single-graph and
 * batched workspaces, the staging of mst_solve_host and the row buffer of
 * mst_solve_csr, together; a solve whose growth would exceed it returns
 * MST_ERR_BUDGET.  *h receives the handle.
 */
mst_status mst_create(mst_handle *h, int device, size_t mem_budget_bytes);

/* Waits for the handle's work, frees its workspace and the handle. */
mst_status mst_destroy(mst_handle h);

/*
 * Minimum spanning tree of one graph with uint32 weights (Section 2.1 rounds).
 *   n, m          vertex and edge counts.
 *   src, dst      int32[m] edge endpoints in [0, n).
 *   w             uint32[m] weights.
 *   out_edge_ids  int32 capacity >= max(n-1, 0): receives the ids of the
 *                 tree edges in ascending order.
 *   out_count     one int64: receives the number of ids written
 *                 (n - number of connected components).
 * Runs asynchronously on `stream`.  Returns MST_ERR_INVALID_ARG for negative
 * or too-large sizes, NULL pointers with nonzero sizes, or a NULL handle.
 * Under the default (fused) schedule the solve is one cooperative launch
 * whose CTAs wait on each other at grid barriers, so all of its CTAs must be
 * resident at once.  The library orders fused solves on one device among
 * themselves: each waits on its stream for the previous fused solve of the
 * process on that device (any handle, any stream) to finish, so concurrent
 * callers are safe; batched solves and other kernels still run beside a
 * fused solve.  A stream being captured into a CUDA graph is left out of
 * that ordering, and the caller orders what it replays.
 */
mst_status mst_solve(mst_handle h, int32_t n, int64_t m,
                     const int32_t *src, const int32_t *dst, const void *w,
                     int32_t *out_edge_ids, int64_t *out_count, void *stream);

/* As mst_solve, with the weight type given explicitly (uint32 or float32). */
mst_status mst_solve_ex(mst_handle h, mst_weight_type wt, int32_t n, int64_t m,
                        const int32_t *src, const int32_t *dst, const void *w,
                        int32_t *out_edge_ids, int64_t *out_count, void *stream);

/* Flags of mst_solve_csr. */
#define MST_CSR_SYMMETRIC 1u

/*
 * Minimum spanning forest of a graph given as an adjacency CSR (a layout
 * the paper does not use: its graphs are edge lists, Section 2.1 data
 * structures).  row_ptr (device, int64, n+1 entries) holds the offsets of
 * each vertex's entries; col (device, int32, nnz) the other endpoint and w
 * (device, uint32 or float32 per wt, nnz) the weight of each entry.  Entry
 * p of row u is the edge (u, col[p]) with id p, so out_edge_ids (device,
 * capacity >= max(n-1,0)) receives CSR positions, ascending, and
 * *out_count (device int64) their number: the same result as mst_solve_ex
 * on the edge list (row of p, col[p], w[p]).  With MST_CSR_SYMMETRIC the
 * caller declares every undirected edge stored from both ends with one
 * weight; the copy in the higher row can then never enter the tree (the
 * lower position wins the tie) and is skipped, which halves the edges of
 * the later rounds without changing the result.  Entries in the higher row
 * without a mirror are dropped under that flag.
 * The row of each entry is written into device memory owned by the handle
 * (4 B per entry, grown on demand, counted in the memory budget), so
 * row_ptr, col and w are not modified and need not outlive the call's
 * stream work.  With nnz = 0, row_ptr is not read.  A malformed offset
 * table (row_ptr[0] != 0, row_ptr[n] != nnz, or decreasing offsets) is
 * reported on the device as MST_ERR_INVALID_ARG by mst_get_status, as a bad
 * vertex id in col is.  Host errors: MST_ERR_INVALID_ARG for a NULL handle,
 * bad wt or flags, negative sizes, nnz > INT32_MAX or missing pointers;
 * MST_ERR_BUDGET or MST_ERR_OOM when the row buffer cannot grow.
 */
mst_status mst_solve_csr(mst_handle h, mst_weight_type wt, int32_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col, const void *w,
                         uint32_t flags, int32_t *out_edge_ids, int64_t *out_count,
                         void *stream);

/*
 * Host-buffer form of mst_solve_ex for callers whose graph is in host memory
 * (src, dst, w are host pointers).  If all three are page-locked (pinned)
 * and the fused schedule is selected, the kernel reads them itself in round
 * 0 over the host link and writes their device copy into staging owned by
 * the handle; otherwise they are first copied into that staging.  The
 * tree's edge ids (host int32 capacity >= max(n-1,0)) and *out_count (host
 * int64) are written by the kernel itself when they too are pinned (and the
 * inputs are), else copied back; the call returns after the result is in
 * host memory (synchronises `stream`).  The host inputs must not change until the
 * call returns.  Returns an argument error, or else the device status as
 * mst_get_status.
 */
mst_status mst_solve_host(mst_handle h, mst_weight_type wt, int32_t n, int64_t m,
                          const int32_t *src, const int32_t *dst, const void *w,
                          int32_t *out_edge_ids, int64_t *out_count, void *stream);

/*
 * Minimum spanning trees of G independent graphs in one launch.  Each graph
 * gets the Section 2.1 rounds (find-min, union, "covered" edges dropped)
 * and the tree of Section 1; the batching itself has no counterpart in the
 * paper, which solves one graph at a time.
 *   vtx_off, edge_off  int64[G+1] device offset tables: graph g has
 *                      n_g = vtx_off[g+1]-vtx_off[g] vertices and edges
 *                      edge_off[g] .. edge_off[g+1]-1 of src/dst/w.
 *   src, dst           int32 endpoints, LOCAL to their graph (0..n_g-1).
 *   w                  uint32 or float32 weights (per `wt`).
 *   total_n, total_m   vtx_off[G] and edge_off[G] (used to size workspace;
 *                      a mismatch found on the device is MST_ERR_INVALID_ARG).
 *   out_edge_ids       int32[total_n]: graph g writes its tree's LOCAL edge
 *                      ids, ascending, at out_edge_ids + vtx_off[g].
 *   out_counts         int64[G]: number of ids written for each graph.
 * Each graph's result is the same as mst_solve_ex on that graph alone.
 * Constraints per graph: n_g, m_g <= 2^31-1.
 */
mst_status mst_solve_batched(mst_handle h, mst_weight_type wt, int32_t G,
                             const int64_t *vtx_off, const int64_t *edge_off,
                             int64_t total_n, int64_t total_m,
                             const int32_t *src, const int32_t *dst, const void *w,
                             int32_t *out_edge_ids, int64_t *out_counts, void *stream);

/*
 * Synchronises `stream` and returns the device status of the handle's last
 * solve: MST_OK, MST_ERR_DISCONNECTED (forest written), MST_ERR_INVALID_ARG
 * (bad vertex id or NaN weight seen), MST_ERR_TIMEOUT or MST_ERR_INTERNAL.
 * The status word is cleared at the start of each solve.
 */
mst_status mst_get_status(mst_handle h, void *stream);

/*
 * Per-graph outcome of the handle's last batched solve (mst_solve_batched or
 * mst_autotune_batched); synchronises `stream`.  statuses (host, G entries,
 * G <= the batch's graph count) receives for each graph the status
 * mst_get_status would report for a solve of that graph alone: MST_OK,
 * MST_ERR_DISCONNECTED (forest written), MST_ERR_INVALID_ARG (a bad vertex
 * id or NaN weight in that graph, or a malformed offset table, which leaves
 * every graph of the batch unsolved), MST_ERR_INTERNAL.  One graph's bad
 * input does not change its batch-mates' results or statuses; the combined
 * status of mst_get_status is the union of all graphs' conditions.
 * MST_ERR_INVALID_ARG when the last solve on the handle was not batched.
 * The paper solves one graph at a time (Section 2.1); this is the batched
 * path's per-graph form of its result.
 */
mst_status mst_get_batched_status(mst_handle h, void *stream, int32_t G, int32_t *statuses);

/*
 * Per-round sizes of the handle's last single-graph solve (synchronises
 * `stream`): live_edges[r] = edges entering round r (round 0 = m),
 * live_vertices[r] = components entering round r; *rounds = number of
 * rounds run.  At most `cap` entries are written.  Used to count the bytes
 * the method moves.
 */
mst_status mst_get_round_stats(mst_handle h, void *stream, int64_t *live_edges,
                               int64_t *live_vertices, int32_t cap, int32_t *rounds);

/* Time and traffic model of one kernel of a solve (see mst_profile_last_solve). */
typedef struct {
    char name[32];       /* kernel name, e.g. "k_compact<R>" */
    int32_t launches;    /* launches in the solve */
    double total_ms;     /* sum of CUDA-event durations of those launches */
    double alg_bytes;    /* algorithmic DRAM bytes of those launches (model) */
} mst_kernel_profile;

/*
 * Per-kernel (or per-phase) time and traffic model of the handle's last
 * single-graph solve.  Under the fused schedule (the default) the entries
 * are the phases of the one cooperative kernel (init, find0, hook,
 * compress, compact, tail, emit), timed inside that kernel itself by %globaltimer
 * stamps at each grid barrier; nothing is re-run.  Under the graph schedule
 * the solve is re-run (same device buffers, which must still be valid) with
 * each kernel launched separately between two CUDA events on `stream`, and
 * the outputs are written again.  alg_bytes counts the bytes the method must
 * move through DRAM (edge lists and per-vertex arrays; label gathers and
 * atomics, which stay in L2, are not counted).  Writes at most `cap`
 * entries, sets *count, and synchronises `stream`.
 */
mst_status mst_profile_last_solve(mst_handle h, void *stream, mst_kernel_profile *out,
                                  int32_t cap, int32_t *count);

/*
 * Schedule of single-graph solves.  schedule: 0 = default: one cooperative
 * persistent launch per solve whose phases are separated by grid barriers,
 * with its shape chosen per solve (one CTA per SM: 256 threads up to 600,000
 * edges, 1024 above); 1 = the same kernel with a fixed shape, where
 * block_threads (256, 512, 768 or 1024; 0 = keep, default 256) sets the CTA
 * size and blocks_per_sm (1..8, 0 = keep, default 4) the CTAs per SM, clamped
 * to what fits (64 registers a thread: 1024 threads a CTA fit once per SM,
 * 256 four times); 2 = one kernel per phase replayed from a CUDA graph whose
 * round loop is a device-side conditional WHILE node; 3 = an ablation of
 * schedule 0 after the sequential "covered" optimisation (Section 2.1): the
 * edge list is never compacted, every round reads all m slots and edges that
 * became internal are flagged in their slot and skipped; 4 = an ablation of
 * schedule 0 after the compare-and-swap algorithm (Section 2.2.2): each
 * component's minimum edge joins the current roots of its endpoints by a
 * compare-and-swap of the higher root's parent to the lower root, retried
 * after fresh finds when it fails, and the roots left are numbered in a
 * phase of their own.  Results are identical under every setting.
 */
mst_status mst_set_single_schedule(mst_handle h, int schedule, int blocks_per_sm,
                                   int block_threads);

/*
 * Failure injection for the bounded waits of the default (fused) schedule.
 * Its CTAs meet at grid barriers whose waits are bounded; a wait that runs
 * out sets MST_ERR_TIMEOUT in the device status, every CTA leaves the solve
 * at its next barrier (no phase reads the results of an incomplete one),
 * *out_count is set to 0, and the handle stays usable.  polls sets how many
 * polls a barrier wait makes before it gives up (0 restores the default,
 * 2^22 polls, long enough that only a grid that can never complete gives
 * up).  A tiny value makes solves time out on purpose, to exercise that
 * path.  Kept by the handle across workspace growth.  The paper's waits are
 * lock acquisitions (Section 2.2.1); this library has none, only these.
 */
mst_status mst_set_wait_limit(mst_handle h, uint32_t polls);

/*
 * Schedule control for the batched solver (the autotuner's knob).
 * schedule: 0 = automatic (cached autotune result per size bucket, else the
 * built-in default), 1 = one thread block per graph, 2 = one warp per graph
 * for small graphs and a block per graph otherwise.  block_threads: 128,
 * 256, 512 or 1024 (0 = automatic).
 */
mst_status mst_set_batched_schedule(mst_handle h, int schedule, int block_threads);

/*
 * Autotunes the batched solver on the given batch (same arguments as
 * mst_solve_batched): times each candidate schedule five times (after one
 * warm-up launch) per size bucket, keeps the one with the lowest median,
 * and, when cache_path is not NULL, stores the choice as
 * JSON there (and loads it on later calls).  Synchronises `stream`.
 */
mst_status mst_autotune_batched(mst_handle h, mst_weight_type wt, int32_t G,
                                const int64_t *vtx_off, const int64_t *edge_off,
                                int64_t total_n, int64_t total_m,
                                const int32_t *src, const int32_t *dst, const void *w,
                                int32_t *out_edge_ids, int64_t *out_counts,
                                const char *cache_path, void *stream);

/*
 * Allocation-free solve of one small graph.  For callers that cannot
 * allocate device memory at the point where they solve: a real-time or
 * plugin host that hands out all of its device memory once at start-up and
 * must not call the allocator later (cudaMalloc and cudaFree can
 * synchronise the device and take unbounded time), or a process whose
 * device memory a framework's caching allocator already holds, so that a
 * cudaMalloc would fail.  The paper has no counterpart; it is a deployment
 * form of the same Section 2.1 rounds.
 *   Takes no handle and calls no cudaMalloc, cudaFree or allocating
 *   library routine.  One thread block solves the graph on `stream`, with
 *   its working arrays in shared memory or in a fixed scratch array that the
 *   library declares at file scope: every GPU that loads the library holds
 *   that array (6,062,340 bytes) until the process exits.
 *   Limits: n <= 65536 and m <= 262144; larger graphs return MST_ERR_BUDGET
 *   before anything is queued.
 *   Arguments as in mst_solve_ex (device pointers, current device).
 *   out_status: optional device int32 (NULL = none) receiving the device
 *   outcome as an mst_status (MST_OK, MST_ERR_DISCONNECTED,
 *   MST_ERR_INVALID_ARG for a bad vertex id or NaN, MST_ERR_TIMEOUT,
 *   MST_ERR_INTERNAL).
 *   The first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress, with that device current) and sets the kernel's
 *   shared-memory limit; that first call should come before any stream
 *   capture.  All calls share the one array, which keeps the last call's
 *   contents (the kernel clears what must start empty): calls that may
 *   overlap on the GPU (other streams, other host threads) race on it and
 *   must be serialised by the caller.
 */
mst_status mst_solve_noalloc(mst_weight_type wt, int32_t n, int64_t m,
                             const int32_t *src, const int32_t *dst, const void *w,
                             int32_t *out_edge_ids, int64_t *out_count, int32_t *out_status,
                             void *stream);

/* ---------------------------------------------------------------- serving */

/*
 * Continuous-batching server on top of the batched solver (the paper has no
 * counterpart; each request's result is the Section 1 tree of its graph, as
 * computed by the Section 2.1 rounds).  A host thread
 * admits submitted graphs under the handle's memory budget, launches each
 * admitted group as one batched solve on one of `streams` CUDA streams, and
 * admits new requests as soon as a stream and memory are free, so solves of
 * requests that arrive while others run overlap on the GPU.  max_batch caps
 * the graphs per launch.  A request with more than 131072 edges is not
 * batched with the small ones: it goes to the fused lane, where the fused
 * single-graph kernel solves it in a workspace owned by the server (on the
 * whole co-resident grid when nothing else is in flight, else on half of
 * it), while small requests keep being batched past it on other streams.
 * Lane requests that queue up behind one another (up to 16, of one weight
 * type) are solved in one launch as a single union graph and cut back
 * apart, which gives each the tree and the status of a solve of it alone.
 */
mst_status mst_server_start(mst_handle h, int streams, int max_batch);

/*
 * Queues one graph (device pointers, as in mst_solve_ex; they must stay
 * valid until the request completes).  *ticket receives the request id.
 * The submit time is taken now; latency = completion - submit.
 */
mst_status mst_submit(mst_handle h, mst_weight_type wt, int32_t n, int64_t m,
                      const int32_t *src, const int32_t *dst, const void *w,
                      int32_t *out_edge_ids, int64_t *out_count, uint64_t *ticket);

/*
 * Non-blocking poll: *done = 1 once the request's outputs are written.
 * When done and latency_us is not NULL, *latency_us = completion - submit in
 * microseconds (host clock, completion seen by the server thread).
 */
mst_status mst_poll(mst_handle h, uint64_t ticket, int *done, double *latency_us);

/* Blocks until every submitted request has completed. */
mst_status mst_server_drain(mst_handle h);

/* Drains, stops the server thread and releases its streams. */
mst_status mst_server_stop(mst_handle h);

#ifdef __cplusplus
}
#endif

#endif /* MST_H */
