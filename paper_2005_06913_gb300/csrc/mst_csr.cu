// Adjacency-CSR input: the row of every CSR entry, so that the entries can
// be solved as an edge list whose ids are their CSR positions.
//
// The paper's graphs are edge lists (Section 2.1, graph_edge[] with src,
// dest, weight); a CSR of the same graph lists each vertex's incident edges
// contiguously.  Entry p of row u is the edge (u, col[p]) with id p.  Under
// the edge order (weight, id) the lighter of two parallel entries wins, so
// when the caller declares the CSR symmetric (each undirected edge stored
// from both ends with one weight), the copy in the higher row can never
// enter the tree: it is turned into a self-loop, which no step offers, and
// the result is unchanged.
#include "mst_internal.h"

namespace mst {

constexpr int kCsrThreads = 256, kCsrIpt = 8;
constexpr uint32_t kCsrTile = kCsrThreads * kCsrIpt;  // CSR positions per CTA
constexpr uint32_t kCsrSpan = kCsrTile + 1;           // row offsets staged per CTA

// Largest u in [lo, hi] with rp[u] <= p (lo when there is none).
__device__ __forceinline__ uint32_t csr_row_of(const int64_t *rp, uint32_t lo, uint32_t hi,
                                               int64_t p)
{
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo + 1) / 2;
        if (__ldg(rp + mid) <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One CTA writes the rows of kCsrTile consecutive positions.  The rows its
// tile spans are found by two searches; their offsets are staged in shared
// memory when they fit (they always do unless the tile crosses more than
// kCsrTile empty rows), and each position then searches the stage.
__global__ void __launch_bounds__(kCsrThreads) k_csr_rows(const int64_t *rp, const int32_t *col,
                                                         uint32_t n, uint32_t nnz,
                                                         uint32_t symmetric, int32_t *rows)
{
    __shared__ int64_t span[kCsrSpan];
    __shared__ uint32_t r_lo, r_hi;
    const uint32_t p0 = blockIdx.x * kCsrTile;
    const uint32_t p_last = (nnz - p0 < kCsrTile ? nnz : p0 + kCsrTile) - 1;
    if (threadIdx.x == 0) {
        r_lo = csr_row_of(rp, 0, n - 1, p0);
        r_hi = csr_row_of(rp, 0, n - 1, p_last);
    }
    __syncthreads();
    const uint32_t r0 = r_lo, r1 = r_hi;
    const bool staged = r1 >= r0 && r1 - r0 + 1 < kCsrSpan;
    if (staged)
        for (uint32_t i = threadIdx.x; i <= r1 - r0; i += kCsrThreads)
            span[i] = __ldg(rp + r0 + i);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kCsrIpt; j++) {
        const uint32_t p = p0 + j * kCsrThreads + threadIdx.x;
        if (p > p_last)
            break;
        uint32_t u;
        if (staged) {
            uint32_t lo = 0, hi = r1 - r0;
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo + 1) / 2;
                if (span[mid] <= (int64_t)p)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            u = r0 + lo;
        } else {
            u = csr_row_of(rp, 0, n - 1, p);
        }
        int32_t r = (int32_t)u;
        if (symmetric) {
            const int32_t v = __ldg(col + p);
            if (v >= 0 && (uint32_t)v < u)
                r = v;  // the copy in the higher row: a self-loop (v, v)
        }
        rows[p] = r;
    }
}

// Checks the offsets (rp[0] = 0, rp[n] = nnz, non-decreasing).  A malformed
// table marks position 0 with row -1, which the solve reports as a bad
// vertex id.  Runs after k_csr_rows on the same stream, so its mark wins.
__global__ void k_csr_check(const int64_t *rp, uint32_t n, uint32_t nnz, int32_t *rows)
{
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    bool bad = gtid == 0 && (__ldg(rp) != 0 || __ldg(rp + n) != (int64_t)nnz);
    for (size_t u = gtid; u < n; u += stride)
        bad |= __ldg(rp + u) > __ldg(rp + u + 1);
    if (bad)
        rows[0] = -1;
}

cudaError_t csr_rows(const int64_t *row_ptr, const int32_t *col, uint32_t n, uint32_t nnz,
                     bool symmetric, int32_t *rows, int num_sms, cudaStream_t stream)
{
    if (nnz == 0 || n == 0)
        return cudaSuccess;
    const uint32_t tiles = (nnz + kCsrTile - 1) / kCsrTile;
    k_csr_rows<<<tiles, kCsrThreads, 0, stream>>>(row_ptr, col, n, nnz, symmetric ? 1u : 0u,
                                                  rows);
    const uint32_t want = (n + kCsrThreads - 1) / kCsrThreads;
    const uint32_t cap = (uint32_t)(num_sms > 0 ? num_sms : 1) * 8;
    k_csr_check<<<want < cap ? want : cap, kCsrThreads, 0, stream>>>(row_ptr, n, nnz, rows);
    return cudaGetLastError();
}

}  // namespace mst
