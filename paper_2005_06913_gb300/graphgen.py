"""Seeded synthetic graph generators.

The paper evaluates on graphs made by its own generator from a vertex count
and an average degree (Section 3, Table 1: 10K/100K/1M vertices, degree
3/6/9); that generator and its graph files are not published.  These
generators stand in for them with five workload families of the same shape:

* ``random_connected``  random spanning tree (vertex i>0 joined to a uniform
  j<i) plus uniform random extra edges, no self-loops, no duplicates;
* ``grid2d``            R x C 4-neighbour grid, row-major vertex ids;
* ``rmat``              R-MAT power-law graph made connected by a random
  spanning tree;
* ``batched``           many ``random_connected`` graphs of log-uniform size,
  concatenated with int64 offset tables;
* ``serving_pool``      a pool of ``random_connected`` graphs with float32
  weights, replayed by the serving benchmark;
* ``to_csr``            any of these as an adjacency CSR (each undirected
  edge stored from both ends), and ``csr_entries`` back to per-entry COO.

Every generator is a pure function of its arguments and seed (numpy PCG64).
Nothing here computes a spanning tree or any part of one: the module only
builds inputs, and both the CPU oracle and the CUDA path consume them.

Edge arrays are ``int32`` COO (``src``, ``dst``); weights are ``uint32``
(distinct unless stated) or ``float32``.  An undirected edge is stored once.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph", "Batch", "random_connected", "grid2d", "rmat", "batched",
    "serving_pool", "paper_table1", "permutation_weights", "CSR", "to_csr", "csr_entries",
]

SEED_BASE = 0x4D5354  # "MST"


@dataclass
class Graph:
    """One undirected graph as COO arrays (edge id = index into the arrays)."""

    n: int
    src: np.ndarray  # int32 [m]
    dst: np.ndarray  # int32 [m]
    w: np.ndarray    # uint32 or float32 [m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    @property
    def wtype(self) -> str:
        return "f32" if self.w.dtype == np.float32 else "u32"


@dataclass
class Batch:
    """G graphs concatenated; vertex and edge ids are local to their graph."""

    vtx_off: np.ndarray  # int64 [G+1]
    edge_off: np.ndarray  # int64 [G+1]
    src: np.ndarray  # int32 [sum m]
    dst: np.ndarray  # int32 [sum m]
    w: np.ndarray    # uint32 or float32 [sum m]
    name: str = ""
    seeds: list = field(default_factory=list)

    @property
    def G(self) -> int:
        return int(self.vtx_off.shape[0] - 1)

    def graph(self, g: int) -> Graph:
        e0, e1 = int(self.edge_off[g]), int(self.edge_off[g + 1])
        return Graph(int(self.vtx_off[g + 1] - self.vtx_off[g]),
                     self.src[e0:e1], self.dst[e0:e1], self.w[e0:e1],
                     f"{self.name}[{g}]")


def permutation_weights(rng: np.random.Generator, m: int) -> np.ndarray:
    """A uniformly random permutation of 1..m as uint32 (all distinct)."""
    return (rng.permutation(m) + 1).astype(np.uint32)


def _float_weights(rng: np.random.Generator, m: int) -> np.ndarray:
    """float32 uniform in (0,1); ties are allowed (24-bit resolution)."""
    w = rng.random(m, dtype=np.float32)
    w[w == 0] = np.float32(2.0 ** -24)
    return w


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent compare)."""
    x = np.sort(x)
    if x.shape[0] < 2:
        return x
    return x[np.r_[True, x[1:] != x[:-1]]]


def _unique_first(keys: np.ndarray) -> np.ndarray:
    """Indices of the first occurrence of each distinct key, in input order."""
    _, first = np.unique(keys, return_index=True)
    first.sort()
    return first


def random_connected(n: int, m: int, seed: int, weights: str = "u32",
                     shuffle: bool = True) -> Graph:
    """Random spanning tree plus uniform extra edges; exactly ``m`` edges.

    Vertex i>0 is joined to a uniform j<i (n-1 tree edges); then uniform
    random vertex pairs are added, rejecting self-loops and pairs already
    present, until there are ``m`` edges.  ``weights`` is ``"u32"`` (a random
    permutation of 1..m) or ``"f32"`` (uniform in (0,1), ties possible).  With
    ``shuffle`` the edge order is randomly permuted once.
    """
    if n < 0 or m < 0:
        raise ValueError("n and m must be >= 0")
    if n == 0 and m:
        raise ValueError("edges need vertices")
    if n > 0 and m < n - 1:
        raise ValueError("m must be >= n-1 for a connected graph")
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the simple-graph maximum n(n-1)/2")
    rng = np.random.default_rng(seed)
    if n > 1:
        tv = np.arange(1, n, dtype=np.int64)
        tu = rng.integers(0, tv)  # uniform j < i
    else:
        tv = np.zeros(0, np.int64)
        tu = np.zeros(0, np.int64)
    us, vs = [tv], [tu]
    keys = np.minimum(tu, tv) * n + np.maximum(tu, tv)
    have = keys.shape[0]
    while have < m:
        need = m - have
        k = int(need * 1.25) + 64
        a = rng.integers(0, n, k)
        b = rng.integers(0, n, k)
        ok = a != b
        a, b = a[ok], b[ok]
        allk = np.concatenate([keys, np.minimum(a, b) * n + np.maximum(a, b)])
        first = _unique_first(allk)
        new = first[first >= keys.shape[0]] - keys.shape[0]
        new = new[:need]
        us.append(a[new])
        vs.append(b[new])
        keys = np.concatenate([keys, allk[keys.shape[0]:][new]])
        have = keys.shape[0]
    src = np.concatenate(us).astype(np.int32)[:m]
    dst = np.concatenate(vs).astype(np.int32)[:m]
    if shuffle and m:
        p = rng.permutation(m)
        src, dst = src[p], dst[p]
    w = permutation_weights(rng, m) if weights == "u32" else _float_weights(rng, m)
    return Graph(n, np.ascontiguousarray(src), np.ascontiguousarray(dst), w,
                 f"random_connected(n={n},m={m})")


def grid2d(rows: int, cols: int, seed: int, shuffle: bool = True) -> Graph:
    """``rows`` x ``cols`` 4-neighbour grid, vertex ``r*cols+c``.

    In generation order each vertex emits its right edge, then its down edge
    (m = rows(cols-1) + (rows-1)cols).  Weights are a random permutation of
    1..m.  With ``shuffle`` the edge order is randomly permuted once.
    """
    rng = np.random.default_rng(seed)
    r, c = np.meshgrid(np.arange(rows, dtype=np.int64),
                       np.arange(cols, dtype=np.int64), indexing="ij")
    v = (r * cols + c).ravel()
    right = (c < cols - 1).ravel()
    down = (r < rows - 1).ravel()
    # interleave: for each vertex, right edge (if any) then down edge (if any)
    su = np.stack([v, v], axis=1).ravel()
    sv = np.stack([v + 1, v + cols], axis=1).ravel()
    keep = np.stack([right, down], axis=1).ravel()
    src = su[keep].astype(np.int32)
    dst = sv[keep].astype(np.int32)
    m = src.shape[0]
    if shuffle and m:
        p = rng.permutation(m)
        src, dst = src[p], dst[p]
    w = permutation_weights(rng, m)
    return Graph(rows * cols, np.ascontiguousarray(src), np.ascontiguousarray(dst),
                 w, f"grid2d({rows}x{cols})")


def rmat(scale: int, edge_factor: int, seed: int,
         probs=(0.57, 0.19, 0.19, 0.05)) -> Graph:
    """R-MAT graph on 2**scale vertices with exactly edge_factor*2**scale edges.

    The edge set is a random spanning tree over a random vertex order (so the
    graph is connected) plus distinct R-MAT edges: batches of draws with
    quadrant probabilities ``probs``, each canonicalised to (min, max), with
    self-loops and edges already present dropped; from the last batch a
    uniform random subset is kept so that the total is exactly
    ``edge_factor * 2**scale``.  Weights are ``(rand24 << 8) | t`` with t the
    rank of the edge (by edge id) among edges with the same 24-bit random
    value, so all weights are distinct.  The edge order is randomly permuted.
    """
    n = 1 << scale
    target = edge_factor * n
    if target < n - 1:
        raise ValueError("edge_factor too small for a spanning tree")
    rng = np.random.default_rng(seed)
    order = rng.permutation(n).astype(np.int64)
    tv = order[1:]
    tu = order[rng.integers(0, np.arange(1, n, dtype=np.int64))]
    have = np.sort(np.minimum(tu, tv) * n + np.maximum(tu, tv))
    a, b, c, _ = probs
    # quadrant thresholds on a 16-bit uniform draw (resolution 2**-16)
    t1, t2, t3 = (np.uint16(min(65535, round(x * 65536))) for x in (a, a + b, a + b + c))
    while have.shape[0] < target:
        need = target - have.shape[0]
        k = int(need * 1.3) + 1024
        u = np.zeros(k, np.uint32)
        v = np.zeros(k, np.uint32)
        for _lvl in range(scale):
            x = np.frombuffer(rng.bytes(2 * k), dtype=np.uint16)
            ubit = x >= t2                                  # quadrants c, d
            vbit = ((x >= t1) & (x < t2)) | (x >= t3)      # quadrants b, d
            u <<= 1
            u |= ubit
            v <<= 1
            v |= vbit
        u = u.astype(np.int64)
        v = v.astype(np.int64)
        ok = u != v
        cand = _sorted_unique(np.minimum(u, v)[ok] * n + np.maximum(u, v)[ok])
        cand = cand[~np.isin(cand, have, assume_unique=True)]
        if cand.shape[0] > need:
            cand = cand[np.sort(rng.permutation(cand.shape[0])[:need])]
        have = np.sort(np.concatenate([have, cand]))
    keys = have[rng.permutation(target)]
    src = np.ascontiguousarray((keys // n).astype(np.int32))
    dst = np.ascontiguousarray((keys % n).astype(np.int32))
    r24 = rng.integers(0, 1 << 24, target, dtype=np.int64)
    packed = np.sort((r24 << 32) | np.arange(target, dtype=np.int64))
    rs = packed >> 32
    idx = packed & 0xFFFFFFFF
    starts = np.flatnonzero(np.r_[True, rs[1:] != rs[:-1]])
    rank = np.arange(target) - np.repeat(starts, np.diff(np.r_[starts, target]))
    if rank.max(initial=0) >= 256:
        raise RuntimeError("R-MAT weight tie group exceeds 256; reseed")
    w = np.empty(target, np.uint32)
    w[idx] = ((rs << 8) | rank).astype(np.uint32)
    ws = np.sort(w)
    if target > 1 and not np.all(ws[1:] != ws[:-1]):
        raise RuntimeError("R-MAT weights not distinct")
    return Graph(n, src, dst, w, f"rmat(scale={scale},ef={edge_factor})")


def _log_uniform_sizes(rng, count, lo, hi):
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def _one_graph(args):
    n, m, seed, weights = args
    return random_connected(n, m, seed, weights=weights)


def batched(G: int, nmin: int, nmax: int, degree: int, seed: int,
            weights: str = "u32", workers: int = 1) -> Batch:
    """G independent ``random_connected`` graphs, vertex counts log-uniform in
    [nmin, nmax], m_g = n_g*degree/2, each with its own sub-seed; packed with
    int64 ``vtx_off``/``edge_off`` offset tables (graph-local ids).  With
    ``workers`` > 1 the graphs are made by that many processes (started with
    ``spawn``); every graph depends only on its sub-seed, so the batch is the
    same either way."""
    rng = np.random.default_rng(seed)
    ns = _log_uniform_sizes(rng, G, nmin, nmax)
    subseeds = rng.integers(0, 2 ** 63 - 1, G)
    jobs = []
    for g in range(G):
        n = int(ns[g])
        m = min(n * degree // 2, n * (n - 1) // 2)
        jobs.append((n, m, int(subseeds[g]), weights))
    if workers > 1 and G > 1:
        import multiprocessing
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers,
                                 mp_context=multiprocessing.get_context("spawn")) as ex:
            parts = list(ex.map(_one_graph, jobs, chunksize=max(1, G // (8 * workers))))
    else:
        parts = [_one_graph(j) for j in jobs]
    vtx_off = np.zeros(G + 1, np.int64)
    edge_off = np.zeros(G + 1, np.int64)
    vtx_off[1:] = np.cumsum([p.n for p in parts])
    edge_off[1:] = np.cumsum([p.m for p in parts])
    cat = lambda xs, dt: (np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    wdt = np.uint32 if weights == "u32" else np.float32
    return Batch(vtx_off, edge_off, cat([p.src for p in parts], np.int32),
                 cat([p.dst for p in parts], np.int32), cat([p.w for p in parts], wdt),
                 f"batched(G={G},n=[{nmin},{nmax}],deg={degree})",
                 [int(s) for s in subseeds])


@dataclass
class CSR:
    """An adjacency CSR: entry p of row u is the edge (u, col[p]) with id p."""

    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    w: np.ndarray        # uint32 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def to_csr(g: Graph, symmetric: bool = True) -> CSR:
    """``g`` as an adjacency CSR.  With ``symmetric`` every edge is stored
    from both ends with its weight (self-loops once); otherwise only from
    its ``src``.  Rows are in vertex order and, within a row, entries keep
    the order of the edge ids."""
    if symmetric:
        loop = g.src == g.dst
        u = np.concatenate([g.src, g.dst[~loop]])
        v = np.concatenate([g.dst, g.src[~loop]])
        w = np.concatenate([g.w, g.w[~loop]])
        eid = np.concatenate([np.arange(g.m), np.flatnonzero(~loop)])
    else:
        u, v, w, eid = g.src, g.dst, g.w, np.arange(g.m)
    order = np.lexsort((eid, u))
    counts = np.bincount(u, minlength=g.n).astype(np.int64)
    row_ptr = np.zeros(g.n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(g.n, row_ptr, np.ascontiguousarray(v[order], np.int32),
               np.ascontiguousarray(w[order]))


def csr_entries(c: CSR) -> Graph:
    """The CSR's entries as an edge list: edge p = (row of p, col[p])."""
    rows = np.repeat(np.arange(c.n, dtype=np.int32), np.diff(c.row_ptr))
    return Graph(c.n, rows, c.col.copy(), c.w.copy(), "csr-entries")


def serving_pool(P: int, nmin: int, nmax: int, degree: int, seed: int,
                 workers: int = 1) -> Batch:
    """A pool of P graphs for the serving benchmark: log-uniform vertex counts
    in [nmin, nmax], average degree ``degree``, float32 weights in (0,1)."""
    return batched(P, nmin, nmax, degree, seed, weights="f32", workers=workers)


def paper_table1(name: str, seed: int = SEED_BASE) -> Graph:
    """The Table 1 shapes: ``Graph10K_3`` ... ``Graph1M_9`` (n vertices,
    average degree d, so m = n*d/2), built with ``random_connected``."""
    size, deg = name.replace("Graph", "").split("_")
    n = {"10K": 10_000, "100K": 100_000, "1M": 1_000_000}[size]
    d = int(deg)
    return random_connected(n, n * d // 2, seed)


# The five benchmark workloads, C1..C5 in order.
def config(i: int, small: bool = False):
    """Workload ``i`` (1..5).  ``small`` shrinks C3-C5 for quick checks."""
    s = SEED_BASE + i - 1
    if i == 1:
        return random_connected(4096, 32768, s)
    if i == 2:
        return grid2d(1024, 1024, s)
    if i == 3:
        return rmat(16 if small else 22, 8, s)
    if i == 4:
        return batched(64 if small else 4096, 64, 4096 if small else 65536, 8, s)
    if i == 5:
        return serving_pool(16 if small else 4096, 1024, 16384 if small else 1048576, 6, s)
    raise ValueError(i)
