"""Adjacency-CSR input on the host (no GPU): the generator's CSR layout, the
claim behind the symmetric flag, and a model of the row-expansion kernel's
tiling and search (index logic only)."""
import numpy as np
import pytest

from paper_2005_06913_gb300 import graphgen as gg


def test_one_sided_csr_keeps_every_edge():
    g = gg.random_connected(500, 2000, 1)
    c = gg.to_csr(g, symmetric=False)
    e = gg.csr_entries(c)
    assert c.nnz == g.m and c.row_ptr[0] == 0 and c.row_ptr[-1] == g.m
    assert np.all(np.diff(c.row_ptr) >= 0)
    got = sorted(zip(e.src.tolist(), e.dst.tolist(), e.w.tolist()))
    assert got == sorted(zip(g.src.tolist(), g.dst.tolist(), g.w.tolist()))


def test_symmetric_csr_stores_both_ends():
    g = gg.random_connected(300, 1200, 2)
    g.dst[:5] = g.src[:5]  # self-loops are stored once
    c = gg.to_csr(g)
    e = gg.csr_entries(c)
    assert c.nnz == 2 * g.m - 5
    fwd = {(int(u), int(v), int(x)) for u, v, x in zip(e.src, e.dst, e.w)}
    for u, v, x in zip(g.src, g.dst, g.w):
        assert (int(u), int(v), int(x)) in fwd and (int(v), int(u), int(x)) in fwd


@pytest.mark.parametrize("seed", range(6))
def test_mirror_copies_never_win(oracle_mod, seed):
    """The symmetric flag turns each entry whose column is below its row into
    a self-loop; the tree over the entries must not change."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 400))
    m = int(rng.integers(1, 1500))
    g = gg.Graph(n, rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32),
                 rng.integers(0, 1 + int(rng.choice([2, 30, 1 << 20])), m).astype(np.uint32))
    e = gg.csr_entries(gg.to_csr(g))
    full = oracle_mod.kruskal(e.n, e.src, e.dst, e.w)
    src = np.where(e.dst < e.src, e.dst, e.src).astype(np.int32)
    assert np.array_equal(oracle_mod.kruskal(e.n, src, e.dst, e.w), full)


# --- a model of k_csr_rows: CTA tiles of 2,048 positions; thread 0 finds the
# rows of the tile's first and last positions; rows r0..r1 are staged when
# r1 - r0 + 1 < 2,049, else each position searches the whole table.
TILE, SPAN = 2048, 2049


def row_of(rp, lo, hi, p):
    while lo < hi:
        mid = lo + (hi - lo + 1) // 2
        if rp[mid] <= p:
            lo = mid
        else:
            hi = mid - 1
    return lo


def model_rows(rp, n, nnz):
    rows = np.empty(nnz, np.int64)
    staged_tiles = 0
    for p0 in range(0, nnz, TILE):
        p_last = min(nnz, p0 + TILE) - 1
        r0, r1 = row_of(rp, 0, n - 1, p0), row_of(rp, 0, n - 1, p_last)
        staged = r1 >= r0 and r1 - r0 + 1 < SPAN
        staged_tiles += staged
        if staged:
            span = rp[r0:r1 + 1]
            assert r1 <= n - 1 and len(span) <= SPAN  # stays inside row_ptr and the stage
        for p in range(p0, p_last + 1):
            rows[p] = r0 + row_of(span, 0, r1 - r0, p) if staged else row_of(rp, 0, n - 1, p)
    return rows, staged_tiles


@pytest.mark.parametrize("shape", ["dense", "empty-rows", "hub", "ragged"])
def test_row_expansion_model(shape):
    rng = np.random.default_rng(3)
    if shape == "dense":
        deg = rng.integers(1, 6, 3000)
    elif shape == "empty-rows":  # long runs of empty rows force the unstaged search
        deg = np.zeros(20000, np.int64)
        deg[::4000] = rng.integers(1, 3000, 5)
    elif shape == "hub":
        deg = rng.integers(0, 3, 5000)
        deg[17] = 9000
    else:
        deg = rng.integers(0, 2, 4097)
    n = deg.shape[0]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    nnz = int(rp[-1])
    rows, staged = model_rows(rp, n, nnz)
    assert np.array_equal(rows, np.repeat(np.arange(n), deg))
    if shape == "empty-rows":
        assert staged < (nnz + TILE - 1) // TILE
