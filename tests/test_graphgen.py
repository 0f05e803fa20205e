"""Seeded generators: shapes, exact sizes, simple graphs, connectivity,
distinct weights, determinism (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from paper_2005_06913_gb300 import graphgen as gg


def check_simple_connected(g, distinct=True):
    assert g.src.dtype == np.int32 and g.dst.dtype == np.int32
    assert g.src.shape == g.dst.shape == g.w.shape
    assert (g.src >= 0).all() and (g.src < g.n).all()
    assert (g.dst >= 0).all() and (g.dst < g.n).all()
    assert (g.src != g.dst).all()
    lo = np.minimum(g.src, g.dst).astype(np.int64)
    hi = np.maximum(g.src, g.dst).astype(np.int64)
    key = np.sort(lo * g.n + hi)
    assert (key[1:] != key[:-1]).all(), "duplicate edge"
    if distinct:
        ws = np.sort(g.w)
        assert (ws[1:] != ws[:-1]).all(), "weights not distinct"
    mat = sp.coo_matrix((np.ones(g.m), (g.src, g.dst)), shape=(g.n, g.n))
    assert connected_components(mat, directed=False)[0] == 1


@pytest.mark.parametrize("n,m", [(2, 1), (10, 20), (4096, 32768), (1000, 999), (50, 1225)])
def test_random_connected(n, m):
    g = gg.random_connected(n, m, 123)
    assert g.m == m and g.n == n
    check_simple_connected(g)
    assert sorted(g.w.tolist()) == list(range(1, m + 1))


def test_random_connected_float():
    g = gg.random_connected(5000, 15000, 9, weights="f32")
    assert g.w.dtype == np.float32 and (g.w > 0).all() and (g.w < 1).all()
    check_simple_connected(g, distinct=False)


def test_grid():
    g = gg.grid2d(33, 17, 5)
    assert g.m == 33 * 16 + 32 * 17
    check_simple_connected(g)
    d = np.abs(g.src.astype(np.int64) - g.dst)
    assert set(np.unique(d).tolist()) == {1, 17}
    c2 = gg.config(2)
    assert c2.n == 1 << 20 and c2.m == 2 * 1024 * 1023


def test_rmat_small():
    g = gg.rmat(12, 8, 3)
    assert g.n == 4096 and g.m == 8 * 4096
    check_simple_connected(g)
    deg = np.bincount(np.r_[g.src, g.dst], minlength=g.n)
    assert deg.max() > 20 * deg.mean()  # power-law hubs


def test_batched_offsets():
    b = gg.batched(40, 64, 2048, 8, 4)
    assert b.vtx_off[0] == 0 and b.edge_off[0] == 0
    assert b.edge_off[-1] == b.src.shape[0]
    ns = np.diff(b.vtx_off)
    assert (ns >= 64).all() and (ns <= 2048).all()
    assert (np.diff(b.edge_off) == ns * 4).all()
    for g in range(b.G):
        check_simple_connected(b.graph(g))


def test_deterministic():
    a = gg.random_connected(300, 900, 77)
    b = gg.random_connected(300, 900, 77)
    c = gg.random_connected(300, 900, 78)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.w, b.w)
    assert not np.array_equal(a.src, c.src)


def test_paper_table1_shapes():
    g = gg.paper_table1("Graph10K_6")
    assert g.n == 10_000 and g.m == 30_000
    check_simple_connected(g)
