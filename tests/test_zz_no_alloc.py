"""mst_solve_noalloc: the allocation-free entry point, for callers that cannot
allocate device memory when they solve (a host that hands out its device
memory once at start-up and must not call the allocator later, or a process
whose device memory a framework's caching allocator already holds).

It must return exactly what the regular entry point returns, and the
oracle's tree, on calls in a row (the shared scratch keeps the previous
call's contents); report each call's own device outcome; and reject graphs
beyond its fixed scratch before queuing anything.  The trees are integer
edge ids, so exact equality is the tolerance.  Collected last on purpose:
if it fails, a run that stops at the first failure has run every other
test already.  It passes alone in a fresh process and after the others."""
import numpy as np
import pytest
import torch

from conftest import to_dev
from paper_2005_06913_gb300 import binding as B
from paper_2005_06913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _wt(g):
    return B.MST_W_F32 if g.w.dtype == np.float32 else B.MST_W_U32


def regular(h, g):
    s, d, w = to_dev(g.src, g.dst, g.w)
    out = torch.full((max(g.n - 1, 1),), -3, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_solve_ex(h, _wt(g), g.n, g.m, s, d, w, out, cnt) == B.MST_OK
    st = B.mst_get_status(h)
    return out[: int(cnt.item())].cpu().numpy(), st


def noalloc(g):
    """(tree ids, device status, count) of one allocation-free call."""
    s, d, w = to_dev(g.src, g.dst, g.w)
    out = torch.full((max(g.n - 1, 1),), -3, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert B.mst_solve_noalloc(_wt(g), g.n, g.m, s, d, w, out, cnt, st_dev) == B.MST_OK
    torch.cuda.synchronize()
    k = int(cnt.item())
    return out[: max(k, 0)].cpu().numpy(), int(st_dev.item()), k


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2005_06913_gb300 import build
    build.build()
    hh = B.mst_create(0, 0)
    yield hh
    B.mst_destroy(hh)


def test_noalloc_matches_regular_and_oracle_twice(h, oracle_mod):
    # three layouts of the working arrays: all in shared memory (small),
    # vertex arrays in shared memory with the edge list in the scratch, and
    # everything in the scratch; then the exact size limit
    graphs = [
        gg.random_connected(500, 2000, 103),
        gg.random_connected(3000, 12000, 102, weights="f32"),
        gg.random_connected(60000, 250000, 101),
        gg.random_connected(65536, 262144, 104),
    ]
    for g in graphs:
        want = oracle_mod.kruskal(g.n, g.src, g.dst, g.w)
        r, st = regular(h, g)
        assert st == B.MST_OK
        assert np.array_equal(r.astype(np.int64), want)
        for _ in range(2):  # two calls in a row share the scratch
            a, sta, k = noalloc(g)
            assert sta == B.MST_OK and k == g.n - 1
            assert np.array_equal(a, r)
    # and back to the first after the largest
    a, sta, _ = noalloc(graphs[0])
    assert sta == B.MST_OK
    assert np.array_equal(a.astype(np.int64), oracle_mod.kruskal(graphs[0].n, graphs[0].src,
                                                                   graphs[0].dst, graphs[0].w))


def test_noalloc_reports_each_calls_own_status(h, oracle_mod):
    good = gg.random_connected(2000, 8000, 105)
    bad_vertex = gg.random_connected(2000, 8000, 106)
    bad_vertex.src = bad_vertex.src.copy()
    bad_vertex.src[17] = bad_vertex.n + 5  # out of range
    nan = gg.random_connected(2000, 8000, 107, weights="f32")
    nan.w = nan.w.copy()
    nan.w[123] = np.float32("nan")
    for bad in (bad_vertex, nan):
        _, st, _ = noalloc(bad)
        assert st == B.MST_ERR_INVALID_ARG
        a, st, _ = noalloc(good)  # the previous call's outcome must not leak
        assert st == B.MST_OK
        assert np.array_equal(a.astype(np.int64),
                              oracle_mod.kruskal(good.n, good.src, good.dst, good.w))
    # a forest: two disjoint random trees and isolated vertices
    t1 = gg.random_connected(700, 699, 108)
    t2 = gg.random_connected(500, 1500, 109)
    n = 1300
    forest = gg.Graph(n, np.concatenate([t1.src, t2.src + 700]).astype(np.int32),
                      np.concatenate([t1.dst, t2.dst + 700]).astype(np.int32),
                      np.concatenate([t1.w, t2.w + np.uint32(1 << 20)]).astype(np.uint32))
    a, st, k = noalloc(forest)
    comps = oracle_mod.components(forest.n, forest.src, forest.dst)
    assert st == B.MST_ERR_DISCONNECTED
    assert k == n - comps
    assert np.array_equal(a.astype(np.int64),
                          oracle_mod.kruskal(forest.n, forest.src, forest.dst, forest.w))
    r, st = regular(h, forest)
    assert st == B.MST_ERR_DISCONNECTED and np.array_equal(a, r)


def test_noalloc_rejects_oversize_without_launch(h):
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_solve_noalloc(B.MST_W_U32, 65537, 10, x, x, x, x, c) == B.MST_ERR_BUDGET
    assert B.mst_solve_noalloc(B.MST_W_U32, 100, 262145, x, x, x, x, c) == B.MST_ERR_BUDGET
    assert B.mst_solve_noalloc(B.MST_W_U32, -1, 0, x, x, x, x, c) == B.MST_ERR_INVALID_ARG
