"""Single-graph CUDA path vs the CPU oracle (bit-exact edge-id sets).

Every case compares the ascending edge ids returned through the C ABI with
the oracle's Kruskal result on the same seeded input.  Integer work: the bar
is exact equality.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import to_dev
from paper_2005_06913_gb300 import binding as B
from paper_2005_06913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def gpu_solve(h, n, src, dst, w, stream=None):
    m = src.shape[0]
    s, d, ww = to_dev(src, dst, w)
    out = torch.full((max(n - 1, 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    wt = B.MST_W_F32 if w.dtype == np.float32 else B.MST_W_U32
    st = B.mst_solve_ex(h, wt, n, m, s, d, ww, out, cnt, stream)
    assert st == B.MST_OK, B.mst_status_string(st)
    status = B.mst_get_status(h, stream)
    k = int(cnt.item())
    return out[:k].cpu().numpy().astype(np.int64), status


def check(h, n, src, dst, w):
    got, status = gpu_solve(h, n, src, dst, w)
    expect = oracle.kruskal(n, src, dst, w)
    assert got.shape == expect.shape, (got.shape, expect.shape)
    assert np.array_equal(got, expect)
    comps = oracle.components(n, src, dst)
    assert status == (B.MST_OK if comps <= 1 else B.MST_ERR_DISCONNECTED)
    return got


@pytest.fixture(params=[0, 1, 2, 3, 4],
                ids=["fused-auto", "fused-fixed", "graph", "covered", "cas-hook"])
def sched(request, handle):
    """Runs a test under each single-graph schedule."""
    assert B.mst_set_single_schedule(handle, request.param, 0) == B.MST_OK
    yield handle
    B.mst_set_single_schedule(handle, 0, 0)


@pytest.mark.parametrize("n,m", [(2, 1), (3, 3), (17, 40), (1000, 3001), (1023, 1022),
                                 (1025, 4100), (4096, 32768), (5000, 200000), (70001, 250003)])
def test_random_connected(sched, n, m):
    g = gg.random_connected(n, m, n * 7 + m)
    check(sched, g.n, g.src, g.dst, g.w)


@pytest.mark.parametrize("bps,threads", [(1, 1024), (1, 256), (4, 256), (8, 256), (2, 512),
                                         (1, 768), (4, 1024)])
def test_fused_grid_sizes(handle, bps, threads):
    """Every CTA size and CTAs-per-SM setting (clamped to what fits) gives
    the same tree, on a graph that reaches the tail and one that does not."""
    assert B.mst_set_single_schedule(handle, 1, bps, threads) == B.MST_OK
    try:
        for g in (gg.random_connected(30000, 90001, 5 + bps), gg.grid2d(200, 300, threads)):
            check(handle, g.n, g.src, g.dst, g.w)
    finally:
        B.mst_set_single_schedule(handle, 0, 4, 256)


def test_schedule_arg_errors(handle):
    for bad in [(5, 0, 0), (-1, 0, 0), (1, 9, 0), (1, -1, 0), (1, 0, 100), (1, 0, 2048)]:
        assert B.mst_set_single_schedule(handle, *bad) == B.MST_ERR_INVALID_ARG


def test_config1(handle):
    g = gg.config(1)
    check(handle, g.n, g.src, g.dst, g.w)


def test_config2_grid_full(sched):
    g = gg.config(2)
    check(sched, g.n, g.src, g.dst, g.w)


def test_grid_unshuffled(handle):
    g = gg.grid2d(300, 517, 3, shuffle=False)
    check(handle, g.n, g.src, g.dst, g.w)


@pytest.mark.parametrize("scale", [10, 14, 18])
def test_rmat(sched, scale):
    g = gg.rmat(scale, 8, 50 + scale)
    check(sched, g.n, g.src, g.dst, g.w)


@pytest.mark.slow
def test_config3_rmat_full(sched):
    g = gg.config(3)
    check(sched, g.n, g.src, g.dst, g.w)


@pytest.mark.parametrize("name", ["Graph10K_3", "Graph100K_6", "Graph1M_9"])
def test_paper_table1_shapes(handle, name):
    g = gg.paper_table1(name)
    check(handle, g.n, g.src, g.dst, g.w)


def test_float_weights_with_ties(sched):
    handle = sched
    g = gg.random_connected(20000, 60000, 5, weights="f32")
    g.w[:] = np.round(g.w * 64) / 64  # force many ties
    g.w[::7] = np.float32(-0.0)
    g.w[1::7] = np.float32(0.0)
    check(handle, g.n, g.src, g.dst, g.w)


def test_u32_ties_and_multi_edges(handle):
    rng = np.random.default_rng(3)
    n, m = 3000, 40000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)  # self-loops and parallel edges included
    w = rng.integers(0, 5, m).astype(np.uint32)
    check(handle, n, src, dst, w)


def test_increasing_path_deep_chain(sched):
    n = 300000  # every vertex hooks to its left neighbour: depth n-1 chain
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    w = np.arange(1, n, dtype=np.uint32)
    got = check(sched, n, src, dst, w)
    assert len(got) == n - 1
    rev = (n - 1 - np.arange(n - 1)).astype(np.uint32)  # decreasing: chain the other way
    check(sched, n, src, dst, rev)


def test_star_and_cycle(handle):
    n = 5000
    src = np.zeros(n - 1, np.int32)
    dst = np.arange(1, n, dtype=np.int32)
    w = (np.random.default_rng(1).permutation(n - 1) + 1).astype(np.uint32)
    check(handle, n, src, dst, w)
    cs = np.arange(n, dtype=np.int32)
    cd = ((np.arange(n) + 1) % n).astype(np.int32)
    cw = (np.random.default_rng(2).permutation(n) + 1).astype(np.uint32)
    got = check(handle, n, cs, cd, cw)
    assert int(np.argmax(cw)) not in set(got.tolist())


def test_parallel_edges_only(handle):
    k = 999
    src = np.zeros(k, np.int32)
    dst = np.ones(k, np.int32)
    w = (np.random.default_rng(4).permutation(k) + 1).astype(np.uint32)
    assert list(check(handle, 2, src, dst, w)) == [int(np.argmin(w))]


def test_disconnected_and_isolated(sched):
    handle = sched
    a = gg.random_connected(4000, 9000, 1)
    b = gg.random_connected(3000, 7000, 2)
    src = np.concatenate([a.src, b.src + 4000]).astype(np.int32)
    dst = np.concatenate([a.dst, b.dst + 4000]).astype(np.int32)
    w = np.concatenate([a.w, b.w]).astype(np.uint32)  # duplicate weights across parts
    got, status = gpu_solve(handle, 7050, src, dst, w)
    assert np.array_equal(got, oracle.kruskal(7050, src, dst, w))
    assert status == B.MST_ERR_DISCONNECTED


def test_degenerate_sizes(handle):
    z = np.zeros(0, np.int32)
    zw = np.zeros(0, np.uint32)
    for n in (0, 1, 5):
        got, status = gpu_solve(handle, n, z, z, zw)
        assert len(got) == 0
        assert status == (B.MST_ERR_DISCONNECTED if n > 1 else B.MST_OK)
    got, _ = gpu_solve(handle, 3, np.array([1], np.int32), np.array([1], np.int32),
                       np.array([5], np.uint32))  # a self-loop only
    assert len(got) == 0


def test_unaligned_inputs_scalar_path(handle):
    g = gg.random_connected(9000, 30001, 8)
    src, dst, w = to_dev(np.r_[np.int32(0), g.src], np.r_[np.int32(0), g.dst],
                         np.r_[np.uint32(0), g.w])
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = B.mst_solve(handle, g.n, g.m, src.data_ptr() + 4, dst.data_ptr() + 4, w.data_ptr() + 4,
                     out, cnt)
    assert st == B.MST_OK and B.mst_get_status(handle) == B.MST_OK
    got = out[: int(cnt.item())].cpu().numpy()
    assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w))


def test_bad_vertex_and_nan_reported(handle):
    g = gg.random_connected(1000, 3000, 9)
    src = g.src.copy()
    src[5] = 1000  # out of range
    src[6] = -3
    _, status = gpu_solve(handle, g.n, src, g.dst, g.w)
    assert status == B.MST_ERR_INVALID_ARG
    gf = gg.random_connected(1000, 3000, 9, weights="f32")
    gf.w[10] = np.float32("nan")
    _, status = gpu_solve(handle, gf.n, gf.src, gf.dst, gf.w)
    assert status == B.MST_ERR_INVALID_ARG
    # the handle still works afterwards
    check(handle, g.n, g.src, g.dst, g.w)


def test_host_argument_errors(handle):
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_solve(handle, -1, 0, x, x, x, x, c) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve(handle, 4, -2, x, x, x, x, c) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve(handle, 4, 2, None, x, x, x, c) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve(handle, 4, 2, x, x, x, x, None) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve(handle, 0, 2, x, x, x, x, c) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve_ex(handle, 9, 4, 2, x, x, x, x, c) == B.MST_ERR_INVALID_ARG


def test_budget_enforced(lib_built):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    h = B.mst_create(0, 1 << 20)  # 1 MiB budget
    try:
        g = gg.random_connected(100000, 400000, 3)
        s, d, w = to_dev(g.src, g.dst, g.w)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert B.mst_solve(h, g.n, g.m, s, d, w, out, c) == B.MST_ERR_BUDGET
    finally:
        B.mst_destroy(h)


def test_workspace_reuse_and_growth(handle):
    for (n, m, seed) in [(500, 2000, 1), (60000, 200000, 2), (700, 900, 3), (60000, 200000, 2)]:
        g = gg.random_connected(n, m, seed)
        check(handle, g.n, g.src, g.dst, g.w)


def test_deterministic_rounds(sched):
    handle = sched
    g = gg.random_connected(50000, 200000, 11)
    ref = None
    for _ in range(10):
        got, _ = gpu_solve(handle, g.n, g.src, g.dst, g.w)
        stats = B.mst_get_round_stats(handle)
        if ref is None:
            ref = (got, stats)
        assert np.array_equal(got, ref[0]) and stats == ref[1]
    edges, verts = ref[1]
    assert edges[0] == g.m and verts[0] == g.n
    assert edges[-1] == 0 and verts[-1] == 1
    assert all(a > b for a, b in zip(verts, verts[1:]))  # components at least halve... strictly fall
    assert all(2 * b <= a for a, b in zip(verts, verts[1:]))
    assert len(verts) - 1 <= math.ceil(math.log2(g.n))


def test_async_on_side_stream(handle):
    g = gg.random_connected(30000, 120000, 12)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got, status = gpu_solve(handle, g.n, g.src, g.dst, g.w, stream=s)
    assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w))


@pytest.mark.parametrize("pinned", ["none", "inputs", "all"])
@pytest.mark.parametrize("shape", [(20000, 80000, 17), (1024, 1024 * 3 + 1, 5), (300000, 900001, 9)])
def test_host_buffer_solve(sched, pinned, shape):
    """Host buffers: pageable inputs are copied in first; pinned inputs are
    read by the fused kernel in round 0 while it writes the device copy (the
    graph schedule copies them in); pinned outputs are written by the kernel
    directly.  Odd m exercises the ragged last group."""
    n, m, seed = shape
    g = gg.random_connected(n, m, seed)
    pin_in = (lambda t: t.pin_memory()) if pinned != "none" else (lambda t: t)
    pin_out = (lambda t: t.pin_memory()) if pinned == "all" else (lambda t: t)
    hs, hd = pin_in(torch.from_numpy(g.src)), pin_in(torch.from_numpy(g.dst))
    hw = pin_in(torch.from_numpy(g.w.view(np.int32)))
    ho = pin_out(torch.full((g.n - 1,), -1, dtype=torch.int32))
    hc = pin_out(torch.zeros(1, dtype=torch.int64))
    ref = oracle.kruskal(g.n, g.src, g.dst, g.w)
    for _ in range(2):  # twice: the second solve reuses the staging and the copy
        st = B.mst_solve_host(sched, B.MST_W_U32, g.n, g.m, hs, hd, hw, ho, hc)
        assert st == B.MST_OK
        assert np.array_equal(ho[: int(hc.item())].numpy(), ref)


def test_host_buffer_then_replay(handle):
    """A profile replay after a pinned host-buffer solve reads the device copy."""
    g = gg.random_connected(30000, 120000, 31)
    hs, hd = torch.from_numpy(g.src).pin_memory(), torch.from_numpy(g.dst).pin_memory()
    hw = torch.from_numpy(g.w.view(np.int32)).pin_memory()
    ho = torch.full((g.n - 1,), -1, dtype=torch.int32).pin_memory()
    hc = torch.zeros(1, dtype=torch.int64).pin_memory()
    assert B.mst_solve_host(handle, B.MST_W_U32, g.n, g.m, hs, hd, hw, ho, hc) == B.MST_OK
    prof = B.mst_profile_last_solve(handle)
    assert any(p["name"].startswith("k_solve:find0") for p in prof)
    assert np.array_equal(ho[: int(hc.item())].numpy(), oracle.kruskal(g.n, g.src, g.dst, g.w))


def test_profile_replay_matches(handle):
    g = gg.random_connected(50000, 200000, 23)
    s, d, w = to_dev(g.src, g.dst, g.w)  # kept alive: the replay reuses these buffers
    out = torch.full((g.n - 1,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_set_single_schedule(handle, 2, 0) == B.MST_OK
    try:
        assert B.mst_solve(handle, g.n, g.m, s, d, w, out, cnt) == B.MST_OK
        first = out.clone()
        prof = B.mst_profile_last_solve(handle)
        assert torch.equal(first, out)  # the replay writes the same tree again
        names = [p["name"] for p in prof]
        assert "k_find0" in names and "k_compact<R0>" in names and "k_emit" in names
        assert all(p["total_ms"] > 0 and p["launches"] >= 1 for p in prof)
    finally:
        B.mst_set_single_schedule(handle, 0, 0)


def test_fused_phase_log(handle):
    g = gg.random_connected(50000, 200000, 29)
    s, d, w = to_dev(g.src, g.dst, g.w)
    out = torch.full((g.n - 1,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_set_single_schedule(handle, 1, 0) == B.MST_OK
    assert B.mst_solve(handle, g.n, g.m, s, d, w, out, cnt) == B.MST_OK
    prof = B.mst_profile_last_solve(handle)
    rounds = len(B.mst_get_round_stats(handle)[0]) - 1

    def count(kind):
        return sum(p["launches"] for p in prof if p["name"].startswith("k_solve:" + kind))

    assert count("find0") == 1 and count("emit") == 1 and count("init") == 1
    # grid rounds have a hook, compress and compaction phase each; once few
    # components remain, one tail phase finishes the remaining rounds
    assert count("hook") == count("compact") <= rounds
    assert count("compress") >= count("hook")
    assert count("tail") <= 1
    if count("tail") == 0:
        assert count("hook") == rounds
    assert all(p["total_ms"] > 0 for p in prof)
    B.mst_set_single_schedule(handle, 0, 0)
