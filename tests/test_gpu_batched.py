"""Batched solver (one persistent launch for many graphs) vs the CPU oracle.

Every graph's ascending edge ids must equal the oracle's for that graph
alone, bit for bit, under every schedule (CTA per graph; warps for small
graphs) and block size.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from conftest import to_dev
from paper_2005_06913_gb300 import binding as B
from paper_2005_06913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def run_batch(h, b, check_all=True, sample=None, seed=0):
    vo, eo, s, d, w = to_dev(b.vtx_off, b.edge_off, b.src, b.dst, b.w)
    tn, tm = int(b.vtx_off[-1]), int(b.edge_off[-1])
    out = torch.full((max(tn, 1),), -9, dtype=torch.int32, device="cuda")
    cnt = torch.full((max(b.G, 1),), -9, dtype=torch.int64, device="cuda")
    wt = B.MST_W_F32 if b.w.dtype == np.float32 else B.MST_W_U32
    st = B.mst_solve_batched(h, wt, b.G, vo, eo, tn, tm, s, d, w, out, cnt)
    assert st == B.MST_OK, B.mst_status_string(st)
    status = B.mst_get_status(h)
    assert status in (B.MST_OK, B.MST_ERR_DISCONNECTED), B.mst_status_string(status)
    out_h, cnt_h = out.cpu().numpy(), cnt.cpu().numpy()
    gs = range(b.G)
    if sample is not None and sample < b.G:
        gs = np.random.default_rng(seed).choice(b.G, sample, replace=False)
    for g in gs:
        gr = b.graph(int(g))
        got = out_h[b.vtx_off[g]: b.vtx_off[g] + cnt_h[g]].astype(np.int64)
        expect = oracle.kruskal(gr.n, gr.src, gr.dst, gr.w)
        assert np.array_equal(got, expect), f"graph {g} (n={gr.n}, m={gr.m})"
    return status, cnt_h


@pytest.mark.parametrize("schedule,threads", [(1, 128), (1, 256), (1, 512), (1, 1024),
                                              (2, 256), (2, 512), (0, 0)])
def test_batch_schedules(handle, schedule, threads):
    b = gg.batched(96, 8, 6000, 8, 1234)
    assert B.mst_set_batched_schedule(handle, schedule, threads) == B.MST_OK
    try:
        status, _ = run_batch(handle, b)
        assert status == B.MST_OK
    finally:
        B.mst_set_batched_schedule(handle, 0, 0)


def test_batch_float_weights_with_ties(handle):
    b = gg.batched(64, 16, 3000, 6, 77, weights="f32")
    b.w[:] = np.round(b.w * 32) / 32
    status, _ = run_batch(handle, b)
    assert status == B.MST_OK


def test_batch_large_graphs_global_memory(handle):
    b = gg.batched(12, 40000, 150000, 8, 99)  # too big for shared memory
    status, _ = run_batch(handle, b)
    assert status == B.MST_OK


def test_batch_degenerate_graphs(handle):
    parts = [gg.random_connected(50, 200, 1), gg.random_connected(1, 0, 2),
             gg.random_connected(0, 0, 3), gg.random_connected(2, 1, 4)]
    # a graph with self-loops and parallel edges, and a disconnected one
    rng = np.random.default_rng(5)
    parts.append(gg.Graph(300, rng.integers(0, 300, 900).astype(np.int32),
                          rng.integers(0, 300, 900).astype(np.int32),
                          rng.integers(0, 4, 900).astype(np.uint32)))
    a, c = gg.random_connected(40, 60, 6), gg.random_connected(30, 50, 7)
    parts.append(gg.Graph(75, np.r_[a.src, c.src + 40].astype(np.int32),
                          np.r_[a.dst, c.dst + 40].astype(np.int32),
                          np.r_[a.w, c.w].astype(np.uint32)))
    vo = np.r_[0, np.cumsum([p.n for p in parts])].astype(np.int64)
    eo = np.r_[0, np.cumsum([p.m for p in parts])].astype(np.int64)
    b = gg.Batch(vo, eo, np.concatenate([p.src for p in parts]).astype(np.int32),
                 np.concatenate([p.dst for p in parts]).astype(np.int32),
                 np.concatenate([p.w for p in parts]).astype(np.uint32))
    for sched in (1, 2):
        B.mst_set_batched_schedule(handle, sched, 0)
        status, cnt = run_batch(handle, b)
        assert status == B.MST_ERR_DISCONNECTED
        assert cnt[2] == 0 and cnt[1] == 0
    B.mst_set_batched_schedule(handle, 0, 0)


def test_batch_equals_single_solves(handle):
    b = gg.batched(20, 100, 20000, 8, 31)
    _, cnt = run_batch(handle, b, check_all=False, sample=0)
    vo, eo, s, d, w = to_dev(b.vtx_off, b.edge_off, b.src, b.dst, b.w)
    out = torch.full((int(b.vtx_off[-1]),), -9, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(b.G, dtype=torch.int64, device="cuda")
    B.mst_solve_batched(handle, B.MST_W_U32, b.G, vo, eo, int(b.vtx_off[-1]), int(b.edge_off[-1]),
                        s, d, w, out, cnt)
    out_h, cnt_h = out.cpu().numpy(), cnt.cpu().numpy()
    h2 = B.mst_create(0, 0)
    try:
        for g in range(b.G):
            gr = b.graph(g)
            ss, dd, ww = to_dev(gr.src, gr.dst, gr.w)
            ids, st = B.solve(h2, gr.n, ss, dd, ww)
            assert st == B.MST_OK
            assert np.array_equal(ids.cpu().numpy(), out_h[b.vtx_off[g]: b.vtx_off[g] + cnt_h[g]])
    finally:
        B.mst_destroy(h2)


def test_batch_bad_offsets_reported(handle):
    b = gg.batched(8, 64, 500, 8, 3)
    vo = b.vtx_off.copy()
    vo[3], vo[4] = vo[4], vo[3]  # not monotone
    vo_d, eo_d, s, d, w = to_dev(vo, b.edge_off, b.src, b.dst, b.w)
    out = torch.zeros(int(vo[-1]), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(b.G, dtype=torch.int64, device="cuda")
    st = B.mst_solve_batched(handle, B.MST_W_U32, b.G, vo_d, eo_d, int(vo[-1]), int(b.edge_off[-1]),
                             s, d, w, out, cnt)
    assert st == B.MST_OK
    assert B.mst_get_status(handle) == B.MST_ERR_INVALID_ARG
    # the handle recovers
    assert run_batch(handle, b)[0] == B.MST_OK


def test_batch_host_argument_errors(handle):
    x = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert B.mst_solve_batched(handle, 0, -1, x, x, 0, 0, x, x, x, x, x) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve_batched(handle, 0, 2, None, x, 4, 4, x, x, x, x, x) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve_batched(handle, 5, 2, x, x, 4, 4, x, x, x, x, x) == B.MST_ERR_INVALID_ARG
    assert B.mst_solve_batched(handle, 0, 0, None, None, 0, 0, None, None, None, None, None) == B.MST_OK


def test_autotune_cache_roundtrip(handle, tmp_path):
    b = gg.batched(64, 64, 4096, 8, 11)
    vo, eo, s, d, w = to_dev(b.vtx_off, b.edge_off, b.src, b.dst, b.w)
    tn, tm = int(b.vtx_off[-1]), int(b.edge_off[-1])
    out = torch.zeros(tn, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(b.G, dtype=torch.int64, device="cuda")
    path = str(tmp_path / "tune.json")
    h = B.mst_create(0, 0)
    try:
        assert B.mst_autotune_batched(h, 0, b.G, vo, eo, tn, tm, s, d, w, out, cnt, path) == B.MST_OK
        data = json.load(open(path))
        assert data["mst_batched_autotune"] and "threads" in data["mst_batched_autotune"][0]
        status, _ = run_batch(h, b)  # the tuned schedule is correct too
        assert status == B.MST_OK
    finally:
        B.mst_destroy(h)
    h = B.mst_create(0, 0)  # a new handle loads the cache instead of timing
    try:
        assert B.mst_autotune_batched(h, 0, b.G, vo, eo, tn, tm, s, d, w, out, cnt, path) == B.MST_OK
        assert run_batch(h, b)[0] == B.MST_OK
    finally:
        B.mst_destroy(h)


@pytest.mark.slow
def test_config4_full_batch_sampled(handle):
    b = gg.config(4)
    status, cnt = run_batch(handle, b, sample=300, seed=4)
    assert status == B.MST_OK
    assert np.array_equal(cnt, np.diff(b.vtx_off) - 1)  # every graph is connected


def test_batch_per_graph_status(handle):
    """A NaN weight or an out-of-range vertex id in one graph, and a forest in
    another, are reported for those graphs only: their batch-mates return
    MST_OK and the oracle's trees, and the combined status is the union."""
    b = gg.batched(40, 64, 4000, 6, 4242, weights="f32")
    nan_g, bad_g, forest_g = 3, 17, 29
    w = b.w.copy()
    w[b.edge_off[nan_g] + 5] = np.float32("nan")
    src = b.src.copy()
    src[b.edge_off[bad_g] + 2] = int(b.vtx_off[bad_g + 1] - b.vtx_off[bad_g]) + 3
    # graph forest_g: every edge end at its last vertex moves to vertex 0 (or
    # 1, never making a self-loop), which leaves that vertex isolated and the
    # graph a forest of two trees
    e0, e1 = int(b.edge_off[forest_g]), int(b.edge_off[forest_g + 1])
    n_f = int(b.vtx_off[forest_g + 1] - b.vtx_off[forest_g])
    dst = b.dst.copy()
    iso = n_f - 1
    for e in range(e0, e1):
        if src[e] == iso:
            src[e] = 0 if dst[e] != 0 else 1
        if dst[e] == iso:
            dst[e] = 0 if src[e] != 0 else 1
    b2 = gg.Batch(b.vtx_off, b.edge_off, src, dst, w, "per-graph status")
    vo, eo, s, d, ww = to_dev(b2.vtx_off, b2.edge_off, b2.src, b2.dst, b2.w)
    tn, tm = int(b2.vtx_off[-1]), int(b2.edge_off[-1])
    out = torch.full((tn,), -9, dtype=torch.int32, device="cuda")
    cnt = torch.full((b2.G,), -9, dtype=torch.int64, device="cuda")
    assert B.mst_solve_batched(handle, B.MST_W_F32, b2.G, vo, eo, tn, tm, s, d, ww, out,
                               cnt) == B.MST_OK
    assert B.mst_get_status(handle) == B.MST_ERR_INVALID_ARG  # the union of all graphs
    st, per = B.mst_get_batched_status(handle, b2.G)
    assert st == B.MST_OK
    out_h, cnt_h = out.cpu().numpy(), cnt.cpu().numpy()
    for g in range(b2.G):
        if g in (nan_g, bad_g):
            assert per[g] == B.MST_ERR_INVALID_ARG, (g, per[g])
            continue
        gr = b2.graph(g)
        assert per[g] == (B.MST_ERR_DISCONNECTED if g == forest_g else B.MST_OK), (g, per[g])
        got = out_h[b2.vtx_off[g]: b2.vtx_off[g] + cnt_h[g]].astype(np.int64)
        assert np.array_equal(got, oracle.kruskal(gr.n, gr.src, gr.dst, gr.w)), g
    # after a single-graph solve there is no batch to report on
    g0 = b2.graph(0)
    s0, d0, w0 = to_dev(g0.src, g0.dst, g0.w)
    B.solve(handle, g0.n, s0, d0, w0)
    assert B.mst_get_batched_status(handle, b2.G)[0] == B.MST_ERR_INVALID_ARG


def _multigraph(n, m, seed, weights):
    """A connected multigraph: a random spanning tree plus m - (n - 1) edges
    drawn among few vertex groups, so that after a round or two almost every
    live edge is parallel to others between the same components; weights
    with heavy ties."""
    rng = np.random.default_rng(seed)
    tv = np.arange(1, n)
    tu = rng.integers(0, tv)
    k = m - (n - 1)
    groups = rng.integers(0, 6, n)
    a = rng.integers(0, n, k)
    b = rng.integers(0, n, k)
    b = np.where(groups[a] == groups[b], (b + 1) % n, b)  # cross-group extra edges
    src = np.r_[tv, a].astype(np.int32)
    dst = np.r_[tu, b].astype(np.int32)
    if weights == "f32":
        w = (rng.integers(0, 16, m) / 16.0).astype(np.float32)
    else:
        w = rng.integers(0, 40, m).astype(np.uint32)
    return gg.Graph(n, src, dst, w)


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
@pytest.mark.parametrize("weights", ["u32", "f32"])
def test_batch_merging_tail(handle, threads, weights):
    """Graphs whose rounds reach few components while most live edges are
    parallel: the block team's merging tail keeps the lightest record per
    component pair, ties broken by edge id.  Also a forest with isolated
    vertices and graphs in global and in shared memory."""
    parts = [_multigraph(n, 6 * n, 600 + n, weights) for n in (300, 1500, 5000, 30000)]
    a, c = _multigraph(2000, 9000, 701, weights), _multigraph(900, 4000, 702, weights)
    parts.append(gg.Graph(2900 + 50, np.r_[a.src, c.src + 2000].astype(np.int32),
                          np.r_[a.dst, c.dst + 2000].astype(np.int32), np.r_[a.w, c.w]))
    vo = np.r_[0, np.cumsum([p.n for p in parts])].astype(np.int64)
    eo = np.r_[0, np.cumsum([p.m for p in parts])].astype(np.int64)
    wdt = np.float32 if weights == "f32" else np.uint32
    b = gg.Batch(vo, eo, np.concatenate([p.src for p in parts]).astype(np.int32),
                 np.concatenate([p.dst for p in parts]).astype(np.int32),
                 np.concatenate([p.w for p in parts]).astype(wdt))
    B.mst_set_batched_schedule(handle, 1, threads)
    try:
        status, cnt = run_batch(handle, b)
    finally:
        B.mst_set_batched_schedule(handle, 0, 0)
    assert status == B.MST_ERR_DISCONNECTED  # the last graph is a forest
    st, per = B.mst_get_batched_status(handle, b.G)
    assert st == B.MST_OK and per[:-1] == [B.MST_OK] * (b.G - 1)
    assert per[-1] == B.MST_ERR_DISCONNECTED and cnt[-1] == 2950 - 52
