"""Continuous-batching server: every request's tree equals the oracle's for
that graph alone while other requests are queued and in flight; admission
respects the memory budget."""
import time

import numpy as np
import pytest
import torch

import oracle
from conftest import to_dev
from paper_2005_06913_gb300 import binding as B
from paper_2005_06913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def submit_all(h, graphs, gap_s=0.0):
    reqs = []
    for g in graphs:
        s, d, w = to_dev(g.src, g.dst, g.w)
        out = torch.full((max(g.n - 1, 1),), -5, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -5, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        wt = B.MST_W_F32 if g.w.dtype == np.float32 else B.MST_W_U32
        st, t = B.mst_submit(h, wt, g.n, g.m, s, d, w, out, cnt)
        assert st == B.MST_OK
        reqs.append((t, g, out, cnt, (s, d, w)))
        if gap_s:
            time.sleep(gap_s)
    return reqs


def wait_all(h, reqs, timeout_s=120):
    res = {}
    t0 = time.time()
    while len(res) < len(reqs):
        assert time.time() - t0 < timeout_s, "server did not finish"
        for t, *_ in reqs:
            if t in res:
                continue
            st, done, lat = B.mst_poll(h, t)
            if done:
                res[t] = (st, lat)
        time.sleep(0.001)
    return res


def test_serving_mix_matches_oracle(lib_built):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pool = gg.serving_pool(60, 64, 30000, 6, 21)
    graphs = [pool.graph(i) for i in range(pool.G)]
    h = B.mst_create(0, 0)
    try:
        assert B.mst_server_start(h, 3, 16) == B.MST_OK
        reqs = submit_all(h, graphs, gap_s=0.0005)
        res = wait_all(h, reqs)
        assert B.mst_server_drain(h) == B.MST_OK
        for t, g, out, cnt, _ in reqs:
            st, lat = res[t]
            assert st == B.MST_OK and lat > 0
            got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
            assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w))
        # alone == in the mix: a plain single solve of each graph gives the same ids
        for t, g, out, cnt, (s, d, w) in reqs[:10]:
            ids, _ = B.solve(h, g.n, s, d, w)
            assert np.array_equal(ids.cpu().numpy(), out[: int(cnt.item())].cpu().numpy())
    finally:
        B.mst_server_stop(h)
        B.mst_destroy(h)


def test_serving_budget_admission(lib_built):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    small = [gg.random_connected(2000, 6000, i, weights="f32") for i in range(12)]
    big = gg.random_connected(200000, 600000, 99, weights="f32")
    h = B.mst_create(0, 8 << 20)  # 8 MiB: the big request can never be admitted
    try:
        assert B.mst_server_start(h, 2, 4) == B.MST_OK
        reqs = submit_all(h, small[:6] + [big] + small[6:])
        res = wait_all(h, reqs)
        for t, g, out, cnt, _ in reqs:
            st, _ = res[t]
            if g is big:
                assert st == B.MST_ERR_BUDGET
            else:
                assert st == B.MST_OK
                got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
                assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w))
    finally:
        B.mst_server_stop(h)
        B.mst_destroy(h)


def test_server_lifecycle_errors(lib_built):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    h = B.mst_create(0, 0)
    try:
        assert B.mst_submit(h, 0, 3, 0, None, None, None, None, 0)[0] != B.MST_OK
        assert B.mst_server_start(h, 0, 4) == B.MST_ERR_INVALID_ARG
        assert B.mst_server_start(h, 2, 4) == B.MST_OK
        assert B.mst_server_start(h, 2, 4) == B.MST_ERR_INVALID_ARG
        assert B.mst_poll(h, 12345)[0] == B.MST_ERR_INVALID_ARG
        assert B.mst_server_stop(h) == B.MST_OK
        assert B.mst_server_stop(h) == B.MST_ERR_INVALID_ARG
    finally:
        B.mst_destroy(h)


def test_serving_large_requests_use_fused_path(lib_built):
    """Requests above the batching threshold are solved alone by the fused
    multi-CTA kernel on a slot while other slots serve batches: two large ones
    back to back (both slots fused at once), a larger one after a smaller one
    (the slot's workspace grows), a disconnected large one (a forest)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    small = [gg.random_connected(500 + 300 * i, 3000 + 900 * i, 40 + i, weights="f32")
             for i in range(10)]
    big1 = gg.random_connected(60000, 180000, 7, weights="f32")
    big2 = gg.grid2d(400, 400, 8)
    big3 = gg.random_connected(150000, 450000, 9, weights="f32")
    a = gg.random_connected(50000, 150000, 10)
    b = gg.random_connected(30000, 90000, 11)
    forest = gg.Graph(a.n + b.n, np.r_[a.src, b.src + a.n].astype(np.int32),
                      np.r_[a.dst, b.dst + a.n].astype(np.int32), np.r_[a.w, b.w], "two parts")
    graphs = small[:3] + [big1, big2] + small[3:6] + [big3] + small[6:8] + [forest] + small[8:]
    h = B.mst_create(0, 0)
    try:
        assert B.mst_server_start(h, 2, 8) == B.MST_OK
        reqs = submit_all(h, graphs)
        res = wait_all(h, reqs)
        assert B.mst_server_drain(h) == B.MST_OK
        for t, g, out, cnt, _ in reqs:
            st, lat = res[t]
            # a forest reports what mst_solve_ex reports for it alone
            want = B.MST_ERR_DISCONNECTED if g is forest else B.MST_OK
            assert st == want and lat > 0, (g.name, B.mst_status_string(st))
            got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
            assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w)), g.name
    finally:
        B.mst_server_stop(h)
        B.mst_destroy(h)


def test_serving_bad_request_does_not_poison_its_batch(lib_built):
    """Requests batched together each get their own status: one with a NaN
    weight and one with an out-of-range vertex id report MST_ERR_INVALID_ARG,
    a forest reports MST_ERR_DISCONNECTED, and every other request of the
    same batches returns MST_OK with the oracle's tree."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    graphs = [gg.random_connected(800 + 97 * i, 2400 + 300 * i, 300 + i, weights="f32")
              for i in range(24)]
    nan = graphs[5]
    nan.w = nan.w.copy()
    nan.w[7] = np.float32("nan")
    badv = graphs[11]
    badv.src = badv.src.copy()
    badv.src[3] = badv.n + 1
    a = gg.random_connected(900, 2700, 350, weights="f32")
    b = gg.random_connected(600, 1800, 351, weights="f32")
    forest = gg.Graph(a.n + b.n, np.r_[a.src, b.src + a.n].astype(np.int32),
                      np.r_[a.dst, b.dst + a.n].astype(np.int32), np.r_[a.w, b.w], "forest")
    graphs[17] = forest
    h = B.mst_create(0, 0)
    try:
        # one stream and a large max_batch: the requests share batches
        assert B.mst_server_start(h, 1, 64) == B.MST_OK
        reqs = submit_all(h, graphs)
        res = wait_all(h, reqs)
        assert B.mst_server_drain(h) == B.MST_OK
        for t, g, out, cnt, _ in reqs:
            st, _ = res[t]
            if g is nan or g is badv:
                assert st == B.MST_ERR_INVALID_ARG, B.mst_status_string(st)
                continue
            want = B.MST_ERR_DISCONNECTED if g is forest else B.MST_OK
            assert st == want, (g.name, B.mst_status_string(st))
            got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
            assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w)), g.name
    finally:
        B.mst_server_stop(h)
        B.mst_destroy(h)


def test_serving_lane_unions(lib_built):
    """Requests for the fused lane that queue up behind one another are solved
    together as one union graph: each must still get the oracle's tree and
    its own status (a NaN weight and an out-of-range vertex id in two of
    them, a forest in a third), with uint32 and float32 requests in separate
    unions."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    graphs = []
    for i in range(14):
        wts = "f32" if i % 3 else "u32"
        graphs.append(gg.random_connected(20000 + 3000 * i, 60000 + 9000 * i, 500 + i,
                                          weights=wts))
    nan = graphs[4]  # f32
    nan.w = nan.w.copy()
    nan.w[11] = np.float32("nan")
    badv = graphs[7]
    badv.dst = badv.dst.copy()
    badv.dst[5] = badv.n + 9
    a = gg.random_connected(30000, 90000, 520, weights="f32")
    b = gg.random_connected(12000, 36000, 521, weights="f32")
    forest = gg.Graph(a.n + b.n + 7, np.r_[a.src, b.src + a.n].astype(np.int32),
                      np.r_[a.dst, b.dst + a.n].astype(np.int32), np.r_[a.w, b.w], "forest")
    graphs.insert(9, forest)
    h = B.mst_create(0, 0)
    try:
        assert B.mst_server_start(h, 1, 64) == B.MST_OK
        reqs = submit_all(h, graphs)
        res = wait_all(h, reqs)
        assert B.mst_server_drain(h) == B.MST_OK
        for t, g, out, cnt, _ in reqs:
            st, _ = res[t]
            got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
            if g is nan or g is badv:
                assert st == B.MST_ERR_INVALID_ARG, B.mst_status_string(st)
                # the same tree as the graph alone (a bad edge ignored, a NaN
                # weight sorting last), which the oracle does not define
                s2, d2, w2 = to_dev(g.src, g.dst, g.w)
                ids, st2 = B.solve(h, g.n, s2, d2, w2, check=False)
                assert st2 == B.MST_ERR_INVALID_ARG
                assert np.array_equal(got, ids.cpu().numpy().astype(np.int64))
                continue
            if g is forest:
                assert st == B.MST_ERR_DISCONNECTED, B.mst_status_string(st)
                assert int(cnt.item()) == g.n - oracle.components(g.n, g.src, g.dst)
            else:
                assert st == B.MST_OK, (g.name, B.mst_status_string(st))
            assert np.array_equal(got, oracle.kruskal(g.n, g.src, g.dst, g.w)), g.name
    finally:
        B.mst_server_stop(h)
        B.mst_destroy(h)
