"""Bounded waits of the fused schedule, and fused solves from several
handles and streams at once.

The fused kernel's CTAs meet at grid barriers whose waits are bounded.  A
short wait limit (mst_set_wait_limit) makes them run out on purpose: the
solve must then report MST_ERR_TIMEOUT with no ids written, return promptly,
and leave the handle usable, so that the next solve with the default limit
gives the oracle's tree.  No GPU hang or fault is involved: the wait simply
gives up early.

Fused solves queued on two handles and two streams at the same time must
each give the oracle's tree: the library orders fused grids per device.
"""
import numpy as np
import pytest
import torch

from conftest import to_dev
from paper_2005_06913_gb300 import binding as B
from paper_2005_06913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _buffers(g):
    s, d, w = to_dev(g.src, g.dst, g.w)
    out = torch.full((max(g.n - 1, 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    return s, d, w, out, cnt


def _queue(h, g, bufs, stream=None):
    s, d, w, out, cnt = bufs
    wt = B.MST_W_F32 if g.w.dtype == np.float32 else B.MST_W_U32
    assert B.mst_solve_ex(h, wt, g.n, g.m, s, d, w, out, cnt, stream) == B.MST_OK
    return out, cnt


def _solve(h, g):
    bufs = _buffers(g)
    return _queue(h, g, bufs)


@pytest.mark.parametrize("shape", ["256-thread CTAs", "1024-thread CTAs"])
def test_injected_wait_timeout_then_recovery(handle, oracle_mod, shape):
    # the default schedule takes 1024-thread CTAs above 600,000 edges
    g = (gg.random_connected(4096, 32768, 901) if shape.startswith("256")
         else gg.random_connected(200000, 700000, 902))
    want = oracle_mod.kruskal(g.n, g.src, g.dst, g.w)
    assert B.mst_set_wait_limit(handle, 1) == B.MST_OK
    seen = []
    try:
        for _ in range(5):
            out, cnt = _solve(handle, g)
            st = B.mst_get_status(handle)
            seen.append(st)
            if st == B.MST_ERR_TIMEOUT:
                assert int(cnt.item()) == 0
            else:  # every barrier happened to complete within the limit
                assert st == B.MST_OK
                got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
                assert np.array_equal(got, want)
    finally:
        assert B.mst_set_wait_limit(handle, 0) == B.MST_OK
    assert B.MST_ERR_TIMEOUT in seen, seen
    out, cnt = _solve(handle, g)
    assert B.mst_get_status(handle) == B.MST_OK
    assert np.array_equal(out[: int(cnt.item())].cpu().numpy().astype(np.int64), want)


def test_concurrent_fused_solves_on_two_handles(lib_built, oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    graphs = [gg.random_connected(5000 + 1000 * i, 30000 + 8000 * i, 910 + i) for i in range(4)]
    graphs += [gg.random_connected(150000, 650000, 920), gg.grid2d(500, 500, 921),
               gg.random_connected(120000, 620000, 922, weights="f32"),
               gg.random_connected(9000, 40000, 923, weights="f32")]
    h1, h2 = B.mst_create(0, 0), B.mst_create(0, 0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        big = max(graphs, key=lambda x: x.m)
        for h in (h1, h2):  # size the workspaces first
            _solve(h, big)
        # every buffer is made and filled before any solve is queued, so the
        # solves on the two side streams race only with each other
        runs = []
        for rep in range(3):
            for i, g in enumerate(graphs):
                h, s = (h1, s1) if (i + rep) % 2 == 0 else (h2, s2)
                runs.append((g, h, s, _buffers(g)))
        torch.cuda.synchronize()
        for g, h, s, bufs in runs:
            _queue(h, g, bufs, s)
        torch.cuda.synchronize()
        for g, h, s, (_, _, _, out, cnt) in runs:
            got = out[: int(cnt.item())].cpu().numpy().astype(np.int64)
            assert np.array_equal(got, oracle_mod.kruskal(g.n, g.src, g.dst, g.w))
        assert B.mst_get_status(h1, s1) == B.MST_OK
        assert B.mst_get_status(h2, s2) == B.MST_OK
    finally:
        B.mst_destroy(h1)
        B.mst_destroy(h2)
