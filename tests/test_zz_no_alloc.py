"""mst_solve_noalloc: the allocation-free entry point for callers that
cannot allocate device memory when they solve (inside a stream capture, in
a host that reserves its device memory up front).  It must return exactly
what the regular entry point returns, on two calls in a row (the shared
scratch keeps the previous call's contents), and reject graphs beyond its
fixed scratch before queuing anything.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from conftest import to_dev
from paper_2005_06913_gb300 import binding as B
from paper_2005_06913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def regular(h, g):
    s, d, w = to_dev(g.src, g.dst, g.w)
    out = torch.full((max(g.n - 1, 1),), -3, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    wt = B.MST_W_F32 if g.w.dtype == np.float32 else B.MST_W_U32
    assert B.mst_solve_ex(h, wt, g.n, g.m, s, d, w, out, cnt) == B.MST_OK
    assert B.mst_get_status(h) in (B.MST_OK, B.MST_ERR_DISCONNECTED)
    return out[: int(cnt.item())].cpu().numpy()


def noalloc(g):
    s, d, w = to_dev(g.src, g.dst, g.w)
    out = torch.full((max(g.n - 1, 1),), -3, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    wt = B.MST_W_F32 if g.w.dtype == np.float32 else B.MST_W_U32
    assert B.mst_solve_noalloc(wt, g.n, g.m, s, d, w, out, cnt, st_dev) == B.MST_OK
    torch.cuda.synchronize()
    assert int(st_dev.item()) in (B.MST_OK, B.MST_ERR_DISCONNECTED)
    return out[: int(cnt.item())].cpu().numpy()


def test_noalloc_matches_regular_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2005_06913_gb300 import build
    build.build()
    h = B.mst_create(0, 0)
    try:
        # two calls in a row: a large graph (scratch in global memory), then a
        # smaller one with float weights, which must not see the first's state
        g1 = gg.random_connected(60000, 250000, 101)
        g2 = gg.random_connected(3000, 12000, 102, weights="f32")
        r1, r2 = regular(h, g1), regular(h, g2)
        a1, a2 = noalloc(g1), noalloc(g2)
        assert np.array_equal(a1, r1)  # integer ids: exact equality is the tolerance
        assert np.array_equal(a2, r2)
        assert np.array_equal(noalloc(g1), r1)  # and back again
    finally:
        B.mst_destroy(h)


def test_noalloc_rejects_oversize_without_launch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_solve_noalloc(B.MST_W_U32, 65537, 10, x, x, x, x, c) == B.MST_ERR_BUDGET
    assert B.mst_solve_noalloc(B.MST_W_U32, 100, 262145, x, x, x, x, c) == B.MST_ERR_BUDGET
    assert B.mst_solve_noalloc(B.MST_W_U32, -1, 0, x, x, x, x, c) == B.MST_ERR_INVALID_ARG
