"""Adjacency-CSR input (mst_solve_csr) against the oracle on the CSR's
entries: the tree's ids are CSR positions."""
import numpy as np
import pytest
import torch

from paper_2005_06913_gb300 import binding as B, graphgen as gg

pytestmark = pytest.mark.gpu


def csr_solve(h, c, flags):
    rp = torch.from_numpy(c.row_ptr).cuda()
    col = torch.from_numpy(c.col).cuda()
    w = torch.from_numpy(c.w.view(np.int32) if c.w.dtype == np.uint32 else c.w).cuda()
    out = torch.full((max(c.n - 1, 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    wt = B.MST_W_F32 if c.w.dtype == np.float32 else B.MST_W_U32
    st = B.mst_solve_csr(h, wt, c.n, c.nnz, rp, col, w, flags, out, cnt)
    assert st == B.MST_OK
    status = B.mst_get_status(h)
    k = int(cnt.item())
    return out[:k].cpu().numpy().astype(np.int64), status


def check(h, c, flags, oracle):
    e = gg.csr_entries(c)
    expect = oracle.kruskal(e.n, e.src, e.dst, e.w)
    got, status = csr_solve(h, c, flags)
    assert np.array_equal(got, expect)
    comps = oracle.components(e.n, e.src, e.dst)
    assert status == (B.MST_OK if comps <= 1 else B.MST_ERR_DISCONNECTED)


GRAPHS = {
    "tiny": lambda: gg.random_connected(3, 3, 1),
    "random-ragged": lambda: gg.random_connected(5003, 20011, 2),
    "random-tail": lambda: gg.random_connected(70001, 250003, 3),
    "grid": lambda: gg.grid2d(300, 517, 4),
    "rmat14": lambda: gg.rmat(14, 8, 5),
    "float-ties": lambda: float_ties(),
}


def float_ties():
    g = gg.random_connected(20000, 80000, 6, weights="f32")
    g.w[:] = np.round(g.w * 64) / 64  # many ties
    g.w[::7] = np.float32(-0.0)
    return g


@pytest.fixture(params=[0, 2], ids=["fused", "graph"])
def sched(request, handle):
    assert B.mst_set_single_schedule(handle, request.param, 0) == B.MST_OK
    yield handle
    B.mst_set_single_schedule(handle, 0, 0)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("flags", [0, B.MST_CSR_SYMMETRIC], ids=["plain", "symmetric"])
def test_symmetric_csr(sched, oracle_mod, name, flags):
    check(sched, gg.to_csr(GRAPHS[name](), symmetric=True), flags, oracle_mod)


def test_one_sided_csr(handle, oracle_mod):
    """Each edge stored once, from its src row: entries of either direction."""
    check(handle, gg.to_csr(gg.random_connected(30000, 120000, 7), symmetric=False), 0,
          oracle_mod)


def test_grid_full_size(handle, oracle_mod):
    """The 1024 x 1024 grid as a symmetric CSR (4.2 M entries, the wide
    automatic shape)."""
    check(handle, gg.to_csr(gg.config(2)), B.MST_CSR_SYMMETRIC, oracle_mod)


def test_disconnected_isolated_loops_parallel(handle, oracle_mod):
    rng = np.random.default_rng(8)
    n, m = 3000, 2500  # sparse: many components, isolated vertices
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    dst[:50] = src[:50]  # self-loops
    src[50:100], dst[50:100] = src[100:150], dst[100:150]  # parallel edges
    w = rng.integers(0, 20, m).astype(np.uint32)
    g = gg.Graph(n, src, dst, w)
    for flags in (0, B.MST_CSR_SYMMETRIC):
        check(handle, gg.to_csr(g), flags, oracle_mod)


def test_no_entries(handle):
    c = gg.CSR(5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    got, status = csr_solve(handle, c, 0)
    assert got.size == 0 and status == B.MST_ERR_DISCONNECTED


@pytest.mark.parametrize("defect", ["first", "last", "decreasing"])
def test_malformed_offsets_reported(handle, defect):
    c = gg.to_csr(gg.random_connected(2000, 8000, 9))
    rp = c.row_ptr.copy()
    if defect == "first":
        rp[0] = 1
    elif defect == "last":
        rp[-1] -= 1
    else:
        rp[1000] = rp[1001] + 1
    bad = gg.CSR(c.n, rp, c.col, c.w)
    _, status = csr_solve(handle, bad, 0)
    assert status == B.MST_ERR_INVALID_ARG
    got, status = csr_solve(handle, c, 0)  # the handle stays usable
    assert status == B.MST_OK and got.size == c.n - 1


def test_host_argument_errors(handle):
    bad = B.MST_ERR_INVALID_ARG
    rp = torch.zeros(4, dtype=torch.int64, device="cuda")
    col = torch.zeros(2, dtype=torch.int32, device="cuda")
    w = torch.zeros(2, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert B.mst_solve_csr(handle, 0, 3, 2, rp, col, w, 2, out, cnt) == bad  # unknown flag
    assert B.mst_solve_csr(handle, 5, 3, 2, rp, col, w, 0, out, cnt) == bad  # weight type
    assert B.mst_solve_csr(handle, 0, 3, 2, None, col, w, 0, out, cnt) == bad  # no offsets
    assert B.mst_solve_csr(handle, 0, 3, -1, rp, col, w, 0, out, cnt) == bad
    assert B.mst_solve_csr(handle, 0, 3, 1 << 31, rp, col, w, 0, out, cnt) == bad
