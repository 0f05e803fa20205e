"""Pins for the CPU oracle (no GPU).

The paper prints no worked example with numbers, so the oracle is pinned by
what mathematics fixes: exhaustive brute force on tiny graphs, closed-form
special cases, small instances of the paper's own proof diagrams (golden
fixtures), library MST routines, and MST certificates (cycle and cut
properties).  Kruskal, the Section 2.1 Boruvka (with and without its
"covered" optimisation) and Prim must all return the same edge set.
"""
import math
import os
from itertools import permutations

import numpy as np
import pytest

from brute import brute_msf
from paper_2005_06913_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_oracles(orc, n, src, dst, w):
    k = orc.kruskal(n, src, dst, w)
    b1, _ = orc.boruvka(n, src, dst, w, covered=True)
    b0, _ = orc.boruvka(n, src, dst, w, covered=False)
    p = orc.prim(n, src, dst, w)
    return k, b1, b0, p


def assert_all(orc, n, src, dst, w, expect):
    expect = np.asarray(sorted(expect), dtype=np.int64)
    for name, got in zip(("kruskal", "boruvka", "boruvka-unopt", "prim"),
                         all_oracles(orc, n, src, dst, w)):
        assert np.array_equal(got, expect), (name, got, expect)
    assert orc.check_cycle_property(n, src, dst, w, expect) == 0
    if n <= 2000:
        assert orc.check_cut_property(n, src, dst, w, expect) == 0


def arrays(edges, wdtype=np.uint32):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    w = np.array([e[2] for e in edges], wdtype)
    return src, dst, w


# ---------------------------------------------------------------- golden files

def load_golden(path):
    n, edges, mst = None, [], None
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        if f[0] == "n":
            n = int(f[1])
        elif f[0] == "e":
            assert int(f[1]) == len(edges)
            edges.append((int(f[2]), int(f[3]), int(f[4])))
        elif f[0] == "mst":
            mst = [int(x) for x in f[1:]]
    return n, edges, mst


@pytest.mark.parametrize("name", sorted(os.listdir(GOLDEN)))
def test_golden_fixture(oracle_mod, name):
    n, edges, mst = load_golden(os.path.join(GOLDEN, name))
    src, dst, w = arrays(edges)
    assert brute_msf(n, src, dst, w) == sorted(mst)
    assert_all(oracle_mod, n, src, dst, w, mst)


# ------------------------------------------------------------- brute force

def random_small(rng, n, m, wmax=None, loops=False, f32=False):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if not loops:
        dst = np.where(src == dst, (dst + 1) % n, dst).astype(np.int32)
    if f32:
        w = (rng.integers(1, wmax or 1000, m) / 8.0).astype(np.float32)
    elif wmax is None:
        w = (rng.permutation(m) + 1).astype(np.uint32)
    else:
        w = rng.integers(1, wmax + 1, m).astype(np.uint32)
    return src, dst, w


@pytest.mark.parametrize("seed", range(60))
def test_brute_force_distinct(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 8))
    m = int(rng.integers(1, 13))
    src, dst, w = random_small(rng, n, m, loops=seed % 3 == 0)
    assert_all(oracle_mod, n, src, dst, w, brute_msf(n, src, dst, w))


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_ties(oracle_mod, seed):
    """Many equal weights and parallel edges: the id tie-break decides."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 7))
    m = int(rng.integers(1, 12))
    src, dst, w = random_small(rng, n, m, wmax=3, loops=True)
    assert_all(oracle_mod, n, src, dst, w, brute_msf(n, src, dst, w))


@pytest.mark.parametrize("seed", range(20))
def test_brute_force_float(oracle_mod, seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(2, 7))
    m = int(rng.integers(1, 12))
    src, dst, w = random_small(rng, n, m, wmax=12, f32=True)
    if seed % 4 == 0:
        w[0] = np.float32(-0.0)
        w[-1] = np.float32(0.0)  # -0 and +0 compare equal: tie broken by id
    assert_all(oracle_mod, n, src, dst, w, brute_msf(n, src, dst, w))


def test_exhaustive_k4(oracle_mod):
    """All 720 weight orders of K4, each against brute force."""
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    src = np.array([p[0] for p in pairs], np.int32)
    dst = np.array([p[1] for p in pairs], np.int32)
    for perm in permutations(range(1, 7)):
        w = np.array(perm, np.uint32)
        expect = brute_msf(4, src, dst, w)
        for got in all_oracles(oracle_mod, 4, src, dst, w):
            assert list(got) == expect, (perm, got, expect)


def test_exhaustive_five_edges(oracle_mod):
    """All 120 weight orders of a 4-cycle with one chord."""
    pairs = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]
    src = np.array([p[0] for p in pairs], np.int32)
    dst = np.array([p[1] for p in pairs], np.int32)
    for perm in permutations(range(1, 6)):
        w = np.array(perm, np.uint32)
        expect = brute_msf(4, src, dst, w)
        for got in all_oracles(oracle_mod, 4, src, dst, w):
            assert list(got) == expect


# ------------------------------------------------------------- closed forms

def test_tree_input_keeps_every_edge(oracle_mod):
    g = gg.random_connected(500, 499, 7)
    assert_all(oracle_mod, g.n, g.src, g.dst, g.w, range(g.m))


def test_cycle_drops_heaviest(oracle_mod):
    n = 101
    rng = np.random.default_rng(5)
    src = np.arange(n, dtype=np.int32)
    dst = ((np.arange(n) + 1) % n).astype(np.int32)
    w = (rng.permutation(n) + 1).astype(np.uint32)
    expect = [e for e in range(n) if e != int(np.argmax(w))]
    assert_all(oracle_mod, n, src, dst, w, expect)


def test_complete_graph_star(oracle_mod):
    """K_n where the edges at vertex 0 are the n-1 lightest: the star."""
    n = 30
    edges = []
    for i in range(n):
        for j in range(i + 1, n):
            edges.append((i, j))
    w = np.array([(1 if i == 0 else 1000) + len(edges) - k for k, (i, j) in enumerate(edges)],
                 np.uint32)
    src, dst = np.array(edges, np.int32).T.copy()
    star = [k for k, (i, j) in enumerate(edges) if i == 0]
    assert_all(oracle_mod, n, src, dst, w, star)


def test_increasing_path(oracle_mod):
    """A path with increasing weights: all edges (and a deep hook chain)."""
    n = 3000
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    w = np.arange(1, n, dtype=np.uint32)
    assert_all(oracle_mod, n, src, dst, w, range(n - 1))


def test_parallel_edges_two_vertices(oracle_mod):
    rng = np.random.default_rng(9)
    k = 50
    src = np.zeros(k, np.int32)
    dst = np.ones(k, np.int32)
    w = (rng.permutation(k) + 1).astype(np.uint32)
    assert_all(oracle_mod, 2, src, dst, w, [int(np.argmin(w))])


def test_grid_horizontal_lighter(oracle_mod):
    """R x C grid, every horizontal edge lighter than every vertical edge:
    all R(C-1) horizontal edges plus, between each pair of adjacent rows, the
    single lightest vertical edge."""
    R, C = 12, 9
    rng = np.random.default_rng(11)
    edges, horiz, vert = [], [], {}
    for r in range(R):
        for c in range(C):
            v = r * C + c
            if c < C - 1:
                horiz.append(len(edges))
                edges.append((v, v + 1))
            if r < R - 1:
                vert.setdefault(r, []).append(len(edges))
                edges.append((v, v + C))
    m = len(edges)
    w = np.zeros(m, np.uint32)
    w[horiz] = rng.permutation(len(horiz)) + 1
    vid = sum(vert.values(), [])
    w[vid] = rng.permutation(len(vid)) + 1 + len(horiz)
    expect = list(horiz) + [min(ids, key=lambda e: w[e]) for ids in vert.values()]
    src, dst = np.array(edges, np.int32).T.copy()
    assert_all(oracle_mod, R * C, src, dst, w, expect)


def test_empty_and_single_vertex(oracle_mod):
    z = np.zeros(0, np.int32)
    assert_all(oracle_mod, 1, z, z, np.zeros(0, np.uint32), [])
    assert_all(oracle_mod, 0, z, z, np.zeros(0, np.uint32), [])


def test_self_loops_only(oracle_mod):
    src = np.array([0, 1, 1, 2], np.int32)
    assert_all(oracle_mod, 3, src, src.copy(), np.array([1, 2, 3, 4], np.uint32), [])


def test_disconnected_two_trees(oracle_mod):
    a = gg.random_connected(40, 39, 1)
    b = gg.random_connected(25, 24, 2)
    src = np.concatenate([a.src, b.src + 40]).astype(np.int32)
    dst = np.concatenate([a.dst, b.dst + 40]).astype(np.int32)
    w = np.concatenate([a.w, b.w + 100]).astype(np.uint32)
    assert_all(oracle_mod, 65 + 3, src, dst, w, range(63))  # + 3 isolated vertices
    assert oracle_mod.components(68, src, dst) == 5


def test_boruvka_round_bound(oracle_mod):
    """Every round at least halves the number of components (Section 2.1,
    O(m log n)), so a connected graph needs at most ceil(log2 n) rounds."""
    for seed, (n, m) in enumerate([(1000, 3000), (4096, 32768), (5000, 4999)]):
        g = gg.random_connected(n, m, 40 + seed)
        _, rounds = oracle_mod.boruvka(g.n, g.src, g.dst, g.w)
        assert 1 <= rounds <= math.ceil(math.log2(n))
    n = 2048  # increasing path: every vertex hooks to its left neighbour
    src = np.arange(n - 1, dtype=np.int32)
    ids, rounds = oracle_mod.boruvka(n, src, src + 1, np.arange(1, n, dtype=np.uint32))
    assert rounds == 1 and len(ids) == n - 1


# ------------------------------------------------------------ library checks

@pytest.mark.parametrize("seed", range(6))
def test_against_scipy(oracle_mod, seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = gg.random_connected(800 + 50 * seed, 4000, 100 + seed)
    mat = sp.coo_matrix((g.w.astype(np.float64), (g.src, g.dst)), shape=(g.n, g.n)).tocsr()
    t = csgraph.minimum_spanning_tree(mat).tocoo()
    lookup = {(min(u, v), max(u, v)): e for e, (u, v) in enumerate(zip(g.src, g.dst))}
    expect = sorted(lookup[(min(u, v), max(u, v))] for u, v in zip(t.row, t.col))
    assert_all(oracle_mod, g.n, g.src, g.dst, g.w, expect)


@pytest.mark.parametrize("algo", ["kruskal", "prim", "boruvka"])
def test_against_networkx(oracle_mod, algo):
    nx = pytest.importorskip("networkx")
    g = gg.random_connected(600, 2500, 77)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for e in range(g.m):
        G.add_edge(int(g.src[e]), int(g.dst[e]), weight=int(g.w[e]), id=e)
    expect = sorted(d["id"] for _, _, d in nx.minimum_spanning_edges(G, algorithm=algo, data=True))
    assert list(oracle_mod.kruskal(g.n, g.src, g.dst, g.w)) == expect


# --------------------------------------------------------------- certificates

def test_certificates_reject_wrong_trees(oracle_mod):
    g = gg.random_connected(300, 1500, 13)
    t = oracle_mod.kruskal(g.n, g.src, g.dst, g.w)
    assert oracle_mod.check_cycle_property(g.n, g.src, g.dst, g.w, t) == 0
    assert oracle_mod.check_cut_property(g.n, g.src, g.dst, g.w, t) == 0
    non_tree = np.setdiff1d(np.arange(g.m), t)
    adj = {}
    for x in t:
        adj.setdefault(int(g.src[x]), []).append((int(g.dst[x]), int(x)))
        adj.setdefault(int(g.dst[x]), []).append((int(g.src[x]), int(x)))

    def tree_path(a, b):  # edge ids on the tree path a..b
        prev = {a: None}
        stack = [a]
        while stack:
            x = stack.pop()
            for y, e in adj.get(x, []):
                if y not in prev:
                    prev[y] = (x, e)
                    stack.append(y)
        out = []
        while b != a:
            b, e = prev[b]
            out.append(e)
        return out

    rng = np.random.default_rng(0)
    for e in rng.permutation(non_tree)[:30]:
        path = tree_path(int(g.src[e]), int(g.dst[e]))
        drop = path[int(rng.integers(0, len(path)))]
        wrong = np.sort(np.r_[t[t != drop], e])  # another spanning tree, heavier
        assert oracle_mod.check_cycle_property(g.n, g.src, g.dst, g.w, wrong) == 4
        assert oracle_mod.check_cut_property(g.n, g.src, g.dst, g.w, wrong) == 5
    assert oracle_mod.check_cycle_property(g.n, g.src, g.dst, g.w, t[1:]) == 3  # not spanning
    cyc = np.sort(np.r_[t, non_tree[0]])
    assert oracle_mod.check_cycle_property(g.n, g.src, g.dst, g.w, cyc) == 2


def test_cycle_certificate_both_sides(oracle_mod):
    """Tree 0-1 (w 1), 0-2 (w 5) and non-tree 1-2 (w 3): the heavy edge sits
    on one side of the path next to the common ancestor, so a check that
    looks at only one side would accept this wrong tree.  Mirrored too."""
    for heavy_side in (0, 1):
        wts = [1, 5] if heavy_side else [5, 1]
        src = np.array([0, 0, 1], np.int32)
        dst = np.array([1, 2, 2], np.int32)
        w = np.array(wts + [3], np.uint32)
        assert oracle_mod.check_cycle_property(3, src, dst, w, [0, 1]) == 4
        assert oracle_mod.check_cut_property(3, src, dst, w, [0, 1]) == 5
        good = oracle_mod.kruskal(3, src, dst, w)
        assert oracle_mod.check_cycle_property(3, src, dst, w, good) == 0


# ------------------------------------------------------- agreement at scale

@pytest.mark.parametrize("make", [
    lambda: gg.config(1),
    lambda: gg.grid2d(64, 80, 3),
    lambda: gg.rmat(12, 8, 4),
    lambda: gg.paper_table1("Graph10K_3"),
    lambda: gg.paper_table1("Graph10K_9"),
    lambda: gg.random_connected(3000, 9000, 8, weights="f32"),
])
def test_agreement_and_certificate(oracle_mod, make):
    g = make()
    k, b1, b0, p = all_oracles(oracle_mod, g.n, g.src, g.dst, g.w)
    assert len(k) == g.n - oracle_mod.components(g.n, g.src, g.dst)
    assert np.array_equal(k, b1) and np.array_equal(k, b0) and np.array_equal(k, p)
    assert oracle_mod.check_cycle_property(g.n, g.src, g.dst, g.w, k) == 0


def test_total_weight_lower_bound(oracle_mod):
    """Weights a permutation of 1..m: the n-1 tree edges weigh at least the
    n-1 smallest weights, n(n-1)/2."""
    for g in (gg.config(1), gg.grid2d(50, 50, 2)):
        t = oracle_mod.kruskal(g.n, g.src, g.dst, g.w)
        assert oracle_mod.total_weight(g.w, t) >= g.n * (g.n - 1) // 2


@pytest.mark.parametrize("seed", range(6))
def test_parallel_edges_reduce_to_lightest(oracle_mod, seed):
    """Reading 7 (used when few components remain): of parallel edges between
    the same two vertices only the lightest under (weight, id) can be in the
    tree, so the tree of a multigraph equals the tree of its reduction to
    one edge per vertex pair.  Heavy ties make the id tie-break matter."""
    rng = np.random.default_rng(900 + seed)
    n = 30
    m = 400
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    w = rng.integers(1, 6, m).astype(np.uint32)
    full = set(oracle_mod.kruskal(n, src, dst, w).tolist())
    best = {}
    for e in range(m):
        a, b = int(src[e]), int(dst[e])
        if a == b:
            continue
        pair = (min(a, b), max(a, b))
        if pair not in best or (int(w[e]), e) < (int(w[best[pair]]), best[pair]):
            best[pair] = e
    keep = np.array(sorted(best.values()), dtype=np.int64)
    reduced = oracle_mod.kruskal(n, src[keep], dst[keep], w[keep])
    assert full == set(keep[reduced].tolist())
