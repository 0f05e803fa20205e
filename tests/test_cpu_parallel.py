"""The host-thread parallel Boruvka of Section 2.2.2 (compare-and-swap joins),
the multithreaded CPU baseline, against Kruskal (no GPU)."""
import numpy as np
import pytest

from paper_2005_06913_gb300 import graphgen as gg


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_random_graphs_with_ties(oracle_mod, threads):
    rng = np.random.default_rng(100 + threads)
    for _ in range(30):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(0, 1200))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        w = rng.integers(0, int(rng.choice([3, 50, 1 << 30])), m).astype(np.uint32)
        got, _, used = oracle_mod.boruvka_cas_parallel(n, src, dst, w, threads)
        assert used == threads
        assert np.array_equal(got, oracle_mod.kruskal(n, src, dst, w))


def test_float_weights_and_disconnected(oracle_mod):
    rng = np.random.default_rng(5)
    n, m = 2000, 3000  # sparse: several components and isolated vertices
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    w = rng.choice(np.array([-1.5, 0.0, 0.25, 3.0, 1e9], np.float32), m)
    got, _, _ = oracle_mod.boruvka_cas_parallel(n, src, dst, w, 4)
    expect = oracle_mod.kruskal(n, src, dst, w)
    assert np.array_equal(got, expect)
    assert len(got) == n - oracle_mod.components(n, src, dst)


def test_deep_chains(oracle_mod):
    n = 20000
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    for w in (np.arange(1, n, dtype=np.uint32), np.arange(n - 1, 0, -1).astype(np.uint32)):
        got, _, _ = oracle_mod.boruvka_cas_parallel(n, src, dst, w, 6)
        assert np.array_equal(got, np.arange(n - 1))


def test_paper_table1_shape(oracle_mod):
    g = gg.paper_table1("Graph100K_6")
    got, rounds, _ = oracle_mod.boruvka_cas_parallel(g.n, g.src, g.dst, g.w, 0)
    assert np.array_equal(got, oracle_mod.kruskal(g.n, g.src, g.dst, g.w))
    assert 1 <= rounds <= 40


def test_bad_ids_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.boruvka_cas_parallel(3, np.array([0], np.int32), np.array([3], np.int32),
                                        np.array([1], np.uint32), 2)


def test_golden_fixtures(oracle_mod):
    """The paper's own small examples (tests/golden), at several thread counts."""
    import os
    from test_oracle import GOLDEN, arrays, load_golden
    for name in sorted(os.listdir(GOLDEN)):
        n, edges, mst = load_golden(os.path.join(GOLDEN, name))
        src, dst, w = arrays(edges)
        for t in (1, 2, 3):
            got, _, _ = oracle_mod.boruvka_cas_parallel(n, src, dst, w, t)
            assert got.tolist() == sorted(mst), (name, t)
