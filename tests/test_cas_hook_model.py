"""Host model of the compare-and-swap hook (Section 2.2.2) under adversarial
interleaving (no GPU).

Each thread of a round holds one component's minimum edge: it finds the
roots of the edge's endpoints (path halving), then swaps one root's parent
from itself to the other root, retrying the finds when the swap fails.
Every load, store and swap is one step, and a seeded scheduler picks which
thread steps next.  The model checks the link rule the GPU's schedule 4
uses: the higher-numbered root goes under the lower one.  With the fixed
direction of the paper's union (the destination's root under the source's),
a root found first can be hooked into the other endpoint's tree before the
swap, and the swap then closes a cycle; the model finds one on three
vertices.
"""
import random

import numpy as np
import pytest


class Cycle(Exception):
    pass


def cas_round(parent, minima, by_index, rng):
    """One round of CAS hooks over `minima` (component -> (edge id, a, b))
    with random interleaving; returns the edge ids added."""
    added = []

    def find(x):
        while True:
            p = parent[x]
            yield
            if p == x:
                return x
            gp = parent[p]
            yield
            if gp != p:
                parent[x] = gp
                yield
            x = gp

    def thread(i, a, b):
        while True:
            c1 = yield from find(a)
            c2 = yield from find(b)
            if c1 == c2:
                return
            lo, hi = (min(c1, c2), max(c1, c2)) if by_index else (c1, c2)
            if parent[hi] == hi:  # the swap: one step
                parent[hi] = lo
                added.append(i)
                return
            yield

    active = [thread(*minima[c]) for c in sorted(minima)]
    while active:
        t = rng.choice(active)
        try:
            next(t)
        except StopIteration:
            active.remove(t)
    n = len(parent)
    for v in range(n):  # every pointer chain must end at a root
        x, hops = v, 0
        while parent[x] != x:
            x = parent[x]
            hops += 1
            if hops > n:
                raise Cycle(v)
    return added


def boruvka_cas(n, src, dst, w, by_index, rng):
    """Borůvka rounds whose hook is `cas_round`, keys (weight, id)."""
    comp = list(range(n))
    live = [i for i in range(len(src)) if src[i] != dst[i]]
    tree = []
    ncur = n
    while live:
        minima = {}
        for i in live:
            a, b = comp[src[i]], comp[dst[i]]
            for c in (a, b):
                if c not in minima or (w[i], i) < (w[minima[c][0]], minima[c][0]):
                    minima[c] = (i, a, b)
        parent = list(range(ncur))
        tree += cas_round(parent, minima, by_index, rng)

        def root(x):
            while parent[x] != x:
                x = parent[x]
            return x

        roots = [v for v in range(ncur) if parent[v] == v]
        nid = {r: k for k, r in enumerate(roots)}
        comp = [nid[root(c)] for c in comp]
        ncur = len(roots)
        live = [i for i in live if comp[src[i]] != comp[dst[i]]]
    return np.asarray(sorted(tree), dtype=np.int64)


def random_graph(rng):
    n = rng.randint(2, 12)
    m = rng.randint(1, 30)
    src = [rng.randrange(n) for _ in range(m)]
    dst = [rng.randrange(n) for _ in range(m)]
    w = [rng.randrange(rng.choice([2, 5, 100])) for _ in range(m)]
    return n, src, dst, w


def test_index_ordered_links_match_kruskal(oracle_mod):
    rng = random.Random(12345)
    for _ in range(400):
        n, src, dst, w = random_graph(rng)
        got = boruvka_cas(n, src, dst, w, True, rng)
        expect = oracle_mod.kruskal(n, np.asarray(src, np.int32), np.asarray(dst, np.int32),
                                    np.asarray(w, np.uint32))
        assert np.array_equal(got, expect)


def test_index_ordered_links_deep_paths(oracle_mod):
    rng = random.Random(7)
    n = 200
    src = list(range(n - 1))
    dst = [v + 1 for v in src]
    for w in (list(range(n - 1)), list(range(n - 1, 0, -1))):  # chains both ways
        got = boruvka_cas(n, src, dst, w, True, rng)
        assert np.array_equal(got, np.arange(n - 1))


def test_fixed_direction_can_close_a_cycle():
    """Three components; 0 and 2 choose edge 6 (2->1), 1 chooses edge 1
    (0->1).  Thread for 1 hooks 1 under 2; the thread for 0 fails on 1, then
    hooks 2 under 0; the other thread of edge 6 had found root 2 before that
    and now finds root 0 for vertex 1: it hangs 0 below 2."""
    found = False
    for seed in range(200):
        rng = random.Random(seed)
        parent = [0, 1, 2]
        minima = {0: (1, 0, 1), 1: (6, 2, 1), 2: (6, 2, 1)}
        try:
            cas_round(parent, minima, False, rng)
        except Cycle:
            found = True
            break
    assert found
    for seed in range(200):  # the index rule on the same round never does
        rng = random.Random(seed)
        parent = [0, 1, 2]
        minima = {0: (1, 0, 1), 1: (6, 2, 1), 2: (6, 2, 1)}
        assert sorted(cas_round(parent, minima, True, rng)) == [1, 6]
