"""The oracle's pins catch planted mistakes (no GPU).

Each case copies the oracle's C source, plants one plausible mistake, builds
the mutant into a temporary library and checks that at least one pin from
the oracle test-suite fails against it.  The mistake lives only in the
temporary copy; the real oracle is never modified.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from brute import brute_msf
from paper_2005_06913_gb300 import graphgen as gg

SRC = os.path.join(os.path.dirname(oracle.__file__), "mst_oracle.c")

MUTANTS = {
    "weight order flipped": ("return x < y;", "return x > y;"),
    "tie-break by larger id": ("return a < b;", "return a > b;"),
    "float compare ignores order": ("if (x < y)\n            return 1;", "if (x > y)\n            return 1;"),
    "boruvka skips the re-check": ("            if (c1 == c2)\n                continue;\n            in_tree[e] = 1;",
                                   "            in_tree[e] = 1;"),
    "boruvka keeps first edge": ("if (minimum[c1] == -1 || lighter(w, wt, e, minimum[c1]))",
                                 "if (minimum[c1] == -1)"),
    "kruskal skips find": ("int64_t a = uf_find(parent, src[e]), b = uf_find(parent, dst[e]);\n        if (a != b) {\n            uf_union",
                           "int64_t a = src[e], b = dst[e];\n        if (a != b) {\n            uf_union"),
    "prim takes heaviest": ("if (!lighter(h->w, h->wt, h->heap[i], h->heap[p]))", "if (lighter(h->w, h->wt, h->heap[i], h->heap[p]))"),
    "cycle check misses one side": ("            TAKE(mx[0][a]);\n            TAKE(mx[0][b]);", "            TAKE(mx[0][a]);"),
}


def build_mutant(tmp_path, old, new):
    text = open(SRC).read()
    assert text.count(old) >= 1, old
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(old, new, 1))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-w",
                           "-o", str(so), str(path), oracle._SRC_MT])
    return oracle._bind(str(so))


def pins_hold():
    """A compact subset of the oracle pins; False if any fails."""
    try:
        rng = np.random.default_rng(7)
        for _ in range(25):
            n = int(rng.integers(3, 7))
            m = int(rng.integers(3, 11))
            src = rng.integers(0, n, m).astype(np.int32)
            dst = rng.integers(0, n, m).astype(np.int32)
            for w in (rng.integers(1, 4, m).astype(np.uint32),
                      (rng.integers(1, 4, m) / 2).astype(np.float32)):
                expect = brute_msf(n, src, dst, w)
                if list(oracle.kruskal(n, src, dst, w)) != expect:
                    return False
                if list(oracle.boruvka(n, src, dst, w)[0]) != expect:
                    return False
                if list(oracle.prim(n, src, dst, w)) != expect:
                    return False
        for wts in ([1, 5, 3], [5, 1, 3]):  # heavy path edge on either side
            src = np.array([0, 0, 1], np.int32)
            dst = np.array([1, 2, 2], np.int32)
            if oracle.check_cycle_property(3, src, dst, np.array(wts, np.uint32), [0, 1]) == 0:
                return False
        g = gg.random_connected(200, 800, 3)
        t = oracle.kruskal(g.n, g.src, g.dst, g.w)
        if oracle.check_cycle_property(g.n, g.src, g.dst, g.w, t) != 0:
            return False
        # a heavier spanning tree must be rejected by the certificate
        non_tree = np.setdiff1d(np.arange(g.m), t)
        for e in non_tree[:20]:
            for drop in t:
                wrong = np.sort(np.r_[t[t != drop], e])
                r = oracle.check_cut_property(g.n, g.src, g.dst, g.w, wrong)
                if r == 5 and oracle.check_cycle_property(g.n, g.src, g.dst, g.w, wrong) == 0:
                    return False
                if r == 5:
                    break
        return True
    except (AssertionError, ValueError, MemoryError):
        return False


def test_real_oracle_passes_pins():
    assert pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    old, new = MUTANTS[name]
    monkeypatch.setattr(oracle, "_lib", build_mutant(tmp_path, old, new))
    assert not pins_hold(), f"pins did not catch mutant: {name}"
