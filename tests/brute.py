"""Brute-force minimum spanning forest for tiny graphs (pure Python).

Independent of the oracle: enumerates every edge subset of the right size,
keeps those that form a spanning forest (one tree per connected component),
and returns the one that is smallest by (total weight, sum of edge ids).
For any input, that lexicographic minimiser is the unique minimum spanning
forest under the order "smaller weight, then smaller edge id": perturbing
each weight by epsilon * id with epsilon small makes all weights distinct
without changing the order, and the perturbed total is exactly that pair.
"""
from fractions import Fraction
from itertools import combinations


def _find(p, x):
    while p[x] != x:
        x = p[x]
    return x


def n_components(n, edges):
    p = list(range(n))
    c = n
    for (u, v) in edges:
        a, b = _find(p, u), _find(p, v)
        if a != b:
            p[a] = b
            c -= 1
    return c


def is_forest(n, edges):
    p = list(range(n))
    for (u, v) in edges:
        a, b = _find(p, u), _find(p, v)
        if a == b:
            return False
        p[a] = b
    return True


def brute_msf(n, src, dst, w):
    """Sorted edge ids of the minimum spanning forest (exhaustive search)."""
    m = len(src)
    pairs = [(int(src[e]), int(dst[e])) for e in range(m)]
    k = n - n_components(n, pairs)
    wt = [Fraction(float(x)) for x in w]  # exact for uint32 and float32
    best, best_key = None, None
    for sub in combinations(range(m), k):
        if not is_forest(n, [pairs[e] for e in sub]):
            continue
        key = (sum(wt[e] for e in sub), sum(sub))
        if best_key is None or key < best_key:
            best, best_key = sub, key
    return list(best) if best is not None else []
