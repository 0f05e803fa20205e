"""Splitting a batch of independent graphs across ranks (one GPU each).

Graphs of a batch share nothing, so N ranks solve disjoint subsets with no
data-path collective: each rank takes its share, solves it with one batched
launch, and only the timing (and, if wanted, results) meet on the host.
The split is longest-processing-time-first on edge counts: graphs in
decreasing size go to the currently lightest rank, which keeps every rank's
edge total within one graph of the mean.
"""
from __future__ import annotations

import numpy as np


def shard_graphs(sizes, world: int, rank: int) -> np.ndarray:
    """Indices (ascending) of the graphs that `rank` of `world` solves.

    ``sizes`` are per-graph work estimates (edge counts); ties are broken by
    graph index so every rank computes the same assignment independently.
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    order = np.lexsort((np.arange(sizes.shape[0]), -sizes))
    load = np.zeros(world, np.int64)
    owner = np.empty(sizes.shape[0], np.int64)
    for g in order:
        r = int(np.argmin(load))  # lowest load, lowest rank on ties
        owner[g] = r
        load[r] += sizes[g] + 1
    return np.flatnonzero(owner == rank)


def sub_batch(batch, idx):
    """The graphs ``idx`` of a graphgen.Batch as a new, re-packed Batch."""
    from .graphgen import Batch
    idx = np.asarray(idx, dtype=np.int64)
    ns = (batch.vtx_off[idx + 1] - batch.vtx_off[idx]).astype(np.int64)
    ms = (batch.edge_off[idx + 1] - batch.edge_off[idx]).astype(np.int64)
    vtx_off = np.r_[0, np.cumsum(ns)].astype(np.int64)
    edge_off = np.r_[0, np.cumsum(ms)].astype(np.int64)
    take = np.concatenate([np.arange(batch.edge_off[g], batch.edge_off[g + 1]) for g in idx]) \
        if idx.shape[0] else np.zeros(0, np.int64)
    return Batch(vtx_off, edge_off, batch.src[take], batch.dst[take], batch.w[take],
                 f"{batch.name}[shard of {idx.shape[0]}]")
