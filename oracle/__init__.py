"""CPU oracle for minimum spanning trees — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never loads it, and it
shares no code with the CUDA path.

The arithmetic lives in ``mst_oracle.c`` (plain C, compiled here with gcc);
this module only marshals numpy arrays.  Every function returns the sorted
edge ids (indices into the input arrays) of the minimum spanning forest
under the order "smaller weight, then smaller edge id".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mst_oracle.c")
_SRC_MT = os.path.join(_HERE, "mst_cpu_parallel.c")
_LIB = os.path.join(_HERE, "libmst_oracle.so")
_lib = None

_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``mst_oracle.c`` and ``mst_cpu_parallel.c`` into
    ``libmst_oracle.so`` (gcc, -O2, POSIX threads)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_MT))):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    try:
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               "-Wall", "-o", tmp, _SRC, _SRC_MT])
        os.replace(tmp, _LIB)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return _LIB


def _bind(path):
    """Load a compiled oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    for name in ("orc_kruskal", "orc_prim"):
        f = getattr(lib, name)
        f.restype = _I64
        f.argtypes = [_I64, _I64, _P, _P, _P, ctypes.c_int, _P]
    lib.orc_boruvka.restype = _I64
    lib.orc_boruvka.argtypes = [_I64, _I64, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P]
    lib.orc_boruvka_cas_mt.restype = _I64
    lib.orc_boruvka_cas_mt.argtypes = [_I64, _I64, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P]
    lib.orc_components.restype = _I64
    lib.orc_components.argtypes = [_I64, _I64, _P, _P]
    for name in ("orc_check_cycle_property", "orc_check_cut_property"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [_I64, _I64, _P, _P, _P, ctypes.c_int, _P]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _prep(n, src, dst, w):
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    w = np.ascontiguousarray(w)
    if src.shape != dst.shape or src.shape != w.shape or src.ndim != 1:
        raise ValueError("src, dst and w must be 1-D arrays of equal length")
    if w.dtype == np.uint32:
        wt = 0
    elif w.dtype == np.float32:
        wt = 1
        if np.isnan(w).any():
            raise ValueError("NaN weight")
    else:
        raise TypeError("weights must be uint32 or float32")
    return int(n), src, dst, w, wt


def _ids(rc, flags):
    if rc == -1:
        raise ValueError("vertex id out of range")
    if rc < 0:
        raise MemoryError("oracle out of memory")
    ids = np.flatnonzero(flags).astype(np.int64)
    assert ids.shape[0] == rc
    return ids


def kruskal(n, src, dst, w) -> np.ndarray:
    """Kruskal's algorithm (sort by the edge order, union-find)."""
    n, src, dst, w, wt = _prep(n, src, dst, w)
    flags = np.zeros(max(src.shape[0], 1), np.uint8)
    rc = _load().orc_kruskal(n, src.shape[0], src.ctypes.data, dst.ctypes.data,
                             w.ctypes.data, wt, flags.ctypes.data)
    return _ids(rc, flags[:src.shape[0]])


def boruvka(n, src, dst, w, covered: bool = True):
    """Sequential Boruvka of Section 2.1 (``covered`` = its optimisation).

    Returns ``(ids, rounds)``."""
    n, src, dst, w, wt = _prep(n, src, dst, w)
    flags = np.zeros(max(src.shape[0], 1), np.uint8)
    rounds = ctypes.c_int64(0)
    rc = _load().orc_boruvka(n, src.shape[0], src.ctypes.data, dst.ctypes.data,
                             w.ctypes.data, wt, int(bool(covered)), flags.ctypes.data,
                             ctypes.addressof(rounds))
    return _ids(rc, flags[:src.shape[0]]), int(rounds.value)


def boruvka_cas_parallel(n, src, dst, w, threads: int = 0):
    """The Section 2.2.2 parallel Boruvka (compare-and-swap joins) on
    ``threads`` host threads (0 = every core).  A CPU baseline, checked
    against Kruskal by the tests.  Returns ``(ids, rounds, threads)``."""
    n, src, dst, w, wt = _prep(n, src, dst, w)
    if threads <= 0:
        threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") \
            else (os.cpu_count() or 1)
    threads = max(1, min(int(threads), 256))
    flags = np.zeros(max(src.shape[0], 1), np.uint8)
    rounds = ctypes.c_int64(0)
    rc = _load().orc_boruvka_cas_mt(n, src.shape[0], src.ctypes.data, dst.ctypes.data,
                                    w.ctypes.data, wt, threads, flags.ctypes.data,
                                    ctypes.addressof(rounds))
    if rc == -3:
        raise RuntimeError("could not start the worker threads")
    return _ids(rc, flags[:src.shape[0]]), int(rounds.value), threads


def prim(n, src, dst, w) -> np.ndarray:
    """Prim's algorithm with a binary heap, restarted per component."""
    n, src, dst, w, wt = _prep(n, src, dst, w)
    flags = np.zeros(max(src.shape[0], 1), np.uint8)
    rc = _load().orc_prim(n, src.shape[0], src.ctypes.data, dst.ctypes.data,
                          w.ctypes.data, wt, flags.ctypes.data)
    return _ids(rc, flags[:src.shape[0]])


def components(n, src, dst) -> int:
    """Number of connected components."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    rc = _load().orc_components(int(n), src.shape[0], src.ctypes.data, dst.ctypes.data)
    if rc < 0:
        raise ValueError("bad input")
    return int(rc)


def _flags_of(m, ids):
    flags = np.zeros(max(m, 1), np.uint8)
    flags[np.asarray(ids, dtype=np.int64)] = 1
    return flags


def check_cycle_property(n, src, dst, w, ids) -> int:
    """0 if ``ids`` is a spanning forest satisfying the cycle property."""
    n, src, dst, w, wt = _prep(n, src, dst, w)
    flags = _flags_of(src.shape[0], ids)
    return int(_load().orc_check_cycle_property(n, src.shape[0], src.ctypes.data,
                                                dst.ctypes.data, w.ctypes.data, wt,
                                                flags.ctypes.data))


def check_cut_property(n, src, dst, w, ids) -> int:
    """0 if every edge of ``ids`` is the lightest edge across its cut."""
    n, src, dst, w, wt = _prep(n, src, dst, w)
    flags = _flags_of(src.shape[0], ids)
    return int(_load().orc_check_cut_property(n, src.shape[0], src.ctypes.data,
                                              dst.ctypes.data, w.ctypes.data, wt,
                                              flags.ctypes.data))


def total_weight(w, ids):
    """Total weight: exact uint64 sum for uint32 weights; for float32 a float64
    sum taken in ascending edge-id order (reproducible)."""
    ids = np.sort(np.asarray(ids, dtype=np.int64))
    if w.dtype == np.uint32:
        return int(w[ids].astype(np.uint64).sum())
    acc = 0.0
    for x in w[ids].astype(np.float64):
        acc += float(x)
    return acc
