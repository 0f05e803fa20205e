"""Thin Python binding of libmst's C ABI (include/mst.h), via ctypes.

Every function has the C name and argument order; device buffers may be
passed as torch tensors (their ``data_ptr()`` is used) or raw integer device
addresses, and ``stream`` as a ``torch.cuda.Stream``, a raw ``cudaStream_t``
integer, or None for torch's current stream.  Functions return the
``mst_status`` code; nothing here computes any part of a spanning tree.

The library must have been built (``paper_2005_06913_gb300.build.build()``);
if it is missing, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmst.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mst.h")

MST_OK = 0
MST_ERR_INVALID_ARG = 1
MST_ERR_OOM = 2
MST_ERR_CUDA = 3
MST_ERR_DISCONNECTED = 4
MST_ERR_TIMEOUT = 5
MST_ERR_BUDGET = 6
MST_ERR_INTERNAL = 7
MST_W_U32 = 0
MST_W_F32 = 1

_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_INT = ctypes.c_int

_SIGS = {
    "mst_status_string": (ctypes.c_char_p, [_INT]),
    "mst_create": (_INT, [ctypes.POINTER(_P), _INT, ctypes.c_size_t]),
    "mst_destroy": (_INT, [_P]),
    "mst_solve": (_INT, [_P, _I32, _I64, _P, _P, _P, _P, _P, _P]),
    "mst_solve_ex": (_INT, [_P, _INT, _I32, _I64, _P, _P, _P, _P, _P, _P]),
    "mst_solve_host": (_INT, [_P, _INT, _I32, _I64, _P, _P, _P, _P, _P, _P]),
    "mst_solve_csr": (_INT, [_P, _INT, _I32, _I64, _P, _P, _P, ctypes.c_uint32, _P, _P, _P]),
    "mst_profile_last_solve": (_INT, [_P, _P, _P, _I32, ctypes.POINTER(_I32)]),
    "mst_solve_batched": (_INT, [_P, _INT, _I32, _P, _P, _I64, _I64, _P, _P, _P, _P, _P, _P]),
    "mst_get_status": (_INT, [_P, _P]),
    "mst_get_batched_status": (_INT, [_P, _P, _I32, _P]),
    "mst_get_round_stats": (_INT, [_P, _P, _P, _P, _I32, ctypes.POINTER(_I32)]),
    "mst_set_batched_schedule": (_INT, [_P, _INT, _INT]),
    "mst_set_single_schedule": (_INT, [_P, _INT, _INT, _INT]),
    "mst_set_wait_limit": (_INT, [_P, ctypes.c_uint32]),
    "mst_autotune_batched": (_INT, [_P, _INT, _I32, _P, _P, _I64, _I64, _P, _P, _P, _P, _P,
                                    ctypes.c_char_p, _P]),
    "mst_solve_noalloc": (_INT, [_INT, _I32, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "mst_server_start": (_INT, [_P, _INT, _INT]),
    "mst_submit": (_INT, [_P, _INT, _I32, _I64, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "mst_poll": (_INT, [_P, ctypes.c_uint64, ctypes.POINTER(_INT), ctypes.POINTER(ctypes.c_double)]),
    "mst_server_drain": (_INT, [_P]),
    "mst_server_stop": (_INT, [_P]),
}


class MstError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {mst_status_string(status)}" if what else mst_status_string(status))


def lib() -> ctypes.CDLL:
    """Loads libmst.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmst.so not built (expected at {LIB_PATH}); "
                               "run paper_2005_06913_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols() -> list:
    """Function names declared in include/mst.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:mst_status|const\s+char\s*\*)\s*(mst_\w+)\s*\(", text, re.M)))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"expected a tensor or a device address, got {type(x)}")


def _stream(s) -> int:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def mst_status_string(status: int) -> str:
    if _lib is None and not os.path.exists(LIB_PATH):
        return f"status {status}"
    return lib().mst_status_string(int(status)).decode()


def mst_create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    h = _P()
    st = lib().mst_create(ctypes.byref(h), int(device), int(mem_budget_bytes))
    if st != MST_OK:
        raise MstError(st, "mst_create")
    return h.value


def mst_destroy(h) -> int:
    return lib().mst_destroy(h)


def mst_solve(h, n, m, src, dst, w, out_edge_ids, out_count, stream=None) -> int:
    return lib().mst_solve(h, int(n), int(m), _ptr(src), _ptr(dst), _ptr(w), _ptr(out_edge_ids),
                           _ptr(out_count), _stream(stream))


def mst_solve_ex(h, wt, n, m, src, dst, w, out_edge_ids, out_count, stream=None) -> int:
    return lib().mst_solve_ex(h, int(wt), int(n), int(m), _ptr(src), _ptr(dst), _ptr(w),
                              _ptr(out_edge_ids), _ptr(out_count), _stream(stream))


MST_CSR_SYMMETRIC = 1


def mst_solve_csr(h, wt, n, nnz, row_ptr, col, w, flags, out_edge_ids, out_count,
                  stream=None) -> int:
    """Adjacency-CSR solve: row_ptr (int64, n+1), col (int32), w on the
    device; the tree's ids are CSR positions."""
    return lib().mst_solve_csr(h, int(wt), int(n), int(nnz), _ptr(row_ptr), _ptr(col), _ptr(w),
                               int(flags), _ptr(out_edge_ids), _ptr(out_count), _stream(stream))


def mst_solve_host(h, wt, n, m, src, dst, w, out_edge_ids, out_count, stream=None) -> int:
    """Host-buffer solve: src/dst/w/out/out_count are host addresses (tensors
    on the CPU, ideally pinned, or integer addresses)."""
    return lib().mst_solve_host(h, int(wt), int(n), int(m), _ptr(src), _ptr(dst), _ptr(w),
                                _ptr(out_edge_ids), _ptr(out_count), _stream(stream))


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int32),
                ("total_ms", ctypes.c_double), ("alg_bytes", ctypes.c_double)]


def mst_profile_last_solve(h, stream=None, cap: int = 64):
    """Returns a list of dicts {name, launches, total_ms, alg_bytes}."""
    arr = (KernelProfile * cap)()
    k = _I32(0)
    st = lib().mst_profile_last_solve(h, _stream(stream), ctypes.addressof(arr), cap, ctypes.byref(k))
    if st != MST_OK:
        raise MstError(st, "mst_profile_last_solve")
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches, total_ms=arr[i].total_ms,
                 alg_bytes=arr[i].alg_bytes) for i in range(k.value)]


def mst_solve_batched(h, wt, G, vtx_off, edge_off, total_n, total_m, src, dst, w, out_edge_ids,
                      out_counts, stream=None) -> int:
    return lib().mst_solve_batched(h, int(wt), int(G), _ptr(vtx_off), _ptr(edge_off),
                                   int(total_n), int(total_m), _ptr(src), _ptr(dst), _ptr(w),
                                   _ptr(out_edge_ids), _ptr(out_counts), _stream(stream))


def mst_get_status(h, stream=None) -> int:
    return lib().mst_get_status(h, _stream(stream))


def mst_get_batched_status(h, G: int, stream=None):
    """Returns (status, per-graph statuses as a list) of the last batched solve."""
    arr = (_I32 * max(int(G), 1))()
    st = lib().mst_get_batched_status(h, _stream(stream), int(G), ctypes.addressof(arr))
    return st, list(arr[: int(G)])


def mst_get_round_stats(h, stream=None, cap: int = 65):
    """Returns (live_edges, live_vertices) per round of the last single solve."""
    e = (ctypes.c_int64 * cap)()
    v = (ctypes.c_int64 * cap)()
    r = _I32(0)
    st = lib().mst_get_round_stats(h, _stream(stream), ctypes.addressof(e), ctypes.addressof(v),
                                   cap, ctypes.byref(r))
    if st != MST_OK:
        raise MstError(st, "mst_get_round_stats")
    k = min(r.value + 1, cap)
    return list(e[:k]), list(v[:k])


def mst_set_single_schedule(h, schedule: int, blocks_per_sm: int = 0, block_threads: int = 0) -> int:
    return lib().mst_set_single_schedule(h, int(schedule), int(blocks_per_sm), int(block_threads))


def mst_set_wait_limit(h, polls: int) -> int:
    return lib().mst_set_wait_limit(h, int(polls))


def mst_set_batched_schedule(h, schedule: int, block_threads: int = 0) -> int:
    return lib().mst_set_batched_schedule(h, int(schedule), int(block_threads))


def mst_autotune_batched(h, wt, G, vtx_off, edge_off, total_n, total_m, src, dst, w,
                         out_edge_ids, out_counts, cache_path=None, stream=None) -> int:
    cp = cache_path.encode() if cache_path else None
    return lib().mst_autotune_batched(h, int(wt), int(G), _ptr(vtx_off), _ptr(edge_off),
                                      int(total_n), int(total_m), _ptr(src), _ptr(dst), _ptr(w),
                                      _ptr(out_edge_ids), _ptr(out_counts), cp, _stream(stream))


def mst_solve_noalloc(wt, n, m, src, dst, w, out_edge_ids, out_count, out_status=None,
                      stream=None) -> int:
    """Allocation-free solve of one small graph (no handle; see mst.h)."""
    return lib().mst_solve_noalloc(int(wt), int(n), int(m), _ptr(src), _ptr(dst), _ptr(w),
                                   _ptr(out_edge_ids), _ptr(out_count), _ptr(out_status),
                                   _stream(stream))


def mst_server_start(h, streams: int = 4, max_batch: int = 256) -> int:
    return lib().mst_server_start(h, int(streams), int(max_batch))


def mst_submit(h, wt, n, m, src, dst, w, out_edge_ids, out_count):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64(0)
    st = lib().mst_submit(h, int(wt), int(n), int(m), _ptr(src), _ptr(dst), _ptr(w),
                          _ptr(out_edge_ids), _ptr(out_count), ctypes.byref(t))
    return st, t.value


def mst_poll(h, ticket):
    """Returns (status, done, latency_us)."""
    d = _INT(0)
    lat = ctypes.c_double(0.0)
    st = lib().mst_poll(h, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(lat))
    return st, bool(d.value), lat.value


def mst_server_drain(h) -> int:
    return lib().mst_server_drain(h)


def mst_server_stop(h) -> int:
    return lib().mst_server_stop(h)


# ------------------------------------------------------------ conveniences

def weight_type(w) -> int:
    """MST_W_F32 for float32 tensors/arrays, else MST_W_U32."""
    dt = str(getattr(w, "dtype", ""))
    return MST_W_F32 if "float32" in dt else MST_W_U32


def solve(h, n, src, dst, w, stream=None, check=True):
    """Solves one graph given torch CUDA tensors; returns (ids, status).

    ``ids`` is an int32 tensor of the tree's edge ids in ascending order.
    Allocates the outputs with torch (marshalling only)."""
    import torch
    dev = src.device
    out = torch.empty(max(int(n) - 1, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    st = mst_solve_ex(h, weight_type(w), n, src.numel(), src, dst, w, out, cnt, stream)
    if st != MST_OK:
        raise MstError(st, "mst_solve_ex")
    status = mst_get_status(h, stream)
    if check and status not in (MST_OK, MST_ERR_DISCONNECTED):
        raise MstError(status, "device status")
    return out[: int(cnt.item())], status
