"""The C-ABI library loads and exports every symbol include/mst.h declares;
host-side argument checks answer without a GPU (no compute calls)."""
import ctypes

import pytest

from paper_2005_06913_gb300 import binding as B


def test_exports_every_declared_symbol(lib_built):
    names = B.header_symbols()
    assert "mst_solve" in names and "mst_solve_batched" in names and "mst_create" in names
    L = B.lib()
    missing = [s for s in names if not hasattr(L, s)]
    assert not missing, missing
    assert set(B._SIGS) == set(names)  # the binding covers exactly the ABI


def test_status_strings(lib_built):
    for code in range(8):
        assert B.mst_status_string(code).startswith("MST_")


def test_null_handle_rejected_on_host(lib_built):
    L = B.lib()
    assert L.mst_solve(None, 4, 3, None, None, None, None, None, None) == B.MST_ERR_INVALID_ARG
    assert L.mst_solve_ex(None, 0, 4, 3, None, None, None, None, None, None) == B.MST_ERR_INVALID_ARG
    assert L.mst_destroy(None) == B.MST_ERR_INVALID_ARG
    assert L.mst_get_status(None, None) == B.MST_ERR_INVALID_ARG
    assert L.mst_set_batched_schedule(None, 0, 0) == B.MST_ERR_INVALID_ARG
    assert L.mst_create(None, 0, 0) == B.MST_ERR_INVALID_ARG


def test_every_handle_entry_point_rejects_null(lib_built):
    """Each entry point taking a handle checks it on the host, before any
    CUDA call (so this runs without a GPU)."""
    L = B.lib()
    bad = B.MST_ERR_INVALID_ARG
    tk = ctypes.c_uint64(0)
    done = ctypes.c_int(0)
    cnt = ctypes.c_int32(0)
    assert L.mst_solve_host(None, 0, 4, 3, None, None, None, None, None, None) == bad
    assert L.mst_solve_csr(None, 0, 4, 6, None, None, None, 0, None, None, None) == bad
    assert L.mst_solve_batched(None, 0, 1, None, None, 4, 3, None, None, None, None, None,
                               None) == bad
    assert L.mst_autotune_batched(None, 0, 1, None, None, 4, 3, None, None, None, None, None,
                                  None, None) == bad
    assert L.mst_set_single_schedule(None, 0, 0, 0) == bad
    assert L.mst_profile_last_solve(None, None, None, 0, ctypes.byref(cnt)) == bad
    assert L.mst_get_round_stats(None, None, None, None, 0, ctypes.byref(cnt)) == bad
    assert L.mst_server_start(None, 2, 4) == bad
    assert L.mst_submit(None, 0, 4, 3, None, None, None, None, None, ctypes.byref(tk)) == bad
    assert L.mst_poll(None, 1, ctypes.byref(done), None) == bad
    assert L.mst_server_drain(None) == bad
    assert L.mst_server_stop(None) == bad


def test_create_bad_device(lib_built):
    h = ctypes.c_void_p()
    assert B.lib().mst_create(ctypes.byref(h), -1, 0) == B.MST_ERR_INVALID_ARG
