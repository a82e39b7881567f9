"""The C-ABI library builds, loads and exports every symbol that include/wspdmst.h declares.

No compute call is made here (the container has no GPU); wm_strerror / wm_version /
wm_query_footprint touch no device.
"""
import ctypes
import os
import re

import pytest

import paper_2104_01126_gb300 as wm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "wspdmst.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for required in ["wm_emst", "wm_hdbscan", "wm_single_linkage", "wm_query_footprint", "wm_strerror",
                     "wm_last_error_detail", "wm_release_cache", "wm_version"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(wm.build.build())
    missing = [s for s in _declared() if not hasattr(lib, s)]
    assert not missing, missing


def test_record_layouts_match_header():
    assert ctypes.sizeof(wm._Edge) == 16
    assert ctypes.sizeof(wm._DNode) == 24
    assert wm._Opts.workspace.offset == 16


def test_error_strings_and_footprint_without_gpu():
    lib = wm.load()
    assert lib.wm_strerror(0) == b"success"
    assert lib.wm_strerror(-1) == b"invalid argument"
    assert b"sm_103a" in lib.wm_version()
    assert wm.query_footprint(10_000, 2) > 0
    assert wm.query_footprint(1_000_000, 3, 10) > wm.query_footprint(1_000_000, 3, 0)
    b = ctypes.c_size_t(0)
    assert lib.wm_query_footprint(0, 2, 0, ctypes.byref(b)) == -1
    assert lib.wm_query_footprint(10, 17, 0, ctypes.byref(b)) == -1


def test_tuning_get_set_without_gpu():
    # the tuning calls touch no device: the table lookup and the override are host state
    base = wm.get_tuning(1_000_000, 3, 0)
    assert set(base) == set(wm.TUNING_FIELDS)
    assert ctypes.sizeof(wm._Tuning) == 64
    try:
        with pytest.raises(wm.WMError):
            wm.set_tuning({"dfs_budget": 0})
        with pytest.raises(wm.WMError):
            wm.set_tuning({"medium_max": 64})
        with pytest.raises(wm.WMError):
            wm.set_tuning({"edges_per_point": 65})
        with pytest.raises(wm.WMError):
            wm.set_tuning({"range_ratio": 1})
        with pytest.raises(wm.WMError):
            wm.set_tuning({"range_gate": -1})
        # a larger edge batch is part of the workspace estimate: 3 buffers of 16-byte edges
        small = wm.query_footprint(1_000_000, 3, 0)
        wm.set_tuning({"edges_per_point": 36})
        assert wm.query_footprint(1_000_000, 3, 0) - small >= 32 * 1_000_000 * 48
        wm.set_tuning({"dfs_budget": 4, "tight_diameters": 0})
        got = wm.get_tuning(10, 7, 5)
        assert got["dfs_budget"] == 4 and got["tight_diameters"] == 0
        # every field round-trips through the override
        want = dict(wm.get_tuning(0, 3, 0), range_ratio=8, range_gate=10, edges_per_point=16, getrho_sample=4)
        wm.set_tuning(want)
        assert wm.get_tuning(123, 5, 0) == want
    finally:
        wm.set_tuning(None)
    assert wm.get_tuning(1_000_000, 3, 0) == base
    from paper_2104_01126_gb300 import autotune
    assert wm.get_tuning(0, 3, 0) == autotune.DEFAULTS   # n = 0: the built-in defaults


def test_every_built_in_tuning_row_is_a_valid_setting():
    # the table is generated; each row a call can pick must pass the same range checks as an
    # override (wm_set_tuning rejects what the kernels do not support)
    try:
        for min_pts in (0, 10):
            for d in (1, 2, 3, 4, 5, 6, 7, 8, 12, 16):
                for n in (10, 100_000, 1_000_000, 10_000_000, 100_000_000):
                    row = wm.get_tuning(n, d, min_pts)
                    wm.set_tuning(row)
                    assert wm.get_tuning(n, d, min_pts) == row
                    wm.set_tuning(None)
    finally:
        wm.set_tuning(None)
