"""Tuning changes speed, never results: every setting of the wm_tuning parameters must return the
same K-minimum tree (and for HDBSCAN* the same core distances, dendrogram and plot), equal to the
FP64 oracle.  Covers the box-diagonal and the tighter diameter bounds, small and large traversal
chunks and depth-first budgets, the BCCP size-class cut-offs and dual-tree routing, and the
one-pass (combined GetRho / GetPairs) rounds."""
import numpy as np
import pytest

import oracle
import synthdata
import paper_2104_01126_gb300 as wm
from gpu_common import assert_same_tree, require_gpu, to_np

pytestmark = pytest.mark.gpu

SETTINGS = [
    {"tight_diameters": 0},
    {"tight_diameters": 1},
    {"chunk_log2": 12, "dfs_budget": 1},
    {"chunk_log2": 16, "dfs_budget": 32},
    {"medium_max": 65, "big_max": 65, "route_big": 0},
    {"medium_max": 4096, "big_max": 1 << 20, "route_big": 1 << 30},
    {"route_big": 0},
    {"combined": 1},
    {"combined": 1, "tight_diameters": 1, "chunk_log2": 12, "dfs_budget": 2},
    {"combined": 2},
    {"getrho_sample": 16},
    {"getrho_sample": 4, "combined": 2, "tight_diameters": 1},
    {"edges_per_point": 64},
    {"range_ratio": 2},
    {"range_ratio": 8, "combined": 1},
    {"range_ratio": 4, "range_gate": 10},
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    wm.load()
    yield
    wm.set_tuning(None)


@pytest.mark.parametrize("kind,n,d", [("uniform", 6000, 3), ("varden", 8000, 5), ("gmm", 5000, 7), ("varden", 7000, 2)])
def test_emst_same_under_every_tuning(kind, n, d):
    x = synthdata.generate(kind, n, d, seed=n + d)
    ref = oracle.emst(x)
    for p in SETTINGS:
        with wm.tuning(**p):
            got = wm.emst(x)
        assert_same_tree(got, ref), p


def test_hdbscan_same_under_every_tuning():
    x = synthdata.generate("gmm", 4000, 3, seed=77)
    ref = oracle.hdbscan(x, 10, s=5)
    for p in SETTINGS:
        with wm.tuning(**p):
            got = {k: to_np(v) for k, v in wm.hdbscan(x, min_pts=10, start=5).items()}
        assert np.array_equal(got["cd"], ref["cd"]), p
        assert_same_tree(got, ref)
        for key in ("left", "right", "size", "height", "order", "reach"):
            assert np.array_equal(got[key], ref[key]), (p, key)
