"""Ordered dendrogram and reachability plot (Sec. 4.1, 4.2; Sec. 2.1) of given spanning trees,
CUDA path (wm_single_linkage) against the oracle, element by element.

The trees are shaped to reach the dendrogram's parts that EMST inputs rarely do: sizes on both
sides of the shared-memory block of the lowest heavy/light levels (2048 edges) and of a few
global levels above it; paths (the longest Euler tours, every list-ranking sublist long),
stars (one vertex in every merge) and caterpillars; tied weights ordered by the key's ids.
Weights are distinct or tied integers, so w2 = w * w and sqrt(w2) = w are exact on both sides.
"""
import numpy as np
import pytest

import oracle
import paper_2104_01126_gb300 as wm
from gpu_common import require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    wm.load()


def _tree(shape, n, rng):
    """Edges (u, v) of a spanning tree on n vertices with randomly permuted labels."""
    idx = np.arange(1, n)
    if shape == "random":
        par = np.array([rng.integers(0, i) for i in idx], dtype=np.int64)
    elif shape == "path":
        par = idx - 1
    elif shape == "star":
        par = np.zeros(n - 1, dtype=np.int64)
    elif shape == "caterpillar":   # a spine of n/2 vertices, each other vertex hangs off it
        spine = max(n // 2, 1)
        par = np.where(idx < spine, idx - 1, rng.integers(0, spine, size=n - 1))
    else:
        raise ValueError(shape)
    perm = rng.permutation(n)
    return perm[idx].astype(np.int32), perm[par].astype(np.int32)


def _compare(n, u, v, w, start):
    ref = oracle.single_linkage(n, u, v, w.astype(np.float64) ** 2, s=start)
    got = wm.single_linkage(n, u, v, w.astype(np.float64), start=start)
    for key in ("left", "right", "size", "order"):
        g = to_np(got[key])
        assert np.array_equal(g, ref[key]), (key, np.flatnonzero(g != ref[key])[:5])
    assert np.array_equal(to_np(got["height"]), ref["height"])
    assert np.array_equal(to_np(got["reach"]), ref["reach"])


@pytest.mark.parametrize("shape", ["random", "path", "star", "caterpillar"])
@pytest.mark.parametrize("n", [2, 3, 2048, 2049, 2050, 4097, 65537])
def test_single_linkage_shapes_and_block_boundaries(shape, n):
    rng = np.random.default_rng(n * 7 + len(shape))
    u, v = _tree(shape, n, rng)
    w = rng.permutation(n - 1) + 1                 # distinct integer weights
    _compare(n, u, v, w, int(rng.integers(0, n)))


@pytest.mark.parametrize("n", [5000, 70001])
def test_single_linkage_tied_weights(n):
    rng = np.random.default_rng(n)
    u, v = _tree("random", n, rng)
    w = rng.integers(1, 4, size=n - 1)             # three weights: the ids decide most merges
    _compare(n, u, v, w, 0)


def test_single_linkage_all_equal_weights_on_a_path():
    n = 10000
    rng = np.random.default_rng(1)
    u, v = _tree("path", n, rng)
    _compare(n, u, v, np.ones(n - 1, dtype=np.int64), n // 2)
