"""Full-size checks in the launch configuration bench.py times.

At these sizes the brute-force oracle cannot produce the whole answer, so each test checks
properties that hold at any size plus sampled outputs the oracle computes one by one:
  - the result is a spanning tree of n-1 edges with u < v, listed in non-decreasing weight;
  - EMST: for sampled points p, the K-minimum edge from p to any other point (brute force, FP64)
    is a tree edge with exactly that weight (cut property of the cut {p});
  - HDBSCAN*: sampled core distances equal the oracle's brute-force values bit for bit, and
    sampled tree edges carry exactly max(cd(u), cd(v), d(u,v)) with oracle cd and distances;
  - the dendrogram is consistent (sizes add up, heights grow toward the root) and the
    reachability plot is its in-order leaf sequence with bars at the in-order internal nodes.
"""
import math

import numpy as np
import pytest

import oracle
import synthdata
import paper_2104_01126_gb300 as wm
from gpu_common import require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    wm.load()


def _spanning_tree(n, u, v):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    assert len(u) == n - 1
    assert np.all(u < v) and u.min() >= 0 and v.max() < n
    g = coo_matrix((np.ones(len(u), np.int8), (u, v)), shape=(n, n))
    ncomp, _ = connected_components(g, directed=False)
    assert ncomp == 1


def _edge_lookup(u, v, w):
    key = u.astype(np.int64) * (1 << 32) + v.astype(np.int64)
    order = np.argsort(key)
    return key[order], w[order]


def _find_edge(keys, ws, a, b):
    k = min(a, b) * (1 << 32) + max(a, b)
    i = np.searchsorted(keys, k)
    return ws[i] if i < len(keys) and keys[i] == k else None


@pytest.mark.parametrize("kind,d", [("uniform", 2), ("uniform", 3), ("varden", 3), ("uniform", 5), ("varden", 5),
                                    ("uniform", 7), ("varden", 7)])
def test_emst_ten_million_points(kind, d):
    n = 10_000_000
    x = synthdata.generate(kind, n, d, seed=0)
    r = wm.emst(x)
    u, v, w = r["u"], r["v"], r["w"]
    _spanning_tree(n, u, v)
    assert np.all(np.diff(w) >= 0)
    assert math.isclose(r["total"], math.fsum(w), rel_tol=1e-12)
    keys, ws = _edge_lookup(u, v, w)
    rng = np.random.default_rng(1)
    x64 = np.ascontiguousarray(x, dtype=np.float64)
    for p in rng.choice(n, size=24, replace=False):
        q, w2 = oracle.nearest_edge(x64, int(p))
        got = _find_edge(keys, ws, int(p), q)
        assert got is not None, (p, q)
        assert got == math.sqrt(w2)


@pytest.fixture(scope="module")
def hdb_1m():
    x = synthdata.gaussian_mixture(1_000_000, 3, seed=0)
    r = wm.hdbscan(x, min_pts=10, start=0)
    return x, {k: to_np(v) for k, v in r.items()}


def test_hdbscan_config2_tree_and_sampled_weights(hdb_1m):
    x, r = hdb_1m
    n = len(x)
    u, v, w, cd = r["u"], r["v"], r["w"], r["cd"]
    _spanning_tree(n, u, v)
    assert np.all(np.diff(w) >= 0)
    rng = np.random.default_rng(2)
    pts = rng.choice(n, size=120, replace=False)
    cd2 = oracle.core_dist2_subset(x, 10, pts)
    assert np.array_equal(cd[pts], np.sqrt(cd2))
    es = rng.choice(n - 1, size=120, replace=False)
    ends = np.unique(np.concatenate([u[es], v[es]]))
    cde = dict(zip(ends.tolist(), oracle.core_dist2_subset(x, 10, ends).tolist()))
    for i in es:
        a, b = int(u[i]), int(v[i])
        want = math.sqrt(max(cde[a], cde[b], oracle.sqdist(x, a, b)))
        assert w[i] == want


def test_hdbscan_config2_dendrogram_and_plot(hdb_1m):
    x, r = hdb_1m
    n = len(x)
    left, right, height, size = r["left"], r["right"], r["height"], r["size"]
    assert np.array_equal(height, r["w"])
    sz = np.concatenate([np.ones(n, np.int64), size.astype(np.int64)])
    h = np.concatenate([np.zeros(n), height])
    assert np.array_equal(sz[left] + sz[right], size)
    assert np.all(h[left] <= height) and np.all(h[right] <= height)
    assert size[-1] == n
    # in-order leaf sequence of the ordered dendrogram == the reachability order
    order = r["order"]
    assert order[0] == 0 and r["reach"][0] == math.inf
    assert np.array_equal(np.sort(order), np.arange(n))
    first = np.empty(2 * n - 1, np.int64)   # in-order index of each node's first leaf
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    first[:n] = pos
    # internal nodes in merge order: children precede parents
    for i in range(n - 1):
        first[n + i] = first[left[i]]
    # left subtree ends right before the right subtree starts
    assert np.array_equal(first[left] + sz[left], first[right])
    reach = r["reach"]
    assert np.array_equal(reach[first[right]], height)
