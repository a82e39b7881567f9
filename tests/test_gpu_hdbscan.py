"""HDBSCAN* parity: core distances, MST of G_MR, ordered dendrogram and reachability plot from
the CUDA path against the FP64 oracle, element by element (Sec. 2.1, Sec. 3.1, Sec. 4)."""
import numpy as np
import pytest

import oracle
import synthdata
import paper_2104_01126_gb300 as wm
from gpu_common import assert_same_tree, require_gpu, to_np, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    wm.load()


def _check_all(got, ref, n):
    got = {k: to_np(v) for k, v in got.items() if k != "stats"}
    assert np.array_equal(got["cd"], ref["cd"]), np.flatnonzero(got["cd"] != ref["cd"])[:5]
    assert_same_tree(got, ref)
    if n >= 2:
        for key in ("left", "right", "size"):
            assert np.array_equal(got[key], ref[key]), (key, np.flatnonzero(got[key] != ref[key])[:5])
        assert np.array_equal(got["height"], ref["height"])
    assert np.array_equal(got["order"], ref["order"])
    assert np.array_equal(got["reach"], ref["reach"])


CASES = [
    ("gmm", 3000, 3, 10, 0), ("gmm", 4000, 2, 5, 1), ("uniform", 3000, 2, 10, 2), ("varden", 5000, 3, 10, 3),
    ("gmm", 2000, 5, 50, 4), ("uniform", 1500, 7, 20, 5), ("gmm", 257, 3, 3, 6), ("gmm", 40, 2, 10, 7),
    ("uniform", 1000, 1, 4, 8), ("gmm", 1200, 10, 8, 9),
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind,n,d,mp,seed", CASES)
def test_hdbscan_matches_oracle(kind, n, d, mp, seed, precision):
    x = synthdata.generate(kind, n, d, seed)
    start = seed % n
    ref = oracle.hdbscan(x, mp, s=start)
    got = wm.hdbscan(x, min_pts=mp, start=start, precision=precision)
    _check_all(got, ref, n)


@pytest.mark.parametrize("mp", [1, 2])
def test_hdbscan_small_min_pts_equals_emst(mp):
    x = synthdata.gaussian_mixture(3000, 3, seed=mp)
    e = oracle.emst(x)
    got = wm.hdbscan(x, min_pts=mp)
    assert_same_tree({k: to_np(got[k]) for k in ("u", "v", "w")}, e)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_hdbscan_tiny(n):
    x = synthdata.uniform(n, 2, seed=n)
    ref = oracle.hdbscan(x, 1, s=0)
    _check_all(wm.hdbscan(x, min_pts=1), ref, n)


def test_hdbscan_min_pts_equal_n():
    x = synthdata.uniform(30, 3, seed=4)
    _check_all(wm.hdbscan(x, min_pts=30, start=5), oracle.hdbscan(x, 30, s=5), 30)


def test_hdbscan_device_tensors():
    x = synthdata.gaussian_mixture(6000, 3, seed=11)
    ref = oracle.hdbscan(x, 10, s=17)
    got = wm.hdbscan(torch.from_numpy(x).cuda(), min_pts=10, start=17)
    assert got["order"].is_cuda
    _check_all(got, ref, len(x))


def test_single_linkage_of_emst_matches_oracle():
    x = synthdata.uniform(5000, 2, seed=31)
    e = oracle.emst(x)
    ref = oracle.single_linkage(len(x), e["u"], e["v"], e["w2"], s=9)
    got = wm.single_linkage(len(x), e["u"], e["v"], e["w"], start=9)
    for key in ("left", "right", "size", "order"):
        assert np.array_equal(got[key], ref[key]), key
    assert np.array_equal(got["height"], ref["height"])
    assert np.array_equal(got["reach"], ref["reach"])


def test_single_linkage_path_with_increasing_weights():
    """A chain whose weights increase along it: the dendrogram is a caterpillar of depth n-1."""
    n = 3000
    u = np.arange(n - 1, dtype=np.int32)
    v = u + 1
    w = np.arange(1, n, dtype=np.float64)
    ref = oracle.single_linkage(n, u, v, w * w, s=n - 1)
    got = wm.single_linkage(n, u, v, w, start=n - 1)
    for key in ("left", "right", "size", "order"):
        assert np.array_equal(got[key], ref[key]), key
