"""The ablation forms of the method against the FP64 oracle, element by element:

- GFK (Sec. 3.2.2, Algorithm 2): the full WSPD materialised, each pair's BCCP computed once;
- EMST-Naive (Sec. 5): the BCCP of every pair of the full WSPD, then one Kruskal;
- GanTao (Sec. 3.1.1): HDBSCAN* with the standard (geometric) well-separation and BCCP*.

Every form computes the same K-minimum tree; the counters show what each one does: Naive
evaluates the BCCP of every WSPD pair, GFK of at most as many, and the disjunctive separation
of Sec. 3.1.2 needs fewer pairs than GanTao's geometric one.
"""
import math

import numpy as np
import pytest

import oracle
import synthdata
import paper_2104_01126_gb300 as wm
from gpu_common import assert_same_tree, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    wm.load()


EMST_CASES = [("uniform", 3000, 2, 0), ("gmm", 5000, 3, 1), ("varden", 4000, 5, 2), ("uniform", 1500, 7, 3),
              ("uniform", 2, 2, 4), ("uniform", 3, 3, 5), ("uniform", 40, 2, 6)]


@pytest.mark.parametrize("method", ["gfk", "naive"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind,n,d,seed", EMST_CASES)
def test_emst_methods_match_oracle(method, precision, kind, n, d, seed):
    x = synthdata.generate(kind, n, d, seed)
    ref = oracle.emst(x)
    got = wm.emst(x, precision=precision, method=method, return_stats=True)
    assert_same_tree({k: to_np(got[k]) for k in ("u", "v", "w")}, ref)
    assert abs(got["total"] - ref["total"]) <= 1e-12 * max(ref["total"], 1e-300)
    s = got["stats"]
    if n > 2:
        assert s.wspd_pairs > 0
        assert s.pairs_retrieved <= s.wspd_pairs
        if method == "naive":
            assert s.pairs_retrieved == s.wspd_pairs


def test_emst_methods_on_ties_and_duplicates():
    g = synthdata.unit_grid(20, 2, seed=3)
    dup = np.repeat(synthdata.uniform(300, 3, seed=4), 3, axis=0)
    for x in (g, dup):
        ref = oracle.emst(x)
        for method in ("gfk", "naive"):
            assert_same_tree({k: to_np(v) for k, v in wm.emst(x, method=method).items() if k != "total"}, ref)


def test_gfk_at_scale_matches_boruvka():
    x = synthdata.generate("uniform", 1_000_000, 3, seed=0, dtype=np.float32)
    ref = oracle.emst_at_scale(x)
    for method in ("gfk", "naive"):
        got = wm.emst(x, method=method)
        assert np.array_equal(to_np(got["u"]), ref["u"]) and np.array_equal(to_np(got["v"]), ref["v"])
        assert np.array_equal(to_np(got["w"]), ref["w"])
        assert math.isclose(got["total"], ref["total"], rel_tol=1e-12)


def _hdb_same(got, ref):
    got = {k: to_np(v) for k, v in got.items() if k != "stats"}
    assert np.array_equal(got["cd"], ref["cd"])
    assert_same_tree(got, ref)
    for key in ("left", "right", "size", "height", "order", "reach"):
        assert np.array_equal(got[key], ref[key]), key


@pytest.mark.parametrize("method", ["gfk", "naive", "gantao"])
@pytest.mark.parametrize("kind,n,d,mp,seed", [("gmm", 3000, 3, 10, 0), ("varden", 3000, 2, 5, 1),
                                              ("uniform", 1200, 5, 20, 2)])
def test_hdbscan_methods_match_oracle(method, kind, n, d, mp, seed):
    x = synthdata.generate(kind, n, d, seed)
    ref = oracle.hdbscan(x, mp, s=seed)
    _hdb_same(wm.hdbscan(x, min_pts=mp, start=seed, method=method), ref)


@pytest.mark.parametrize("mp", [10, 50])
def test_disjunctive_separation_needs_fewer_pairs(mp):
    # the full WSPD of each separation rule, counted by the GFK form: the mutual-unreachability
    # disjunction (Sec. 3.1.2) separates node pairs higher up the tree than geometry alone, and
    # both give the oracle's tree
    x = synthdata.generate("gmm", 20000, 3, seed=5)
    ref = oracle.hdbscan_at_scale(x, mp, 0)
    ours = wm.hdbscan(x, min_pts=mp, method="gfk", return_stats=True)
    geo = wm.hdbscan(x, min_pts=mp, method="gfk-geometric", return_stats=True)
    _hdb_same(ours, ref)
    _hdb_same(geo, ref)
    assert 0 < ours["stats"].wspd_pairs < geo["stats"].wspd_pairs
