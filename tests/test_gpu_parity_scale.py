"""Element-by-element parity at full size.

The brute-force oracle cannot reach 10^6 points, so these tests use its exact k-d tree solvers
(Boruvka for the K-minimum spanning tree, k-NN for the core distances; pinned against the brute
force in tests/test_oracle.py) and compare every output of the CUDA path with them:
  - HDBSCAN* on the bench workload (10^6 Gaussian-mixture points in 3-D, minPts 10, FP32 screen,
    the call bench.py times): MST edges and weights, core distances, dendrogram, order and bars;
  - EMST on the scale generators: 10^7 points (uniform 2-D and 3-D, varden 2-D), and 10^6 points
    for the other generator / dimension pairs (3 x 10^5 for varden 7-D).
"""
import functools
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


def test_hdbscan_bench_workload_full_parity():
    import torch
    x = synthdata.gaussian_mixture(1_000_000, 3, seed=0)
    got = wm.hdbscan(torch.from_numpy(x).cuda(), min_pts=10, start=0, precision="fp32")
    ref = oracle.hdbscan_at_scale(x, 10, 0)
    assert np.array_equal(to_np(got["cd"]), ref["cd"])
    for key in ("u", "v", "w", "left", "right", "height", "size", "order", "reach"):
        assert np.array_equal(to_np(got[key]), ref[key]), key


@pytest.mark.parametrize("kind,d,n", [("uniform", 2, 10_000_000), ("uniform", 3, 10_000_000),
                                      ("varden", 2, 10_000_000), ("uniform", 3, 1_000_000),
                                      ("varden", 2, 1_000_000), ("varden", 3, 1_000_000),
                                      ("uniform", 5, 1_000_000), ("varden", 5, 1_000_000),
                                      ("uniform", 7, 1_000_000), ("varden", 7, 300_000)])
def test_emst_full_parity(kind, d, n):
    import torch
    x = synthdata.generate(kind, n, d, seed=0)
    got = wm.emst(torch.from_numpy(x).cuda())
    _check_emst(got, _emst_ref(kind, d, n))


@functools.lru_cache(maxsize=2)
def _emst_ref(kind, d, n):
    return oracle.emst_at_scale(synthdata.generate(kind, n, d, seed=0))


def _check_emst(got, ref):
    assert np.array_equal(to_np(got["u"]), ref["u"])
    assert np.array_equal(to_np(got["v"]), ref["v"])
    assert np.array_equal(to_np(got["w"]), ref["w"])
    assert math.isclose(got["total"], ref["total"], rel_tol=1e-12)


def test_emst_grown_edge_batch_full_parity():
    """A round whose candidate edges overflow the first part of the batch, in a call whose work so
    far is mostly traversal, grows the batch and redoes the flush with the same range (instead of
    lowering rho_hi): uniform 7-D points at 10^6 with a 16-edges-per-point batch take that path."""
    import torch
    x = synthdata.generate("uniform", 1_000_000, 7, seed=0)
    with wm.tuning(edges_per_point=16, combined=0, getrho_sample=1):
        got = wm.emst(torch.from_numpy(x).cuda(), return_stats=True)
    assert got["stats"].edge_batch_grown == 1 and got["stats"].rho_shrinks == 0
    _check_emst(got, _emst_ref("uniform", 7, 1_000_000))
