"""EMST parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bar: the K-minimum spanning tree's edge list (K order) identical, weights bit-exact, total
weight within a relative 1e-12 (Sec. 2.1 EMST; K = (w2, min id, max id)).
"""
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


CASES = [
    ("uniform", 2, 2, 0), ("uniform", 3, 2, 1), ("uniform", 33, 2, 2), ("uniform", 257, 2, 3),
    ("uniform", 3000, 2, 4), ("uniform", 4099, 3, 5), ("uniform", 3001, 5, 6), ("uniform", 2500, 7, 7),
    ("gmm", 5000, 3, 8), ("varden", 6000, 2, 9), ("varden", 4000, 3, 10), ("uniform", 1500, 1, 11),
    ("uniform", 800, 4, 12), ("uniform", 700, 11, 13), ("uniform", 600, 16, 14),
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kind,n,d,seed", CASES)
def test_emst_matches_oracle(kind, n, d, seed, precision):
    x = synthdata.generate(kind, n, d, seed)
    ref = oracle.emst(x)
    got = wm.emst(x, precision=precision)
    assert_same_tree(got, ref)
    assert abs(got["total"] - ref["total"]) <= 1e-12 * max(ref["total"], 1e-300)


def test_emst_config1_bit_exact():
    """n = 10,000 uniform points in [0,1)^2 from seed 0, FP64 coordinates, plain FP64 form."""
    x = synthdata.uniform(10_000, 2, seed=0)
    ref = oracle.emst(x)
    assert not ref["tie"]
    for prec in ("fp64", "fp32"):
        got = wm.emst(x, precision=prec)
        assert_same_tree(got, ref)
        assert abs(got["total"] - ref["total"]) <= 1e-12 * ref["total"]


def test_emst_device_input_and_stream():
    x = synthdata.uniform(5000, 3, seed=21).astype(np.float32)
    ref = oracle.emst(x)
    xd = torch.from_numpy(x).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = wm.emst(xd)
    assert got["u"].is_cuda
    assert_same_tree({k: to_np(v) for k, v in got.items() if k != "total"}, ref)


@pytest.mark.parametrize("n", [1, 2, 17, 1000])
def test_emst_collinear_closed_form_and_ties(n):
    """Fully tied input: weight n-1; the K tie-break fixes the tree, so it still matches."""
    x = synthdata.collinear(n, d=2, seed=n)
    got = wm.emst(x)
    assert got["total"] == float(n - 1)
    if n > 1:
        assert_same_tree(got, oracle.emst(x))


@pytest.mark.parametrize("k,d", [(30, 2), (9, 3)])
def test_emst_grid_closed_form(k, d):
    x = synthdata.unit_grid(k, d, seed=k)
    got = wm.emst(x)
    assert got["total"] == float(k ** d - 1)
    assert_same_tree(got, oracle.emst(x))


def test_emst_duplicates_and_clusters_of_identical_points():
    g = np.random.default_rng(5)
    base = g.random((300, 3))
    x = np.concatenate([base, base[:100], np.repeat(base[:3], 40, axis=0)])
    x = x[g.permutation(len(x))]
    assert_same_tree(wm.emst(x), oracle.emst(x))


def test_emst_far_from_origin_fp64_input():
    """FP64 input not representable in FP32: the screen's absolute error term must hold."""
    x = 1000.0 + synthdata.uniform(3000, 2, seed=3) * 1e-3
    assert_same_tree(wm.emst(x, precision="fp32"), oracle.emst(x))


def test_emst_rejects_bad_input():
    with pytest.raises(wm.WMError):
        wm.emst(np.array([[0.0, np.nan], [1.0, 2.0]]))
    with pytest.raises(wm.WMError):
        wm.emst(np.zeros((4, 17)))


def test_emst_stats_and_rounds_are_logarithmic():
    x = synthdata.uniform(20_000, 2, seed=7).astype(np.float32)
    got = wm.emst(x, return_stats=True)
    st = got["stats"]
    assert st.rounds <= 2 * int(np.log2(20_000)) + 4
    assert st.bccp_evals > 0 and st.tree_nodes == 2 * 20_000 - 1
