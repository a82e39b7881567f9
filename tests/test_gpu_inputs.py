"""Input paths of the C ABI that the other parity tests do not reach, against the FP64 oracle.

- WM_SOA input (one contiguous array per coordinate), FP32 and FP64, host and device;
- a caller-owned workspace arena (wm_opts.workspace): identical results, and WM_ENOMEM when the
  arena is too small;
- HDBSCAN* on duplicate-heavy inputs (far from general position): with each point repeated
  minPts times every core distance is 0 and the result must still equal the oracle's K-minimum
  tree; with more copies than the k-NN lists keep, the tie-repair buffer overflows, which the call
  reports through stats.tie_overflow while still returning an MST of G_MR (Sec. 2.1).
"""
import math

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


def _hdb_equal(got, ref):
    got = {k: to_np(v) for k, v in got.items() if k != "stats"}
    assert np.array_equal(got["cd"], ref["cd"])
    assert_same_tree(got, ref)
    for key in ("left", "right", "size", "height", "order", "reach"):
        assert np.array_equal(got[key], ref[key]), key


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("device", [False, True])
def test_emst_soa_layout(dtype, device):
    x = synthdata.generate("gmm", 4000, 3, seed=21, dtype=dtype)
    ref = oracle.emst(x)
    soa = np.ascontiguousarray(x.T)
    got = wm.emst(torch.from_numpy(soa).cuda() if device else soa, layout="soa")
    assert_same_tree({k: to_np(got[k]) for k in ("u", "v", "w")}, ref)
    assert abs(got["total"] - ref["total"]) <= 1e-12 * ref["total"]


def test_hdbscan_soa_layout():
    x = synthdata.generate("varden", 3000, 5, seed=22)
    ref = oracle.hdbscan(x, 10, s=7)
    got = wm.hdbscan(np.ascontiguousarray(x.T), min_pts=10, start=7, layout="soa")
    _hdb_equal(got, ref)


def _arena(nbytes):
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    return buf, (buf.data_ptr(), nbytes)


def test_caller_workspace_emst_and_hdbscan():
    x = synthdata.generate("gmm", 20000, 3, seed=23)
    buf, ws = _arena(wm.query_footprint(len(x), 3, 0))
    ref = oracle.emst_at_scale(x)
    for _ in range(2):   # the arena is reused as it is
        got = wm.emst(x, workspace=ws, return_stats=True)
        assert_same_tree({k: to_np(got[k]) for k in ("u", "v", "w")}, ref)
        assert 0 < got["stats"].workspace_bytes_used <= ws[1]
    hbuf, hws = _arena(wm.query_footprint(len(x), 3, 10))
    got = wm.hdbscan(x, min_pts=10, start=3, workspace=hws)
    _hdb_equal(got, oracle.hdbscan_at_scale(x, 10, 3))
    del buf, hbuf


def test_caller_workspace_too_small_is_enomem():
    x = synthdata.generate("uniform", 20000, 3, seed=24)
    buf, ws = _arena(1 << 20)
    with pytest.raises(wm.WMError) as e:
        wm.emst(x, workspace=ws)
    assert e.value.code == -2
    with pytest.raises(wm.WMError) as e:
        wm.hdbscan(x, min_pts=10, workspace=ws)
    assert e.value.code == -2
    # the library still works afterwards
    assert_same_tree({k: to_np(v) for k, v in wm.emst(x).items() if k != "total"}, oracle.emst_at_scale(x))
    del buf


def _duplicated(distinct, copies, d, seed):
    base = synthdata.uniform(distinct, d, seed=seed, dtype=np.float32)
    x = np.repeat(base, copies, axis=0)
    return np.ascontiguousarray(x[np.random.default_rng(seed).permutation(len(x))])


def test_hdbscan_duplicates_within_the_lists_match_oracle():
    # every point repeated minPts = 10 times: all core distances are 0, G_MR's weights are the
    # Euclidean ones, and the K-minimum tree is unique however many ties there are
    x = _duplicated(10_000, 10, 3, seed=25)
    got = wm.hdbscan(x, min_pts=10, start=0, return_stats=True)
    assert got["stats"].tie_overflow == 0
    _hdb_equal(got, oracle.hdbscan_at_scale(x, 10, 0))


def test_hdbscan_duplicate_overflow_reported():
    # 20 copies of each point: more exact ties than the k-NN lists hold; the repair edges (19 per
    # point) exceed their buffer, which the call must report (tie_overflow) while still returning
    # an MST of G_MR with the oracle's weight, core distances and a consistent dendrogram
    n_distinct, copies = 5_000, 20
    x = _duplicated(n_distinct, copies, 2, seed=26)
    n = len(x)
    got = wm.hdbscan(x, min_pts=10, start=0, return_stats=True)
    assert got["stats"].tie_overflow == 1
    ref = oracle.hdbscan_at_scale(x, 10, 0)
    r = {k: to_np(v) for k, v in got.items() if k != "stats"}
    assert np.array_equal(r["cd"], ref["cd"])
    u, v, w = r["u"], r["v"], r["w"]
    assert len(u) == n - 1 and np.all(u < v) and np.all(np.diff(w) >= 0)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    assert connected_components(coo_matrix((np.ones(n - 1), (u, v)), shape=(n, n)), directed=False)[0] == 1
    assert math.isclose(math.fsum(w), math.fsum(ref["w"]), rel_tol=1e-12)
    assert np.array_equal(np.sort(w), np.sort(ref["w"]))   # MST weights form a unique multiset
    assert r["size"][-1] == n and np.array_equal(np.sort(r["order"]), np.arange(n))


def test_screen_error_is_measured_and_within_the_band():
    # the FP32 screen's error against the exact FP64 value, measured per result on the device:
    # positive (rounding happens) and within the a priori relative band 2^-19 for FP32 coordinates
    x = synthdata.generate("gmm", 20000, 3, seed=27)
    for r in (wm.hdbscan(x, min_pts=10, return_stats=True), wm.emst(x, return_stats=True)):
        e = r["stats"].max_rel_screen_err
        assert 0.0 < e <= 2.0 ** -19, e
    assert wm.emst(x, precision="fp64", return_stats=True)["stats"].max_rel_screen_err == 0.0
