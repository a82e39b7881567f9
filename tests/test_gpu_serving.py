"""Serving: jobs of mixed n, d and minPts submitted to a continuous-batching server give exactly
the result of the same job run alone (wm_emst / wm_hdbscan), the server overlaps jobs, and
admission against the HBM budget rejects a job that can never fit and serialises jobs that do
not fit together."""
import time

import numpy as np
import pytest

import synthdata
import paper_2104_01126_gb300 as wm
from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    wm.load()


def _mix(count, seed):
    g = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        n = int(np.exp(g.uniform(np.log(1000), np.log(60000))))
        d = int(g.choice([2, 3, 5, 7]))
        kind = "emst" if i % 2 == 0 else "hdbscan"
        mp = int(g.choice([10, 50]))
        gen = "gmm" if g.random() < 0.5 else "uniform"
        x = synthdata.generate(gen, n, d, seed=1000 + i).astype(np.float32)
        jobs.append((kind, x, mp))
    return jobs


def _alone(kind, x, mp):
    if kind == "emst":
        return wm.emst(x)
    return wm.hdbscan(x, min_pts=mp, start=0)


def _same(got, ref, kind):
    for k in ("u", "v", "w"):
        assert np.array_equal(got[k], ref[k]), k
    if kind == "emst":
        assert got["total"] == ref["total"]
    else:
        for k in ("cd", "left", "right", "height", "size", "order", "reach"):
            assert np.array_equal(got[k], ref[k]), k


def test_result_alone_equals_result_in_mix():
    jobs = _mix(16, seed=3)
    refs = [_alone(*j) for j in jobs]
    with wm.Server(hbm_budget_bytes=48 << 30, workers=4) as srv:
        tickets = []
        for kind, x, mp in jobs:          # arrive while others are running
            tickets.append(srv.submit(x, kind=kind, min_pts=mp))
            time.sleep(0.002)
        outs = [srv.wait(t) for t in tickets]
        c = srv.counters()
    for (kind, _, _), (got, lat), ref in zip(jobs, outs, refs):
        assert lat > 0
        _same(got, ref, kind)
    assert c["finished"] == len(jobs)
    assert c["peak_running"] >= 2          # jobs overlapped on the device


def test_admission_budget():
    x = synthdata.gaussian_mixture(20000, 3, seed=5)
    fp = wm.query_footprint(20000, 3, 10)
    ref = wm.hdbscan(x, min_pts=10)
    # a budget that holds one job at a time: jobs still all finish, never two at once
    with wm.Server(hbm_budget_bytes=int(fp * 1.5), workers=3) as srv:
        ts = [srv.submit(x, kind="hdbscan", min_pts=10) for _ in range(3)]
        for t in ts:
            got, _ = srv.wait(t)
            _same(got, ref, "hdbscan")
        assert srv.counters()["peak_running"] == 1
        # a job larger than the whole budget is rejected at submission
        big = synthdata.uniform(2_000_000, 3, seed=1).astype(np.float32)
        with pytest.raises(wm.WMError) as e:
            srv.submit(big, kind="emst")
        assert e.value.code == -2
