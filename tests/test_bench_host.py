"""Host-side logic of bench.py that needs no GPU: the measured-traffic guard of the roofline and
the per-kernel roofline arithmetic.

A DRAM figure from an ncu capture may be reported only while the kernel's source file is the
measured version (its sha256); any edit of the file turns the figure into null.
"""
import hashlib
import os
import shutil
from types import SimpleNamespace

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = "paper_2104_01126_gb300/csrc/wspd.cu"


def _sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def test_traffic_scales_with_units_for_the_measured_source(monkeypatch):
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "getpairs",
                        {"bytes_per_unit": 12.5, "source": SRC, "sha256": _sha(os.path.join(ROOT, SRC))})
    assert bench.measured_traffic("getpairs", 1000) == 12500.0
    assert bench.measured_traffic("getpairs", 0) is None
    assert bench.measured_traffic("no-such-kernel", 1000) is None


def test_traffic_null_once_the_source_changes(tmp_path, monkeypatch):
    # a copy of the tree layout with one edited kernel source: the guard must see the change
    src = os.path.join(ROOT, SRC)
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "getpairs", {"bytes_per_unit": 1.0, "source": SRC, "sha256": _sha(src)})
    fake_root = tmp_path / "repo"
    dst = fake_root / SRC
    dst.parent.mkdir(parents=True)
    shutil.copyfile(src, dst)
    with open(dst, "ab") as f:
        f.write(b"\n// edited\n")
    fake_bench = fake_root / "bench.py"
    shutil.copyfile(os.path.join(ROOT, "bench.py"), fake_bench)
    monkeypatch.setattr(bench, "__file__", str(fake_bench))
    assert bench.measured_traffic("getpairs", 10) is None


def _stats(**kw):
    base = dict(getpairs_visits=0, ms_getpairs=0.0, getpairs_launches=0, getrho_visits=0, ms_getrho=0.0,
                bccp_evals=0, bccp_tile_evals=0, bccp_dual_evals=0, ms_bccp_group=0.0, ms_tile_kernel=0.0,
                ms_bccp_dual=0.0, knn_evals=0, ms_knn_kernel=0.0)
    base.update(kw)
    return SimpleNamespace(**base)


def test_kernel_rooflines_arithmetic():
    peaks = {"hbm_gbs": 1000.0, "hbm_basis": "test"}
    # d = 3: a visit moves 8 + 32 + 32 + 64 + 16 = 152 B; 10^9 visits in 1 s -> 152 GB/s
    s3 = _stats(getpairs_visits=10**9, ms_getpairs=1000.0, getpairs_launches=7,
                bccp_evals=3 * 10**9, bccp_tile_evals=10**9, bccp_dual_evals=10**9, ms_bccp_group=100.0,
                ms_tile_kernel=200.0, ms_bccp_dual=50.0)
    roof = bench.kernel_rooflines([(3, s3)], peaks, 50.0, "test")
    by = {k["kernel"].split(" ")[0]: k for k in roof["all"]}
    gp = by["findpair_dfs_kernel<1>"]
    assert abs(gp["achieved"] - 152.0) < 1e-9 and abs(gp["frac"] - 0.152) < 1e-12 and gp["launches"] == 7
    # group evaluations = all - tile - dual = 10^9, 8 flop each, in 0.1 s -> 0.08 TFLOP/s
    assert abs(by["bccp_group_kernel<1/8>"]["achieved"] - 0.08) < 1e-12
    assert abs(by["bccp_pair_tile_kernel"]["achieved"] - 0.04) < 1e-12
    assert abs(by["bccp_dual_kernel"]["frac"] - 0.16 / 50.0) < 1e-12
    assert roof["kernel"].startswith("findpair_dfs_kernel<1>")   # the most device time
    # measured traffic: bytes per visit x visits, per launch
    if bench.measured_traffic("getpairs", 1):
        per = bench.MEASURED_TRAFFIC["getpairs"]["bytes_per_unit"]
        assert abs(gp["traffic"] - per * 10**9 / 7) < 1e-3 * per
        assert abs(gp["traffic_total"] - per * 10**9) < 1e-3 * per
    # mutual reachability adds two maxima per evaluation
    roof_h = bench.kernel_rooflines([(3, s3)], peaks, 50.0, "test", hdb=True)
    byh = {k["kernel"].split(" ")[0]: k for k in roof_h["all"]}
    assert abs(byh["bccp_pair_tile_kernel"]["achieved"] - 0.05) < 1e-12


def test_visit_bytes_follow_the_box_stride():
    assert bench.visit_bytes(2) == bench.visit_bytes(4) == 152
    assert bench.visit_bytes(7) == 216
    assert bench.visit_bytes(16) == 344


def test_suite_is_the_eight_ten_million_point_sets():
    names = bench.workload_names("emst-10m-suite")
    assert len(names) == 8
    assert {bench.WORKLOADS[n]["d"] for n in names} == {2, 3, 5, 7}
    assert {bench.WORKLOADS[n]["gen"] for n in names} == {"uniform", "varden"}
    assert all(bench.WORKLOADS[n]["n"] == 10_000_000 for n in names)
