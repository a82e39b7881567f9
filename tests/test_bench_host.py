"""Host-side logic of bench.py that needs no GPU: the measured-traffic guard of the roofline.

A DRAM figure from the committed ncu launch list may be reported only for the workload it was
measured on and only while the kernel's source file is the measured version (its sha256); any
edit of the file turns the figure into null.
"""
import hashlib
import os
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_reported_for_the_measured_sources():
    for key, t in bench.MEASURED_TRAFFIC.items():
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
        want = t["bytes"] if h == t["sha256"] else None
        assert bench.measured_traffic(key, bench.TRAFFIC_WORKLOAD) == want, key


def test_traffic_null_for_other_workloads_and_kernels():
    assert bench.measured_traffic("bccp", "emst-uniform-10m-3d") is None
    assert bench.measured_traffic("no-such-kernel", bench.TRAFFIC_WORKLOAD) is None


def test_traffic_null_once_the_source_changes(tmp_path, monkeypatch):
    # a copy of the tree layout with one edited kernel source: the guard must see the change
    t = bench.MEASURED_TRAFFIC["bccp"]
    src = os.path.join(ROOT, t["source"])
    fake_root = tmp_path / "repo"
    dst = fake_root / t["source"]
    dst.parent.mkdir(parents=True)
    shutil.copyfile(src, dst)
    with open(dst, "ab") as f:
        f.write(b"\n// edited\n")
    fake_bench = fake_root / "bench.py"
    shutil.copyfile(os.path.join(ROOT, "bench.py"), fake_bench)
    monkeypatch.setattr(bench, "__file__", str(fake_bench))
    assert bench.measured_traffic("bccp", bench.TRAFFIC_WORKLOAD) is None
