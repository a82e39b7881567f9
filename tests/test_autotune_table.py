"""The autotuner's table (csrc/tuning_table.inc) on the host: written from rows, compiled with the
header, and queried.  A call takes the rows of its problem (HDBSCAN* falls back to the EMST rows),
the nearest tuned dimension, then the smallest tuned size at or above n (else the largest)."""
import os
import shutil
import subprocess

import pytest

from paper_2104_01126_gb300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MAIN = r'''
#include <cstdio>
#include <cstdlib>
#include "wspdmst.h"
#include TABLE
int main(int argc, char **argv) {
    wm_tuning t{};
    builtin_tuning(atoll(argv[1]), atoi(argv[2]), atoi(argv[3]), &t);
    printf("%d %d\n", t.dfs_budget, t.combined);
    return 0;
}
'''


def _row(problem, d, n, budget, combined=0):
    p = dict(autotune.DEFAULTS)
    p.update(dfs_budget=budget, combined=combined)
    return {"problem": problem, "d": d, "n": n, "default_ms": 1.0, "tuned_ms": 1.0, "params": p}


@pytest.fixture(scope="module")
def query(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    tmp = tmp_path_factory.mktemp("tune")
    rows = [_row("emst", 2, 100_000, 4), _row("emst", 2, 10_000_000, 16), _row("emst", 7, 1_000_000, 32, 1),
            _row("hdbscan", 3, 1_000_000, 2)]
    inc = tmp / "table.inc"
    autotune.write_table(rows, str(inc))
    src = tmp / "main.cpp"
    src.write_text(MAIN)
    exe = tmp / "q"
    subprocess.run(["g++", "-std=c++17", f'-DTABLE="{inc}"', "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)

    def q(n, d, mp):
        out = subprocess.run([str(exe), str(n), str(d), str(mp)], capture_output=True, text=True, check=True).stdout
        return tuple(int(v) for v in out.split())
    return q


def test_nearest_dimension_and_size_bucket(query):
    assert query(50_000, 2, 0) == (4, 0)          # smallest tuned size >= n
    assert query(2_000_000, 2, 0) == (16, 0)
    assert query(10**9, 2, 0) == (16, 0)          # beyond every tuned size: the largest
    assert query(10**9, 3, 0) == (16, 0)          # d = 3 is nearest to 2 among {2, 7}
    assert query(1000, 6, 0) == (32, 1)           # d = 6 is nearest to 7


def test_hdbscan_rows_and_fallback(query):
    assert query(10**5, 3, 10) == (2, 0)          # HDBSCAN* has its own rows
    assert query(10**5, 3, 1) == (4, 0)           # minPts <= 1 is an EMST


def test_empty_table_gives_defaults(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    inc = tmp_path / "t.inc"
    autotune.write_table([], str(inc))
    src = tmp_path / "m.cpp"
    src.write_text(MAIN)
    exe = tmp_path / "q"
    subprocess.run(["g++", "-std=c++17", f'-DTABLE="{inc}"', "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe), "1000", "3", "0"], capture_output=True, text=True, check=True).stdout
    assert tuple(int(v) for v in out.split()) == (autotune.DEFAULTS["dfs_budget"], autotune.DEFAULTS["combined"])


def test_merge_keeps_the_rows_not_retuned():
    old = [_row("emst", 2, 100_000, 4), _row("emst", 7, 1_000_000, 8), _row("hdbscan", 7, 1_000_000, 8)]
    new = [_row("emst", 7, 1_000_000, 32)]
    got = autotune.merge_rows(old, new)
    assert len(got) == 3
    by = {(r["problem"], r["d"], r["n"]): r["params"]["dfs_budget"] for r in got}
    assert by[("emst", 7, 1_000_000)] == 32 and by[("emst", 2, 100_000)] == 4 and by[("hdbscan", 7, 1_000_000)] == 8


def test_rows_without_a_newer_field_take_its_default(tmp_path):
    # a report written before a field existed still gives a complete table
    r = _row("emst", 3, 1_000_000, 4)
    del r["params"]["edges_per_point"]
    path = tmp_path / "t.inc"
    autotune.write_table([r], str(path))
    line = [x for x in path.read_text().splitlines() if x.startswith("    {0, 3, 1000000LL")][0]
    assert line.split("}")[0].split(",")[-1].strip() == str(autotune.DEFAULTS["edges_per_point"])
