"""The N > 1 path of bench.py on CPU: two ranks over gloo (world_size 2).

bench.py runs one independent replica per GPU ("replicas only": the method has no exchange
step), reports the max-over-ranks step time and the whole-job value.  These tests drive that
reduction and the reference arm's rank handling with two CPU processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo", init_method="env://")
local = [12.5, 40.0][rank]
ms = bench.max_over_ranks(local, dist)
val = bench.whole_job_value(1_000_000, dist.get_world_size(), ms)
print(json.dumps({"rank": rank, "ms": ms, "value": val}))
dist.destroy_process_group()
'''


def _run_two(code, extra_args=()):
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_whole_job_value_world_size_two():
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _run_two(WORKER)]
    for o in outs:
        assert o["ms"] == 40.0                       # the slower replica decides
        assert abs(o["value"] - 2 * 1_000_000 / 0.040 / 1e6) < 1e-9


REF = r'''
import os, sys
sys.path.insert(0, sys.argv[1])
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-warmup", "0",
            "--ref-sample", "2000", "--gpus", "2"]
import bench
bench.main()
'''


def test_reference_arm_prints_only_on_rank_zero():
    outs = _run_two(REF)
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    rec = json.loads(lines0[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
