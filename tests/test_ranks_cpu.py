"""Multi-rank host logic of bench.py on CPU: two gloo ranks (one process per
rank, rendezvous on 127.0.0.1) aggregate their replica timings into the
whole-job throughput, and the reference arm does its work on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank()
ms_local = [12.0, 20.0][rank]
ms, value = bench.aggregate_ranks(ms_local, 50, dist.get_world_size(), dist, "cpu")
print(json.dumps({"rank": rank, "ms": ms, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, nproc=2, extra=()):
    port = _free_port()
    procs = []
    for r in range(nproc):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(nproc), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_rank():
    import json
    outs = _run_ranks(WORKER)
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["ms"] == 20.0                      # max over ranks
        assert abs(r["value"] - 2 * 50 / 0.020) < 1e-9   # all ranks' solves / job time


def test_reference_arm_works_on_rank0_only():
    code = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import bench
class A: steps, warmup, gpus = 1, 0, 2
if os.environ["RANK"] != "0":
    bench.run_reference(A)          # returns at once without work or output
    print("done")
"""
    outs = _run_ranks(code)
    assert outs[1].strip() == "done"
