"""Multi-GPU runs are independent replicas (one LP instance per rank, no data-path
collective); the only exchange is the benchmark's whole-job aggregation: the
slowest rank's time and the sum of all ranks' iterations.  Checked here with two
gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
import lpgen
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
secs = [1.5, 2.25][rank]
iters = [1000, 1200][rank]
launches = [3000, 3700][rank]
out = bench.aggregate_over_ranks(dist, secs, iters, launches, "cpu")
single = bench.aggregate_over_ranks(None, secs, iters, launches, "cpu")
# each rank draws its own instance (replicas do not share data)
inst = lpgen.config1(instance=rank, scale=1e-4)
print(json.dumps({"rank": rank, "out": out, "single": single, "c0": float(inst.c[0]),
                  "nnz": int(inst.nnz)}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replica_aggregation_two_gloo_ranks(tmp_path):
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, BENCH_ROOT=ROOT, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="",
                   OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        so, se = p.communicate(timeout=300)
        assert p.returncode == 0, se[-2000:]
        outs.append(json.loads([ln for ln in so.splitlines() if ln.startswith("{")][-1]))
    outs.sort(key=lambda d: d["rank"])
    for d in outs:
        secs, iters, launches = d["out"]
        assert secs == 2.25                      # max over ranks
        assert iters == 2200.0 and launches == 6700.0  # sums over ranks
        # whole-job throughput = all ranks' iterations / slowest rank's time
        assert np.isclose(iters / secs, 2200 / 2.25)
    assert outs[0]["single"] == [1.5, 1000.0, 3000.0]
    assert outs[1]["single"] == [2.25, 1200.0, 3700.0]
    assert outs[0]["c0"] != outs[1]["c0"]
