"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) run the bench's
whole-job aggregation, which must take the slowest rank's time and the sum of
every rank's units, and the workloads each rank builds must be disjoint
shards (different seeds), so that no data-path collective is needed."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
import workloads as W
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
times = [10.0 + 5.0 * rank, 3.0 - rank]          # per-rank ms of two timed regions
units = 1000 * (rank + 1)                          # uneven per-rank work
(t0, t1), u = bench.reduce_over_ranks(times, units, world, "cpu")
specs = W.c2_instances(4, seed_base=1000 + 100000 * rank)
sig = [[b.nx, b.ny, b.nz, b.seed] for b, _ in specs]
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "t": [t0, t1], "u": u,
                  "rate": bench.whole_job_rate(u, t0 * 1e-3), "specs": sig}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.timeout(300)
def test_two_gloo_ranks_aggregate_like_the_bench():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), REPO_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == [15.0, 3.0]          # max over ranks, per timed region
        assert o["u"] == 3000.0               # 1000 + 2000
        assert o["rate"] == pytest.approx(3000.0 / 15e-3)
    assert outs[0]["specs"] != outs[1]["specs"]  # each rank owns its own sensors
    seeds0 = {s[3] for s in outs[0]["specs"]}
    seeds1 = {s[3] for s in outs[1]["specs"]}
    assert not seeds0 & seeds1
