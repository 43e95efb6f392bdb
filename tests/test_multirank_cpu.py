"""The N > 1 bench paths on CPU.

Gloo ranks (127.0.0.1) run the bench's whole-job aggregation, which must
take the slowest rank's time and the sum of every rank's units, and the
placement of one batched sensor set on the ranks: every sensor owned by
exactly one rank, particle loads within one sensor of each other (greedy bin
packing, longest first), no data-path collective.  Replicas of the
single-sensor workload get disjoint seeds.  `bench.py --gpus 2` started
without ranks relaunches itself as two ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
import workloads as W
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
times = [10.0 + 5.0 * rank, 3.0 - rank]          # per-rank ms of two timed regions
all_specs = W.c2_instances(256, seed_base=1000)   # the batched workload's sensor set
sizes = [b.n_particles for b, _ in all_specs]
owners, loads = bench.shard_sensors(sizes, world)
mine = owners[rank]
units = sum(sizes[i] for i in mine)               # this rank's particles
(t0, t1), u = bench.reduce_over_ranks(times, units, world, "cpu")
reps = W.c2_instances(4, seed_base=1000 + 100000 * rank)   # replica seeds of another workload
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "t": [t0, t1], "u": u, "units": units, "mine": mine, "loads": loads,
                  "sizes": sizes, "rate": bench.whole_job_rate(u, t0 * 1e-3),
                  "replica_seeds": [b.seed for b, _ in reps]}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(world):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), REPO_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return outs


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_split_one_sensor_set_and_aggregate_like_the_bench(world):
    pytest.importorskip("torch")
    outs = _run_ranks(world)
    sizes = outs[0]["sizes"]
    total = sum(sizes)
    for o in outs:
        assert o["t"] == [10.0 + 5.0 * (world - 1), 3.0]   # max over ranks, per timed region
        assert o["u"] == total                               # every rank's particles, summed
        assert o["rate"] == pytest.approx(total / ((10.0 + 5.0 * (world - 1)) * 1e-3))
        assert o["loads"] == outs[0]["loads"]                # every rank computes the same split
    owned = sorted(i for o in outs for i in o["mine"])
    assert owned == list(range(len(sizes)))                  # each sensor exactly once
    loads = [o["units"] for o in outs]
    assert loads == outs[0]["loads"]
    assert max(loads) - min(loads) <= max(sizes)             # within one sensor of each other
    assert max(loads) <= total / world + max(sizes)
    seeds = [set(o["replica_seeds"]) for o in outs]
    for a in range(world):
        for b in range(a + 1, world):
            assert not seeds[a] & seeds[b]                   # replicas own their seeds


def test_bin_pack_is_longest_first_and_deterministic():
    from paper_2301_08343_gb300.sharding import bin_pack, round_robin
    owners, loads = bin_pack([5, 9, 1, 7, 3, 3], 2)
    # longest first: 9 -> r0, 7 -> r1, 5 -> r1 (12), 3 -> r0 (12), 3 -> r0 (15), 1 -> r1 (13)
    assert owners == [[1, 4, 5], [0, 2, 3]] and loads == [15, 13]
    assert bin_pack([4, 4, 4], 1) == ([[0, 1, 2]], [12])
    assert bin_pack([], 3) == ([[], [], []], [0, 0, 0])
    with pytest.raises(ValueError):
        bin_pack([1], 0)
    assert round_robin(7, 3, 1) == [1, 4]


@pytest.mark.timeout(300)
def test_bench_gpus_2_relaunches_as_two_ranks():
    """The reference arm needs no GPU: started with --gpus 2 and no ranks,
    bench.py runs again under torch.distributed.run as two ranks; rank 0
    prints the one JSON line, the other rank exits 0."""
    pytest.importorskip("torch")
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--workload", "c0"],
                       env=env, capture_output=True, text=True, timeout=280, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(x) for x in r.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
