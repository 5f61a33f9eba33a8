"""The N > 1 host logic of bench.py on CPU: two gloo ranks, each with its own replica box.  Every rank
must see the slowest rank's time, the whole-job rate counts the units of all ranks, replicas get
distinct seeds, and only rank 0 runs the reference arm."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO"])
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
print(json.dumps({"rank": rank, "world": world, "ms_max": ms, "rate": bench.whole_job_rate(world, 1000, ms),
                  "seed": bench.replica_seed(rank)}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), REPO=ROOT)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_two_gloo_ranks_agree_on_the_slowest_time_and_count_all_units():
    world, port = 2, _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER], env=_env(r, world, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(world)]
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["ms_max"] for d in outs] == [15.0, 15.0]          # the slowest rank's time on every rank
    assert all(abs(d["rate"] - 2 * 1000 / 15e-3) < 1e-6 for d in outs)
    assert outs[0]["seed"] != outs[1]["seed"]


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 1000, 2.0) == 5e5


def test_reference_arm_runs_on_rank_zero_only():
    env = _env(1, 2, _free_port())
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
