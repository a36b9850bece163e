"""Replicas on several processes (the N > 1 path of the benchmark) with gloo on CPU:
distinct problems per rank, the slowest rank's time on every rank, whole-job rate."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
from paper_1807_10151_gb300 import replicas
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
local = 1.0 + 0.5 * rank                      # rank 1 is the slow one
t = replicas.slowest(local, dist)
dist.barrier()
print(json.dumps({"rank": rank, "seeds": replicas.rank_seeds(rank, 2001, 2501), "t": t,
                  "rate": replicas.job_rate(10, world, t)}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    assert [o["t"] for o in outs] == [1.5, 1.5]                 # max over ranks, on every rank
    assert [o["rate"] for o in outs] == [10 * 2 / 1.5] * 2      # whole-job units / slowest time
    assert outs[0]["seeds"] != outs[1]["seeds"]                  # independent problems


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    from paper_1807_10151_gb300 import replicas
    assert replicas.slowest(0.25) == 0.25
    assert replicas.job_rate(100, 1, 0.5) == 200.0
