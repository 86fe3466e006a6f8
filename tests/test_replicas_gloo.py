"""The multi-rank path of bench.py (replicas, one process per GPU): the job's
time is the maximum over ranks.  Two gloo ranks on the CPU, started as
separate processes with a rendezvous on 127.0.0.1."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=int(os.environ["WORLD_SIZE"]))
import bench
rank = dist.get_rank()
print("RESULT", rank, bench.ranks_max(1.5 + 2.0 * rank, dist, "cpu"), bench.ranks_max(7.0 - rank, dist, "cpu"))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_ranks_max_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    results = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        line = [l for l in out.splitlines() if l.startswith("RESULT")][0].split()
        results.append((int(line[1]), float(line[2]), float(line[3])))
    assert sorted(results) == [(0, 3.5, 7.0), (1, 3.5, 7.0)]


def test_ranks_max_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_max(4.25, None, "cpu") == 4.25
