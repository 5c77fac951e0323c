"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Machines and requests are independent, so N GPUs run N replicas with no
exchange on the data path. What the ranks share is host logic: the barrier,
the job time as the maximum over ranks, the whole-job rate (units of all
ranks over that time), and a launcher under which only rank 0 prints. These
tests run that logic on two CPU processes.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t_max = bench._max_over_ranks(1.5 + rank, world)  # rank 1 is the slow one
        rate = bench._whole_job_rate(1000.0, t_max, world)
        q.put((rank, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    # both ranks see the slowest rank's time; the job did 2 x 1000 units in it
    assert [g[1] for g in got] == [2.5, 2.5]
    assert [g[2] for g in got] == [800.0, 800.0]


def test_one_rank_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(3.25, 1) == 3.25
    assert bench._whole_job_rate(10.0, 2.0, 1) == 5.0


def test_reference_arm_under_the_launcher_prints_once():
    # the launch line the two-GPU bench uses, on CPU: rank 0 times the oracle, rank 1 exits 0
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--config", "0", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"
