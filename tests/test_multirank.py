"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

The method needs no exchange between GPUs: every rank runs an independent replica.  What the
ranks share is the timing protocol: the slowest rank's time is the job's time, and only rank 0
prints.  Both are checked here with two gloo processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == 15.0 and out[1] == 15.0


def test_reference_arm_prints_on_rank0_only():
    lines = {}
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2")
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                            "--steps", "1", "--warmup", "3", "--workload", "tgv16"],
                           capture_output=True, text=True, env=env, timeout=600)
        assert r.returncode == 0, r.stderr
        lines[rank] = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert lines[1] == []
    d = json.loads(lines[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
