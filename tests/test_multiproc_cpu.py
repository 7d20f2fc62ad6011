"""The N > 1 path of bench.py, on CPU: ranks are independent replicas (no
data-path collective); the job's time is the slowest rank's, the rate sums
the replicas, and the reference arm runs on rank 0 alone.  world_size 2 over
gloo on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist)          # rank 1 is the slow one
    rate = bench.replica_rate(world, 1000, 10, t)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_rate(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["t"] == 2.0                           # every rank sees the slowest time
        assert d["rate"] == world * 1000 * 10 / 2.0    # whole-job rate sums the replicas


def test_reference_arm_prints_on_rank0_only(tmp_path):
    """Under torchrun the reference arm (the oracle) runs on rank 0 and the
    other ranks exit 0 without work or output."""
    outs = []
    for rank in (1, 0):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1")
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                            "--workload", "config0", "--steps", "1", "--warmup", "0"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(r.stdout.strip())
    assert outs[0] == ""
    line = json.loads(outs[1].splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
