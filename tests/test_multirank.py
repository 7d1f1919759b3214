"""The N > 1 host logic of bench.py, as world-size-2 gloo ranks on the CPU.

bench.py --gpus N runs replicas: each rank solves its own problem, and the only
collective is the max over ranks of the timed region. The whole-job value is
every rank's iterations over that slowest time. The reference arm runs on
rank 0 alone; the other ranks exit 0 without output."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, times, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        t_max, value = bench.replica_throughput(times[rank], 5, 50, world, "cpu")
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"t_max": t_max, "value": value}, f)


def test_replica_throughput_takes_the_slowest_rank(tmp_path):
    times = [100.0, 250.0]  # ms of the timed region on each rank
    mp.spawn(rank_main, args=(2, free_port(), times, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["t_max"] == 250.0
        assert r["value"] == pytest.approx(2 * 5 * 50 / 0.25)  # all ranks' iterations


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    t_max, value = bench.replica_throughput(200.0, 4, 50, 1, "cpu")
    assert t_max == 200.0 and value == pytest.approx(1000.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(free_port()))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
