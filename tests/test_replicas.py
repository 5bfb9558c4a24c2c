"""The multi-GPU form of the benchmark runs independent replicas (the step
does not shard): the job's time is the slowest rank's and its work the leaf
updates of all ranks.  Checked with two gloo ranks on the CPU; the reference
arm under a launcher prints from rank 0 only."""
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


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, leaves = bench.aggregate_replicas(dist, 10.0 + 5.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
        out[rank] = (ms, leaves)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r] == (15.0, 3000.0)  # max of 10 and 15 ms; 1000 + 2000 updates


def test_single_rank_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(None, 7.0, 123, None) == (7.0, 123)


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
