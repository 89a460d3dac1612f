"""The N > 1 path of bench.py: independent replicas, one per rank, the job's
time the slowest rank's (max over ranks), throughput = all units / that time.
Runs two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed (1 + r) seconds and an end-to-end (2 + r) seconds
    t, e2e = bench.max_over_ranks([1.0 + rank, 2.0 + rank], device="cpu")
    out[rank] = (t, e2e, bench.replica_throughput(world, 10, 3, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        t, e2e, thr = res[r]
        assert t == 2.0 and e2e == 3.0  # the slowest rank's times, on every rank
        assert thr == world * 10 * 3 / 2.0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.5], device="cpu") == [1.5, 2.5]
    assert bench.replica_throughput(1, 10, 3, 2.0) == 15.0
