"""The multi-GPU path of the benchmark is replicas only: every rank solves its
own seeded instance and the step time is the slowest rank's.  Its host logic
(instance per rank, max over ranks) runs here as two gloo processes on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_setup()
        t = bench.max_over_ranks(1.5 + rank)  # rank 1 is the slow one
        p, idx = bench.replica_problem(rank, n=2048)
        dist.barrier()
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), w=w, r=r, t=t, X=p.X, y=p.y, idx=idx)
    finally:
        dist.destroy_process_group()


def test_replicas_two_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npz")
    r1 = np.load(tmp_path / "r1.npz")
    assert int(r0["w"]) == 2 and int(r0["r"]) == 0 and int(r1["r"]) == 1
    # every rank reports the slowest rank's time
    assert float(r0["t"]) == 2.5 and float(r1["t"]) == 2.5
    # each rank has its own instance of the same workload
    assert r0["X"].shape == r1["X"].shape == (2048, 8)
    assert not np.array_equal(r0["X"], r1["X"])
    assert not np.array_equal(r0["idx"], r1["idx"])


def test_max_over_ranks_without_a_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
