"""The multi-GPU path of the benchmark is independent replicas: each rank
projects its own seeded batch with the same robot, constraints and obstacles,
and only the step time (max) and the converged count (sum) cross ranks.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl, q, name, _ = bench.make_workload("arm", rank)
    ms, conv = bench.aggregate_replicas(1.0 + rank, 100 + 10 * rank, world, torch.device("cpu"))
    out[rank] = (ms, conv, float(q[0, 0]), float(wl.robot.X[3, 11]), float(wl.obstacles.spheres[0, 0]), name)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_on_cpu():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 2.0           # slowest rank's time
    assert r0[1] == r1[1] == 210.0         # converged projections summed
    assert r0[2] != r1[2]                  # each rank projects its own batch
    assert r0[3] == r1[3] and r0[5] == r1[5]   # ... of the same robot model and workload
