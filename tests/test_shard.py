"""Sharding one batch over ranks: the partitions, and a world-size-2 gloo run
(two CPU processes) whose gathered outputs are bit-identical to the
unsharded run.  On the CPU the per-rank projector is the FP64 oracle (the
only projector without a GPU); what is tested is the partition and the
gather, which do not depend on the projector because every configuration is
projected independently.  tests/test_gpu_shard.py checks the same
independence for the CUDA kernels on one GPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_13323_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("n,world", [(0, 2), (1, 2), (7, 3), (65536, 2), (65537, 8), (5, 8)])
def test_batch_ranges_cover_contiguously(n, world):
    r = shard.batch_ranges(n, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
    assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_segment_ranges_keep_segments_whole_and_balance_points(world):
    rng = np.random.default_rng(3)
    lengths = rng.integers(2, 201, 2644)
    lengths[[5, 17]] = 0                       # empty segments are allowed
    r = shard.segment_ranges(lengths, world)
    assert r[0][0] == 0 and r[-1][1] == lengths.size
    assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
    pts = [int(lengths[a:b].sum()) for a, b in r]
    assert sum(pts) == lengths.sum()
    # each run ends at the boundary nearest its share: off by at most one segment
    assert max(pts) - min(pts) <= 2 * lengths.max()
    pr = shard.point_ranges(lengths, r)
    assert pr[0][0] == 0 and pr[-1][1] == lengths.sum()
    assert all(pr[i][1] == pr[i + 1][0] for i in range(world - 1))


def test_segment_ranges_with_fewer_segments_than_ranks():
    r = shard.segment_ranges([10, 3], 4)
    assert r[0][0] == 0 and r[-1][1] == 2 and sum(b - a for a, b in r) == 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_2604_13323_gb300 import workloads as W
    # a plain batch: contiguous ranges of the arm workload
    wl = W.arm_workload(n=2051)
    q = np.asarray(wl.q, np.float32).astype(np.float64)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    rr = shard.batch_ranges(q.shape[1], world)
    a, b = rr[rank]
    qo, fo, io, ro = O.project_params(q[:, a:b], wl.params, threads=1)
    hit, _ = O.check(qo, threads=1)
    full = shard.gather_columns([qo, fo, io, ro, hit], rr, q.shape[1])
    # uneven segments: runs of whole segments balanced by their lengths
    ws = W.dual_arm_workload(total=3000)
    ex = ws.extra
    Os = orc.Oracle(ws.robot, ws.constraints)
    seg = W.make_segments(Os.project_params(ex["raw_start"], ws.params, threads=1)[0], ex["raw_dir"],
                          ex["lengths"], ex["step"])
    sr = shard.segment_ranges(seg.length, world)
    s0, s1 = sr[rank]
    mine = W.Segments(start=seg.start[:, s0:s1], delta=seg.delta[:, s0:s1], length=seg.length[s0:s1])
    pts = W.segment_points(mine)
    so = Os.project_params(pts, ws.params, threads=1)
    fulls = shard.gather_columns(list(so), shard.point_ranges(seg.length, sr), int(seg.length.sum()))
    out[rank] = (full, fulls, (a, b), (s0, s1))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gather_bit_identical_outputs():
    from oracle import oracle as orc
    from paper_2604_13323_gb300 import workloads as W
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[2] != r1[2] and r0[3] != r1[3]      # the ranks projected different parts
    # the unsharded run, in this process
    wl = W.arm_workload(n=2051)
    q = np.asarray(wl.q, np.float32).astype(np.float64)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    ref = list(O.project_params(q, wl.params))
    ref.append(O.check(ref[0])[0])
    for got0, got1, want in zip(r0[0], r1[0], ref):
        np.testing.assert_array_equal(got0, want)
        np.testing.assert_array_equal(got1, want)
    ws = W.dual_arm_workload(total=3000)
    ex = ws.extra
    Os = orc.Oracle(ws.robot, ws.constraints)
    seg = W.make_segments(Os.project_params(ex["raw_start"], ws.params, threads=1)[0], ex["raw_dir"],
                          ex["lengths"], ex["step"])
    refs = Os.project_params(W.segment_points(seg), ws.params)
    for got0, got1, want in zip(r0[1], r1[1], refs):
        np.testing.assert_array_equal(got0, want)
        np.testing.assert_array_equal(got1, want)
