"""Sharded projection on one GPU: the parts a batch splits into (contiguous
configuration ranges; runs of whole segments balanced by their lengths) are
projected by separate calls, one after the other, as separate ranks would
project them, and their outputs, put side by side, are bit-identical to the
unsharded call's -- each configuration's result depends on nothing else in
the launch.  (No kernel here waits on another: the ranks of a real sharded
run are separate processes on separate GPUs.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_13323_gb300 import shard  # noqa: E402
from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


def _batch(name):
    if name == "arm":
        return W.arm_workload(n=65536)
    if name == "humanoid":
        return W.humanoid_workload(n=65537)
    return W.dual_arm_workload(total=10, n_random=40000)


@pytest.mark.parametrize("name", ["arm", "humanoid", "dual_arm"])
@pytest.mark.parametrize("world", [2, 3])
def test_batch_shards_equal_the_unsharded_call(mcproj, name, world):
    wl = _batch(name)
    q = torch.tensor(f32_exact(wl.q), dtype=torch.float32, device="cuda")
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    ref = P.project_check(q, wl.params)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in ref]
    parts = []
    ranges = shard.batch_ranges(q.shape[1], world)
    for a, b in ranges:
        out = P.project_check(q[:, a:b].contiguous(), wl.params)
        torch.cuda.synchronize()
        parts.append([t.cpu().numpy() for t in out])
    for k in range(5):   # q*, flags, iters, resid, in_collision
        got = np.concatenate([p[k] for p in parts], axis=-1)
        np.testing.assert_array_equal(got, ref[k])


@pytest.mark.parametrize("world", [2, 4])
def test_segment_shards_equal_the_unsharded_call(mcproj, world):
    wl = W.dual_arm_workload()
    ex = wl.extra
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    starts = P.project(torch.tensor(ex["raw_start"], dtype=torch.float32, device="cuda"), wl.params)[0]
    delta = torch.tensor(ex["raw_dir"] * ex["step"], dtype=torch.float32, device="cuda")
    length = torch.tensor(ex["lengths"], dtype=torch.int32, device="cuda")
    ref = [t.cpu().numpy() for t in P.project_segments(starts, delta, length, wl.params)]
    sr = shard.segment_ranges(ex["lengths"], world)
    pr = shard.point_ranges(ex["lengths"], sr)
    parts = []
    for a, b in sr:
        out = P.project_segments(starts[:, a:b].contiguous(), delta[:, a:b].contiguous(), length[a:b].contiguous(),
                                 wl.params)
        parts.append([t.cpu().numpy() for t in out])
    sizes = [b - a for a, b in pr]
    assert max(sizes) - min(sizes) <= 2 * int(ex["lengths"].max())
    for k in range(4):
        got = np.concatenate([p[k] for p in parts], axis=-1)
        np.testing.assert_array_equal(got, ref[k])
