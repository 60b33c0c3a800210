"""Failure paths of the C ABI, made to fail on the host (no kernel faults):
an injected device-allocation failure returns MCP_ERR_OOM and leaves the
context usable; an injected CUDA error of a launch returns MCP_ERR_CUDA with
the label in mcp_last_error and leaves the context usable; the library's
allocation counter moves only when something is allocated."""
import os

import pytest

torch = pytest.importorskip("torch")

from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


@pytest.fixture
def env():
    saved = {k: os.environ.get(k) for k in ("MCP_TEST_FAIL_ALLOC", "MCP_TEST_FAIL_CUDA")}
    yield os.environ
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def test_obstacle_allocation_failure_is_oom_and_recoverable(mcproj, env):
    wl = W.arm_workload(n=256)
    P = mcproj.Projector(wl.robot, wl.constraints)
    q = torch.tensor(f32_exact(wl.q), dtype=torch.float32, device="cuda")
    env["MCP_TEST_FAIL_ALLOC"] = "obstacles"
    with pytest.raises(mcproj.MCPError) as e:
        P.load_obstacles(wl.obstacles)
    assert e.value.status == mcproj.MCP_ERR_OOM and "obstacles" in str(e.value)
    with pytest.raises(mcproj.MCPError) as e:    # no scene: the check refuses, nothing runs
        P.check(q)
    assert e.value.status == mcproj.MCP_ERR_STATE
    out = P.project(q, wl.params)                # projection needs no obstacles: still works
    torch.cuda.synchronize()
    assert ((out[1].cpu().numpy() & mcproj.F_CONVERGED) != 0).mean() > 0.99
    del env["MCP_TEST_FAIL_ALLOC"]
    P.load_obstacles(wl.obstacles)               # and the next load succeeds
    ref = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    assert torch.equal(P.check(out[0]), ref.check(out[0]))


def test_segment_offset_allocation_failure_is_oom_and_recoverable(mcproj, env):
    wl = W.dual_arm_workload(total=3000)
    ex = wl.extra
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    starts = P.project(torch.tensor(ex["raw_start"], dtype=torch.float32, device="cuda"), wl.params)[0]
    delta = torch.tensor(ex["raw_dir"] * ex["step"], dtype=torch.float32, device="cuda")
    length = torch.tensor(ex["lengths"], dtype=torch.int32, device="cuda")
    env["MCP_TEST_FAIL_ALLOC"] = "segment offsets"
    with pytest.raises(mcproj.MCPError) as e:
        P.project_segments(starts, delta, length, wl.params)
    assert e.value.status == mcproj.MCP_ERR_OOM
    del env["MCP_TEST_FAIL_ALLOC"]
    got = P.project_segments(starts, delta, length, wl.params)
    ref = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles).project_segments(starts, delta, length, wl.params)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_injected_launch_error_is_reported_and_the_context_stays_usable(mcproj, env):
    wl = W.arm_workload(n=1024)
    q = torch.tensor(f32_exact(wl.q), dtype=torch.float32, device="cuda")
    env["MCP_TEST_FAIL_CUDA"] = "project_batch launch"
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)   # reads the hook at creation
    del env["MCP_TEST_FAIL_CUDA"]
    with pytest.raises(mcproj.MCPError) as e:
        P.project(q, wl.params)
    assert e.value.status == mcproj.MCP_ERR_CUDA and "project_batch launch" in str(e.value)
    hit = P.check(q)                             # other calls of the same context still work
    ref = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    assert torch.equal(hit, ref.check(q))
    out = ref.project(q, wl.params)              # and a context created without the hook projects
    torch.cuda.synchronize()
    assert ((out[1].cpu().numpy() & mcproj.F_CONVERGED) != 0).mean() > 0.99


def test_allocation_count_moves_only_on_allocation(mcproj):
    wl = W.arm_workload(n=512)
    n0 = mcproj.alloc_count()
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    assert mcproj.alloc_count() > n0             # the context's model, tables, obstacles
    q = torch.tensor(f32_exact(wl.q), dtype=torch.float32, device="cuda")
    out = P.project_check(q, wl.params)          # first calls may set up per-context data
    P.check(out[0])
    torch.cuda.synchronize()
    n1 = mcproj.alloc_count()
    for _ in range(3):
        out = P.project_check(q, wl.params)
        P.check(out[0])
        P.project(q, wl.params)
    torch.cuda.synchronize()
    assert mcproj.alloc_count() == n1            # batch calls allocate nothing
