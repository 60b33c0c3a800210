"""mcp_project_segments_noalloc: the allocation-free segment projection.

Some callers cannot allocate device memory once they are running: a real-time
planning or whole-body control loop, where a cudaMalloc adds unbounded latency
and synchronises the device, or code whose device memory is owned by another
allocator or budget.  For them the library keeps the segment projection's
scratch (work counter and segment offsets) in a fixed device array.  This
test calls that entry point through the C ABI, on a context that never ran
the allocating variant, twice in a row, checks each result against
mcp_project_segments on a second context, and checks with the library's
allocation counter that neither call allocated device memory.  Kept in a file
of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

Q_TOL = 1e-4   # the parity tolerance used throughout the GPU tests (rad)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_2604_13323_gb300 import build, mcproj
    from paper_2604_13323_gb300 import workloads as W

    build.build()
    lib = mcproj.load_library()
    wl = W.dual_arm_workload(total=30000)
    ex = wl.extra
    ref_ctx = mcproj.Projector(wl.robot, wl.constraints)
    starts = ref_ctx.project(torch.tensor(ex["raw_start"], dtype=torch.float32, device="cuda"), wl.params)[0]
    delta = torch.tensor(ex["raw_dir"] * ex["step"], dtype=torch.float32, device="cuda")
    length = torch.tensor(ex["lengths"], dtype=torch.int32, device="cuda")
    n_seg = int(length.shape[0])
    total = int(ex["lengths"].sum())
    q_ref, f_ref, i_ref, r_ref = ref_ctx.project_segments(starts, delta, length, wl.params)
    torch.cuda.synchronize()
    q_ref, f_ref, r_ref = q_ref.cpu().numpy(), f_ref.cpu().numpy(), r_ref.cpu().numpy()
    assert ((f_ref & mcproj.F_CONVERGED) != 0).mean() > 0.99

    fresh = mcproj.Projector(wl.robot, wl.constraints)   # no allocating segment call on this context
    pp = mcproj.Projector.params(wl.params)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for call in range(2):   # the caller's buffers, allocated before the calls
        outs.append((torch.full((14, total), float("nan"), dtype=torch.float32, device="cuda"),
                     torch.full((total,), 255, dtype=torch.uint8, device="cuda"),
                     torch.zeros(total, dtype=torch.uint8, device="cuda"),
                     torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    allocs = lib.mcp_alloc_count()   # the library's device allocations so far (all contexts)
    for call in range(2):
        out, fl, it, res = outs[call]
        st = lib.mcp_project_segments_noalloc(fresh.h, ctypes.byref(pp), n_seg, n_seg, _p(starts), _p(delta),
                                              _p(length), total, total, _p(out), _p(fl), _p(it), _p(res), stream)
        assert st == mcproj.MCP_OK, lib.mcp_last_error(fresh.h)
        torch.cuda.synchronize()
        q, f, r = out.cpu().numpy(), fl.cpu().numpy(), res.cpu().numpy()
        np.testing.assert_array_equal(f, f_ref)
        conv = (f & mcproj.F_CONVERGED) != 0
        assert np.abs(q[:, conv] - q_ref[:, conv]).max() <= Q_TOL, call
        assert (r[conv] < wl.params.tol).all()
        assert lib.mcp_alloc_count() == allocs, call   # neither call allocated device memory


def test_noalloc_rejects_oversized_batch():
    from paper_2604_13323_gb300 import build, mcproj
    from paper_2604_13323_gb300 import workloads as W

    build.build()
    lib = mcproj.load_library()
    wl = W.dual_arm_workload(total=10)
    ctx = mcproj.Projector(wl.robot, wl.constraints)
    pp = mcproj.Projector.params(wl.params)
    big = 65536 + 1
    dummy = torch.zeros(1, device="cuda")
    st = lib.mcp_project_segments_noalloc(ctx.h, ctypes.byref(pp), big, big, _p(dummy), _p(dummy), _p(dummy), 1, 1,
                                          _p(dummy), _p(dummy), _p(dummy), _p(dummy),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == mcproj.MCP_ERR_ARG
    assert b"allocation-free limit" in lib.mcp_last_error(ctx.h)
