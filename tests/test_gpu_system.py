"""GPU tests of the batching and differentiation patterns around the kernels:
autotuning, CUDA-graph replay of the segment projection, the autograd wrapper
of projection + VJP, and path shortening on the manifold."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_autotune_keeps_results(mcproj):
    wl = W.arm_workload(n=8192)
    P = mcproj.Projector(wl.robot, wl.constraints)
    q = dev(f32_exact(wl.q))
    before = [t.clone() for t in P.project(q, wl.params)]
    tpb, bps, chunk, fuse, tpc = P.autotune(q, wl.params)
    assert tpb in (64, 128, 256) and bps in (1, 2, 4, 8) and chunk in (16, 32, 64) and fuse in (0, 1)
    assert tpc == 1  # the arm has one kernel shape per configuration
    after = P.project(q, wl.params)
    torch.cuda.synchronize()
    for x, y in zip(before, after):
        assert torch.equal(x, y)


def test_segment_graph_replay_and_recapture(mcproj):
    wl = W.dual_arm_workload(total=20000)
    ex = wl.extra
    P = mcproj.Projector(wl.robot, wl.constraints)
    starts = P.project(dev(ex["raw_start"]), wl.params)[0]
    delta = dev(ex["raw_dir"] * ex["step"])
    length = dev(ex["lengths"], torch.int32)
    total = int(ex["lengths"].sum())
    outs = []
    for rep in range(3):   # first call captures, the next ones replay the graph
        outs.append([t.clone() for t in P.project_segments(starts, delta, length, wl.params)])
    torch.cuda.synchronize()
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert torch.equal(x, y)
    # new inputs through the same buffers: the replayed graph reads them
    delta.mul_(0.5)
    o2 = P.project_segments(starts, delta, length, wl.params)
    ref = mcproj.Projector(wl.robot, wl.constraints).project_segments(starts, delta, length, wl.params)
    torch.cuda.synchronize()
    assert torch.equal(o2[1], ref[1])
    conv = (ref[1] & 1).bool()
    assert (o2[0][:, conv] - ref[0][:, conv]).abs().max().item() <= 1e-4
    # new buffers / parameters: a new capture
    p2 = W.Params(tol=1e-5, max_iters=12, lam=1e-6)
    o3 = P.project_segments(starts, delta, length, p2, total=total)
    torch.cuda.synchronize()
    assert int(o3[2].max().item()) <= 12


def test_segments_inside_caller_graph(mcproj):
    """Called while the caller captures its own graph, the library enqueues its
    kernels into that graph instead of launching its private one."""
    wl = W.dual_arm_workload(total=5000)
    ex = wl.extra
    P = mcproj.Projector(wl.robot, wl.constraints)
    starts = P.project(dev(ex["raw_start"]), wl.params)[0]
    delta = dev(ex["raw_dir"] * ex["step"])
    length = dev(ex["lengths"], torch.int32)
    total = int(ex["lengths"].sum())
    out = torch.empty((14, total), device="cuda")
    fl = torch.empty(total, dtype=torch.uint8, device="cuda")
    it = torch.empty(total, dtype=torch.uint8, device="cuda")
    rs = torch.empty(total, dtype=torch.float64, device="cuda")
    ref = P.project_segments(starts, delta, length, wl.params)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            P.project_segments(starts, delta, length, wl.params, total=total, out=out, flags=fl, iters=it,
                               resid=rs, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(fl, ref[1])
    conv = (fl & 1).bool()
    assert (out[:, conv] - ref[0][:, conv]).abs().max().item() <= 1e-4


def test_vjp_matches_finite_differences_of_oracle_projection(mcproj):
    """g^T dPi/dq at the GPU's projected points, by central differences of the
    FP64 oracle's projection (h = 1e-4, lambda = 0, tight tolerance), on all
    16 configurations of the batch."""
    wl = W.adjoint_workload(n=16)
    P = mcproj.Projector(wl.robot, wl.constraints)
    O = orc.Oracle(wl.robot, wl.constraints)
    qs, fl, _, _ = P.project(dev(f32_exact(wl.q)), wl.params)
    g = f32_exact(wl.extra["g"][:, :16])
    v, _ = P.vjp(qs, dev(g))
    torch.cuda.synchronize()
    assert ((fl.cpu().numpy() & 1) != 0).all()
    qs, v = qs.cpu().numpy().astype(np.float64), v.cpu().numpy()
    h, d, n = 1e-4, qs.shape[0], qs.shape[1]
    E = np.eye(d) * h
    cols = np.concatenate([np.concatenate([qs[:, [i]] + E, qs[:, [i]] - E], 1) for i in range(n)], 1)
    pp = O.project(cols, 1e-13, 80, 0.0)[0].reshape(d, n, 2, d)   # [row, config, +/-, perturbed joint]
    for i in range(n):
        D = (pp[:, i, 0, :] - pp[:, i, 1, :]) / (2 * h)             # D[:, j] = dPi / dq_j
        ref = g[:, i] @ D
        assert np.linalg.norm(v[:, i] - ref) / np.linalg.norm(ref) < 1e-4, i


def test_autograd_project_backward_is_vjp(mcproj):
    from paper_2604_13323_gb300.shorten import ProjectFn
    wl = W.adjoint_workload(n=256)
    P = mcproj.Projector(wl.robot, wl.constraints)
    q = dev(f32_exact(wl.q)).requires_grad_(True)
    qs = ProjectFn.apply(q, P, wl.params)
    g = dev(f32_exact(wl.extra["g"][:, :256]))
    (qs * g).sum().backward()
    v, _ = P.vjp(qs.detach(), g)
    torch.cuda.synchronize()
    assert torch.equal(q.grad, v)


def test_path_shortening_reduces_length_on_manifold(mcproj):
    from paper_2604_13323_gb300.shorten import initial_paths, shorten_paths
    pw = W.path_workload(n_paths=64, n_way=16)
    wl = pw["workload"]
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    Q = initial_paths(P, pw["qa"], pw["qb"], pw["noise"], wl.params)
    Qf, st = shorten_paths(P, Q, 64, 16, wl.params, steps=20)
    assert st["mean_length_reduction"] > 0.05, st
    assert st["min_length_reduction"] > -1e-3, st
    assert st["converged_fraction"] > 0.99 and st["max_resid"] < 1e-5, st
    # the shortened waypoints are valid points of the manifold (FP64 oracle residual)
    O = orc.Oracle(wl.robot, wl.constraints)
    Qn = Qf.cpu().numpy().astype(np.float64)
    for i in range(0, Qn.shape[1], 97):
        assert np.linalg.norm(O.residual(Qn[:, i])) < 1e-5


def test_graph_shortening_equals_autograd_shortening(mcproj):
    """The graph-captured descent runs the same kernels in the same order as
    the autograd one: identical waypoints and statistics."""
    from paper_2604_13323_gb300.shorten import initial_paths, shorten_paths, shorten_paths_graph
    pw = W.path_workload(n_paths=64, n_way=16)
    wl = pw["workload"]
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    Q = initial_paths(P, pw["qa"], pw["qb"], pw["noise"], wl.params)
    Qa, sa = shorten_paths(P, Q.clone(), 64, 16, wl.params, steps=12)
    Qg, sg = shorten_paths_graph(P, Q.clone(), 64, 16, wl.params, steps=12)
    assert torch.equal(Qa, Qg)
    assert sa == sg


@pytest.mark.parametrize("steps", [1, 10])
def test_path_shortening_trajectory_matches_oracle(mcproj, steps):
    """16 paths x 16 waypoints on the dual-arm manifold, shortened for 1 and
    10 steps by the graph-captured GPU descent (FP32 projection with FP64
    acceptance, length gradient, VJP, clipped step) and by the FP64 oracle
    from the same projected initial waypoints: every final waypoint agrees to
    the 1e-4 rad point bar where the oracle's own trajectory is determined to
    that bar at FP32 precision (it moves less under 8 perturbations of 8 unit
    roundoffs of the initial waypoints), the lengths before and after agree,
    and every GPU waypoint is a valid point of the manifold."""
    from oracle import parity
    from paper_2604_13323_gb300.shorten import initial_paths, shorten_paths_graph
    n_paths, n_way, eta, max_step = 16, 16, 0.1, 0.05
    pw = W.path_workload(n_paths=n_paths, n_way=n_way)
    wl = pw["workload"]
    p = wl.params
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints)
    Q0 = initial_paths(P, pw["qa"], pw["qb"], pw["noise"], p)
    torch.cuda.synchronize()
    q0 = Q0.cpu().numpy().astype(np.float64)
    Qg, st = shorten_paths_graph(P, Q0.clone(), n_paths, n_way, p, steps=steps, eta=eta, max_step=max_step)
    qg = Qg.cpu().numpy().astype(np.float64)
    qo, fo, ro, Lo = O.shorten(q0, n_paths, n_way, p, steps, eta, max_step)
    rng = np.random.default_rng(0)
    dev_max = np.zeros(q0.shape[1])
    for _ in range(8):
        q1 = q0 * (1.0 + parity.REL_FP32 * rng.choice([-1.0, 1.0], size=q0.shape))
        dev_max = np.maximum(dev_max, np.abs(O.shorten(q1, n_paths, n_way, p, steps, eta, max_step)[0] - qo).max(0))
    el = dev_max <= 1e-4
    assert el.mean() > 0.9, el.mean()
    err = np.abs(qg - qo).max(axis=0)
    assert (err[el] <= 1e-4).all(), (err[el].max(), np.flatnonzero((err > 1e-4) & el)[:8])
    L0 = orc.path_length_grad(q0, n_paths, n_way)[0]
    L1 = orc.path_length_grad(qg, n_paths, n_way)[0]
    np.testing.assert_allclose(L0, Lo[:, 0], rtol=1e-12)
    np.testing.assert_allclose(L1, Lo[:, 1], rtol=1e-4)
    assert np.mean(1 - Lo[:, 1] / Lo[:, 0]) == pytest.approx(st["mean_length_reduction"], abs=1e-4)
    assert (fo & orc.CONVERGED).all() and st["converged_fraction"] == 1.0
    for i in range(qg.shape[1]):
        assert np.linalg.norm(O.residual(qg[:, i])) < p.tol


@pytest.mark.parametrize("name", ["arm", "dual", "tray", "tray_cyclic", "humanoid", "arm_fp64"])
def test_project_check_equals_separate_calls(mcproj, name):
    """mcp_project_check_batch (one persistent launch for the FP32 thread
    kernels, two launches otherwise) returns what mcp_project_batch followed by
    mcp_check_batch on its output returns, bit for bit."""
    if name in ("arm", "arm_fp64"):
        wl = W.arm_workload(n=8195)
    elif name == "dual":
        wl = W.dual_arm_workload(total=10, n_random=8195)
    elif name.startswith("tray"):
        wl = W.arm_task_workload("tray", n=8195)
        wl.params.cyclic = name.endswith("cyclic")
    else:
        wl = W.humanoid_workload(n=2051)
    dt = torch.float64 if name == "arm_fp64" else torch.float32
    if name == "arm_fp64":
        wl.params.precision = W.PREC_FP64
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    q = dev(f32_exact(wl.q), dt)
    n = q.shape[1]
    a = P.project(q, wl.params)
    pa = torch.zeros(n, dtype=torch.int32, device="cuda")
    ha = P.check(a[0], pairs=pa)
    for fuse in (1, 0):
        P.set_tuning(128, 4, 32, fuse)
        pb = torch.zeros(n, dtype=torch.int32, device="cuda")
        b = P.project_check(q, wl.params, pairs=pb)
        torch.cuda.synchronize()
        for x, y in zip(a, b[:4]):
            assert torch.equal(x, y)
        assert torch.equal(ha, b[4])
        assert torch.equal(pa, pb)


def test_arm_full_batch_in_the_benchmark_configuration(mcproj):
    """The 65,536-configuration arm batch through the call and launch shape the
    benchmark times (autotuned, projection and check possibly fused), against
    the oracle: flags, points on the eligible starts, FP64 validity and the
    collision verdicts outside the contact band."""
    from tests.gpu_util import compare_collision, compare_projection, eligible_mask
    wl = W.arm_workload(n=65536)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    q = dev(q0)
    P.autotune(q, wl.params)
    out, fl, it, r, hit = P.project_check(q, wl.params)
    torch.cuda.synchronize()
    gpu = (out.cpu().numpy().astype(np.float64), fl.cpu().numpy(), it.cpu().numpy().astype(np.int32), r.cpu().numpy())
    el, ora = eligible_mask(O, q0, wl.params)
    st = compare_projection(gpu, ora, wl.params.tol, oracle=O, eligible=el, min_eligible=0.5, sample_resid=4096)
    assert st["conv_gpu"] > 0.99
    h_o, m_o = O.check(gpu[0])
    compare_collision(hit.cpu().numpy(), h_o, m_o)


def test_dual_segments_in_the_benchmark_configuration(mcproj):
    """The full uneven-segment dual-arm workload (262,240 points) as the
    benchmark runs it: segment starts projected on the device, the launch
    shape and threads per configuration autotuned on the first 65,536
    materialised points, one persistent segment launch, then the collision
    check; against the oracle on the same FP32 points."""
    from tests.gpu_util import compare_collision, compare_projection, eligible_mask
    wl = W.dual_arm_workload()
    ex = wl.extra
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    starts = P.project(dev(ex["raw_start"]), wl.params)[0]
    delta = dev(ex["raw_dir"] * ex["step"])
    length = dev(ex["lengths"], torch.int32)
    s, d = starts.cpu(), delta.cpu()
    t = torch.cat([torch.arange(int(ln), dtype=torch.float32) for ln in ex["lengths"]])
    sid = torch.repeat_interleave(torch.arange(len(ex["lengths"])), torch.tensor(ex["lengths"], dtype=torch.long))
    pts = torch.addcmul(s[:, sid], t[None, :], d[:, sid])
    tpb, bps, chunk, fuse, tpc = P.autotune(pts[:, :65536].contiguous().cuda(), wl.params)
    out, fl, it, r = P.project_segments(starts, delta, length, wl.params)
    hit = P.check(out)
    torch.cuda.synchronize()
    gpu = (out.double().cpu().numpy(), fl.cpu().numpy(), it.cpu().numpy().astype(np.int32), r.cpu().numpy())
    q0 = pts.double().numpy()
    el, ora = eligible_mask(O, q0, wl.params)
    st = compare_projection(gpu, ora, wl.params.tol, oracle=O, eligible=el, min_eligible=0.5, sample_resid=4096)
    assert st["n"] == 262240 and st["conv_gpu"] > 0.99, (st, tpc)
    h_o, m_o = O.check(gpu[0])
    compare_collision(hit.cpu().numpy(), h_o, m_o)


def test_non_finite_obstacles_are_rejected_and_keep_the_scene(mcproj):
    wl = W.arm_workload(n=2048)
    q = dev(f32_exact(wl.q))
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    before = P.check(q).clone()
    bad = wl.obstacles.spheres.copy()
    bad[40, 3] = np.nan
    with pytest.raises(mcproj.MCPError):
        P.load_obstacles(W.Obstacles(spheres=bad, aabbs=wl.obstacles.aabbs))
    after = P.check(q)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
