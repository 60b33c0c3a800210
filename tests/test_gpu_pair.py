"""The two-lanes-per-configuration FP32 kernel of the dual arm (one lane per
arm; threads per configuration = 2 in the tuning): parity with the FP64 oracle
on batches and uneven segments, the edge cases of its work distribution and
of Alg. 2's exits, and its agreement with the thread-per-configuration kernel.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import compare_collision, compare_projection, eligible_mask, f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu

PAIR = (128, 4, 32, 0, 2)
THREAD = (128, 4, 32, 0, 1)


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


@pytest.fixture(scope="module")
def dual():
    return W.dual_arm_workload(total=10, n_random=6000)


def run(P, q0, params, ld=None, tuning=PAIR):
    P.set_tuning(*tuning)
    d, n = q0.shape
    ld = ld or n
    q = torch.zeros((d, ld), dtype=torch.float32, device="cuda")
    q[:, :n] = torch.tensor(q0, dtype=torch.float32, device="cuda")
    out, fl, it, r = P.project(q, params, n=n)
    torch.cuda.synchronize()
    return (out[:, :n].double().cpu().numpy(), fl[:n].cpu().numpy(), it[:n].cpu().numpy().astype(np.int32),
            r[:n].cpu().numpy())


def test_pair_batch_parity(mcproj, dual):
    q0 = f32_exact(dual.q)
    P = mcproj.Projector(dual.robot, dual.constraints)
    O = orc.Oracle(dual.robot, dual.constraints)
    gpu = run(P, q0, dual.params)
    el, ora = eligible_mask(O, q0, dual.params)
    st = compare_projection(gpu, ora, dual.params.tol, oracle=O, eligible=el, min_eligible=0.95)
    assert st["conv_gpu"] > 0.99, st


def test_pair_segments_parity(mcproj):
    """Uneven segments (the points formed on the device) with one lane per arm."""
    wl = W.dual_arm_workload(total=30000)
    ex = wl.extra
    P = mcproj.Projector(wl.robot, wl.constraints)
    O = orc.Oracle(wl.robot, wl.constraints)
    starts, _, _, _ = O.project_params(ex["raw_start"], wl.params)
    seg = W.make_segments(f32_exact(starts), f32_exact(ex["raw_dir"]), ex["lengths"], ex["step"])
    P.set_tuning(*PAIR)
    dv = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    out, fl, it, r = P.project_segments(dv(seg.start), dv(seg.delta), dv(seg.length, torch.int32), wl.params)
    torch.cuda.synchronize()
    gpu = (out.double().cpu().numpy(), fl.cpu().numpy(), it.cpu().numpy().astype(np.int32), r.cpu().numpy())
    d = torch.tensor(seg.delta, dtype=torch.float32)
    s = torch.tensor(seg.start, dtype=torch.float32)
    t = torch.cat([torch.arange(int(ln), dtype=torch.float32) for ln in seg.length])
    sid = torch.repeat_interleave(torch.arange(seg.length.shape[0]), torch.tensor(seg.length, dtype=torch.long))
    pts = torch.addcmul(s[:, sid], t[None, :], d[:, sid]).double().numpy()
    el, ora = eligible_mask(O, pts, wl.params)
    st = compare_projection(gpu, ora, wl.params.tol, oracle=O, eligible=el, min_eligible=0.5, sample_resid=2048)
    assert st["n"] == seg.total and st["conv_gpu"] > 0.99, st


@pytest.mark.parametrize("n", [1, 3, 16, 17, 45])
def test_pair_small_and_ragged_batches(mcproj, dual, n):
    """Fewer configurations than one warp's 16 pairs and ragged tails: each
    configuration's result does not depend on the batch around it."""
    q0 = f32_exact(dual.q[:, :256])
    P = mcproj.Projector(dual.robot, dual.constraints)
    big = run(P, q0, dual.params)
    small = run(P, q0[:, :n], dual.params, ld=((n + 31) // 32) * 32)
    for a, b in zip(small, big):
        np.testing.assert_array_equal(a, b[..., :n] if a.ndim == 1 else b[:, :n])


def test_pair_equals_thread_kernel_where_no_fp32_step_is_taken(mcproj, dual):
    """FK and the residual of one lane per arm are the thread kernel's
    operations in the same order: with no FP32 step taken (cap 0, or every
    pivot below the FP64 re-solve threshold, so each configuration continues
    in FP64 from its start) the two kernels give bit-identical results."""
    q0 = f32_exact(dual.q[:, :2048])
    P = mcproj.Projector(dual.robot, dual.constraints)
    for p in (W.Params(tol=1e-5, max_iters=0, lam=1e-6),
              W.Params(tol=1e-5, max_iters=30, lam=1e-6, pivot_fp64=1e30)):
        a = run(P, q0, p, tuning=PAIR)
        b = run(P, q0, p, tuning=THREAD)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    assert ((a[1] & mcproj.F_FP64_RESOLVE) != 0).mean() > 0.9


def test_pair_agrees_with_thread_kernel(mcproj, dual):
    """The Gram sums run in another order (two partial sums), so iterates
    differ by rounding: flags agree on >= 99.9 % and converged points to 1e-4."""
    q0 = f32_exact(dual.q)
    P = mcproj.Projector(dual.robot, dual.constraints)
    a = run(P, q0, dual.params, tuning=PAIR)
    b = run(P, q0, dual.params, tuning=THREAD)
    assert (a[1] == b[1]).mean() >= 0.999
    both = ((a[1] & mcproj.F_CONVERGED) != 0) & ((b[1] & mcproj.F_CONVERGED) != 0)
    assert both.mean() > 0.98
    # a chaotic start can branch; the bulk lands on the same point
    dq = np.abs(a[0][:, both] - b[0][:, both]).max(axis=0)
    assert (dq <= 1e-4).mean() >= 0.99
    assert (a[3][both] < dual.params.tol).all()


def test_pair_edge_cases(mcproj, dual):
    q0 = f32_exact(dual.q[:, :512])
    P = mcproj.Projector(dual.robot, dual.constraints)
    O = orc.Oracle(dual.robot, dual.constraints)
    # non-finite inputs are flagged and do not disturb the other lane of the pair
    qn = q0.copy()
    qn[3, 5] = np.nan    # arm 0 of configuration 5
    qn[10, 6] = np.inf   # arm 1 of configuration 6
    _, fl, _, _ = run(P, qn, dual.params)
    assert fl[5] & mcproj.F_NONFINITE and fl[6] & mcproj.F_NONFINITE
    ok = np.ones(512, bool)
    ok[[5, 6]] = False
    ref = run(P, q0, dual.params)
    np.testing.assert_array_equal(fl[ok], ref[1][ok])
    # MaxDistance exit (Alg. 2): DIVERGED with the last iterate kept, as the oracle
    p = W.Params(tol=1e-5, max_iters=30, lam=1e-6, max_step=0.8)  # the oracle: 54 % diverge
    g = run(P, q0, p)
    o = O.project(q0, p.tol, p.max_iters, p.lam, max_step=p.max_step)
    dg, do = (g[1] & 4) != 0, (o[1] & 4) != 0
    assert 0.02 < dg.mean() < 0.98
    assert (dg == do).mean() >= 0.98
    same = dg & do & (g[2] == o[2])
    assert same.sum() > 0.5 * dg.sum()
    assert (np.abs(g[0][:, same] - o[0][:, same]).max(axis=0) < 1e-4).mean() >= 0.95
    # step scale: more steps, still converged
    half = run(P, q0, W.Params(tol=1e-5, max_iters=60, lam=1e-6, alpha=0.5))
    assert half[2].mean() > ref[2].mean() and ((half[1] & mcproj.F_CONVERGED) != 0).mean() > 0.97
    # in place
    q = torch.tensor(q0, dtype=torch.float32, device="cuda")
    P.set_tuning(*PAIR)
    want = P.project(q.clone(), dual.params)[0]
    P.project(q, dual.params, out=q)
    torch.cuda.synchronize()
    assert torch.equal(q, want)


def test_pair_setting_is_ignored_by_single_chain_classes(mcproj):
    wl = W.arm_workload(n=4096)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints)
    a = run(P, q0, wl.params, tuning=PAIR)
    b = run(P, q0, wl.params, tuning=THREAD)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    with pytest.raises(mcproj.MCPError):
        P.set_tuning(128, 4, 32, 0, 3)


def test_autotune_times_both_kernels(mcproj, dual):
    q = torch.tensor(f32_exact(dual.q), dtype=torch.float32, device="cuda")
    P = mcproj.Projector(dual.robot, dual.constraints)
    tpb, bps, chunk, fuse, tpc = P.autotune(q, dual.params)
    assert tpc in (1, 2) and fuse in (0, 1)


def test_pair_fused_check(mcproj):
    """The collision check inside the pair kernel (one configuration per lane
    after the acceptance) gives the verdicts and test counts of the check
    kernel run on the same outputs, which match the oracle's verdicts."""
    wl = W.dual_arm_workload(total=10, n_random=8192)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    q = torch.tensor(q0, dtype=torch.float32, device="cuda")
    n = q.shape[1]
    res = []
    for fuse in (1, 0):
        P.set_tuning(128, 4, 32, fuse, 2)
        pairs = torch.zeros(n, dtype=torch.int32, device="cuda")
        res.append((*P.project_check(q, wl.params, pairs=pairs), pairs))
    torch.cuda.synchronize()
    (out, fl, it, r, hit, pairs), (out2, fl2, it2, r2, hit2, pairs2) = res
    for x, y in ((out, out2), (fl, fl2), (it, it2), (r, r2), (hit, hit2), (pairs, pairs2)):
        assert torch.equal(x, y)
    h_o, m_o = O.check(out.double().cpu().numpy())
    st = compare_collision(hit.cpu().numpy(), h_o, m_o)
    assert 0.0 < st["collide_frac"] < 1.0
