"""The group-cooperative FP32 kernel (four lanes per configuration, eight per
warp) that runs the stacked form of the 36-DoF humanoid classes: edge cases
of its work distribution and of Alg. 2's exits, against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import compare_projection, eligible_mask, f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


def run(P, q0, params, ld=None):
    d, n = q0.shape
    ld = ld or n
    q = torch.zeros((d, ld), dtype=torch.float32, device="cuda")
    q[:, :n] = torch.tensor(q0, dtype=torch.float32, device="cuda")
    out, fl, it, r = P.project(q, params, n=n)
    torch.cuda.synchronize()
    return (out[:, :n].double().cpu().numpy(), fl[:n].cpu().numpy(), it[:n].cpu().numpy(),
            r[:n].cpu().numpy())


@pytest.mark.parametrize("n", [1, 5, 8, 13, 67])
def test_small_and_ragged_batches(mcproj, n):
    """Fewer configurations than one warp's groups, and sizes that leave a
    warp's last groups idle: every configuration is projected exactly as in
    a large batch (the work queue hands out single configurations)."""
    wl = W.humanoid_workload(n=128)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints)
    big = run(P, q0, wl.params)
    small = run(P, q0[:, :n], wl.params, ld=((n + 31) // 32) * 32)
    for a, b in zip(small, big):
        np.testing.assert_array_equal(a, b[..., :n] if a.ndim == 1 else b[:, :n])


def test_nonfinite_cap0_and_in_place(mcproj):
    wl = W.humanoid_workload(n=64)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints)
    qn = q0.copy()
    qn[7, 3] = np.nan
    qn[0, 9] = np.inf
    _, fl, _, _ = run(P, qn, wl.params)
    assert fl[3] & mcproj.F_NONFINITE and fl[9] & mcproj.F_NONFINITE
    ok = np.ones(64, bool)
    ok[[3, 9]] = False
    assert ((fl[ok] & mcproj.F_CONVERGED) != 0).mean() > 0.95
    # cap = 0: no step; the FP64 residual of the start is reported
    O = orc.Oracle(wl.robot, wl.constraints)
    p0 = W.Params(tol=1e-5, max_iters=0, lam=1e-6)
    q_out, fl0, it0, r0 = run(P, q0, p0)
    assert (it0 == 0).all()
    np.testing.assert_array_equal(q_out, q0)
    for i in range(0, 64, 7):
        r = np.linalg.norm(O.residual(q0[:, i]))
        assert abs(r - r0[i]) <= 1e-12 * max(1.0, r)
    # in place: q_out aliases q_in
    q = torch.tensor(q0, dtype=torch.float32, device="cuda")
    ref = P.project(q.clone(), wl.params)[0]
    P.project(q, wl.params, out=q)
    torch.cuda.synchronize()
    assert torch.equal(q, ref)


def test_max_distance_exit(mcproj):
    """Alg. 2's MaxDistance exit (|dq| above the bound: DIVERGED, the last
    iterate kept) on the group kernel: the flags agree with the oracle and
    so do the kept points of configurations that left after the same step."""
    wl = W.humanoid_workload(n=1024)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints)
    O = orc.Oracle(wl.robot, wl.constraints)
    p = W.Params(tol=1e-5, max_iters=40, lam=1e-6, max_step=1.6)
    g = run(P, q0, p)
    o = O.project(q0, p.tol, p.max_iters, p.lam, max_step=p.max_step)
    dg, do = (g[1] & 4) != 0, (o[1] & 4) != 0
    assert 0.05 < dg.mean() < 0.95
    assert (dg == do).mean() >= 0.99
    same = dg & do & (g[2] == o[2])
    assert same.mean() > 0.5 * dg.mean()
    assert np.abs(g[0][:, same] - o[0][:, same]).max() < 1e-4


@pytest.mark.parametrize("alpha", [0.5])
def test_step_scale(mcproj, alpha):
    wl = W.humanoid_workload(n=1024)
    q0 = f32_exact(wl.q)
    p = W.Params(tol=1e-5, max_iters=80, lam=1e-6, pivot_fp64=1e-7, alpha=alpha)
    P = mcproj.Projector(wl.robot, wl.constraints)
    O = orc.Oracle(wl.robot, wl.constraints)
    gpu = run(P, q0, p)
    el, ora = eligible_mask(O, q0, p)
    st = compare_projection(gpu, ora, p.tol, oracle=O, eligible=el, min_eligible=0.5, sample_resid=256)
    assert st["conv_gpu"] > 0.95, st
    full = run(P, q0, W.Params(tol=1e-5, max_iters=80, lam=1e-6, pivot_fp64=1e-7))
    assert gpu[2].mean() > full[2].mean()
