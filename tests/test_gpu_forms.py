"""The outer form of the LM step and the step scale alpha of Alg. 2 on the CUDA
path (C ABI), against the FP64 oracle."""
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


def _rt(R, t):
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T.reshape(12)


def run(P, q0, params, dtype=torch.float32):
    q = torch.tensor(q0, dtype=dtype, device="cuda")
    out, fl, it, r = P.project(q, params)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), fl.cpu().numpy(), it.cpu().numpy().astype(np.int32), r.cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["fp32", "fp64"])
def test_outer_form_on_overdetermined_planes(mcproj, dtype):
    """Four planes through one point, a Cartesian point (k = 4 > d = 3): the
    outer step reaches the common point in one step (the inner form's J J^T
    is singular at lambda = 0)."""
    wl = W.sphere_workload(n_pairs=2)
    rng = np.random.default_rng(80)
    c = rng.uniform(-0.5, 0.5, 3)
    cons = [W.Constraint(W.C_PLANE, frame_a=0, P=_rt(W.random_rotation(rng), c)) for _ in range(4)]
    P = mcproj.Projector(wl.robot, cons)
    O = orc.Oracle(wl.robot, cons)
    q0 = f32_exact(rng.uniform(-1, 1, (3, 1000)))
    p = W.Params(tol=1e-6, max_iters=10, lam=0.0, outer=True,
                 precision=W.PREC_FP64 if dtype == torch.float64 else W.PREC_FP32)
    q, fl, it, r = run(P, q0, p, dtype)
    assert ((fl & orc.CONVERGED) != 0).all() and (it <= 2).all()
    np.testing.assert_allclose(q, np.repeat(c[:, None], 1000, 1), atol=1e-6)
    qo, fo, io, ro = O.project_params(q0, p)
    np.testing.assert_allclose(q, qo, atol=1e-6)


def test_outer_form_arm_parity(mcproj):
    """The outer form on the 7-DoF arm (k = 2 < d = 7) with lambda = 1e-3: the
    same iteration as the inner form in exact arithmetic, here against the
    oracle's outer form."""
    wl = W.arm_workload(n=4099)
    p = W.Params(tol=1e-5, max_iters=30, lam=1e-3, outer=True)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints)
    O = orc.Oracle(wl.robot, wl.constraints)
    gpu = run(P, q0, p)
    el, ora = eligible_mask(O, q0, p)
    st = compare_projection(gpu, ora, p.tol, oracle=O, eligible=el, min_eligible=0.5)
    assert st["conv_gpu"] > 0.99


@pytest.mark.parametrize("alpha", [0.5, 0.8])
def test_step_scale_parity(mcproj, alpha):
    wl = W.dual_arm_workload(total=10, n_random=4099)
    p = W.Params(tol=1e-5, max_iters=60, lam=1e-6, pivot_fp64=1e-7, alpha=alpha)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints)
    O = orc.Oracle(wl.robot, wl.constraints)
    gpu = run(P, q0, p)
    el, ora = eligible_mask(O, q0, p)
    st = compare_projection(gpu, ora, p.tol, oracle=O, eligible=el, min_eligible=0.5)
    assert st["conv_oracle"] > 0.95
    # a damped step takes more iterations than the full step
    full = run(P, q0, W.Params(tol=1e-5, max_iters=60, lam=1e-6, pivot_fp64=1e-7))
    assert gpu[2].mean() > full[2].mean()


def test_forms_rejected_where_unsupported(mcproj):
    hw = W.humanoid_workload(n=64)
    H = mcproj.Projector(hw.robot, hw.constraints)
    q = torch.tensor(hw.q, dtype=torch.float32, device="cuda")
    with pytest.raises(mcproj.MCPError):
        H.project(q, W.Params(tol=1e-5, max_iters=40, lam=1e-6, outer=True))
    wl = W.arm_task_workload("tray", n=64)
    P = mcproj.Projector(wl.robot, wl.constraints)
    q = torch.tensor(wl.q, dtype=torch.float32, device="cuda")
    with pytest.raises(mcproj.MCPError):
        P.project(q, W.Params(tol=1e-5, max_iters=30, lam=1e-6, outer=True, cyclic=True))
    with pytest.raises(mcproj.MCPError):
        P.project(q, W.Params(tol=1e-5, max_iters=30, lam=1e-6, alpha=3.0))
