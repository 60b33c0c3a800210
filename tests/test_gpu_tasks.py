"""Parity of the task constraints beyond B^w = 0 (bounded TSR, point on a
plane, point on a line, closed-linkage distance) and of the cyclic form of
getDescentStep (Sec. IV-C), CUDA path (C ABI) against the FP64 oracle.

Same bars as the other parity tests: converged configurations agree to
1e-4 rad on the eligible starts, the FP64 residual of every converged output is
below tol, convergence flags agree on >= 99.9 %.  These workloads have more
starts whose outcome is not a function of the start (a bound's active set, a
slow sweep or a near-singular step decides whether ||F|| < tol is met before
the cap, and the FP64 oracle itself flips under a perturbation of a few FP32
ulps), so the flag bar and the iteration counts apply to the starts where the
oracle's flag, count and point are stable, and all starts must agree on 99 %
of the flags."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import Q_TOL_FP64, compare_collision, compare_projection, eligible_mask, f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


def run(P, q0, params, dtype=torch.float32, ld=None):
    d, n = q0.shape
    ld = n if ld is None else ld
    q = torch.zeros((d, ld), dtype=dtype, device="cuda")
    q[:, :n] = torch.tensor(q0, dtype=dtype, device="cuda")
    out, fl, it, r = P.project(q, params, n=n)
    torch.cuda.synchronize()
    return (out[:, :n].cpu().numpy().astype(np.float64), fl[:n].cpu().numpy(), it[:n].cpu().numpy().astype(np.int32),
            r[:n].cpu().numpy())


def self_consistent_bars(selfst):
    """Overall flag agreement and step-count mismatch allowed on all starts:
    twice what the FP64 oracle shows against itself under the perturbation,
    and never looser than 99 % / 0.1 % where the oracle is self-consistent."""
    return {"overall_flag_agree": 1.0 - max(0.01, 2.0 * selfst["self_flip_rate"]),
            "max_recount": max(0.001, 2.0 * selfst["self_recount_rate"])}


def workload(name):
    if name == "rod":
        return W.dual_rod_workload(n=4099)
    return W.arm_task_workload(name, n=4099)


CASES = [("tray", False), ("peg", False), ("tsr", False), ("rod", False), ("tray", True), ("tsr", True),
         ("rod", True)]


@pytest.mark.parametrize("name,cyclic", CASES, ids=[f"{n}-{'cyclic' if c else 'stacked'}" for n, c in CASES])
def test_task_fp32_parity(mcproj, name, cyclic):
    wl = workload(name)
    if cyclic:
        wl.params.cyclic = True
        wl.params.max_iters = 120
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    for i in range(len(wl.constraints)):   # references resolved alike on both sides
        np.testing.assert_allclose(P.constraint(i)[0], O.constraint_values(i)[0], atol=1e-14)
        np.testing.assert_allclose(P.constraint(i)[2], O.constraint_values(i)[2], atol=1e-14)
    gpu = run(P, q0, wl.params, ld=4128)
    selfst = {}
    el, ora = eligible_mask(O, q0, wl.params, stable_iters=True, stats=selfst)
    bars = self_consistent_bars(selfst)
    if name == "tsr":
        # the bounded TSR's active set is decided on e_i against the bounds in the
        # working precision: a component within ~1e-7 of its bound is inside in
        # one precision and outside in the other; the extra (or missing) row
        # holds that component fixed in the min-norm step and redirects the
        # step, so the count and, for a few starts, the point change while the
        # result stays valid (FP64 residual < tol everywhere).  Points are
        # compared where the counts agree, at the 99th percentile.
        bars["max_recount"] = max(bars["max_recount"], 0.15)
        bars["q_quantile"] = 0.99
        bars["flag_agree"] = bars["overall_flag_agree"]   # the same active-set decisions move the flags
    st = compare_projection(gpu, ora, wl.params.tol, oracle=O, eligible=el, min_eligible=0.5, sample_resid=512,
                            stable_only=True, **bars)
    assert st["conv_oracle"] > 0.5, st
    if not cyclic:
        hit = P.check(torch.tensor(gpu[0], dtype=torch.float32, device="cuda")).cpu().numpy()
        compare_collision(hit, *O.check(gpu[0]))


@pytest.mark.parametrize("cyclic", [False, True], ids=["stacked", "cyclic"])
@pytest.mark.parametrize("name", ["tray", "tsr", "rod"])
def test_task_fp64_plain_parity(mcproj, name, cyclic):
    wl = workload(name)
    wl.params.precision = W.PREC_FP64
    if cyclic:
        wl.params.cyclic = True
        wl.params.max_iters = 120
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    gpu = run(P, wl.q, wl.params, dtype=torch.float64)
    selfst = {}
    el, ora = eligible_mask(O, wl.q, wl.params, stable_iters=True, stats=selfst)
    st = compare_projection(gpu, ora, wl.params.tol, q_tol=Q_TOL_FP64, oracle=O, eligible=el, min_eligible=0.7,
                            stable_only=True, **self_consistent_bars(selfst))
    assert st["iters_equal"] > 0.999, st


def test_cyclic_and_stacked_reach_the_manifold_differently(mcproj):
    """On a stack of coupled constraints the two forms are different iterations
    (the oracle pins this on closed forms); on the GPU both must land on the
    manifold, and the cyclic sweeps are more numerous."""
    wl = W.dual_rod_workload(n=8192)
    P = mcproj.Projector(wl.robot, wl.constraints)
    q = torch.tensor(f32_exact(wl.q), dtype=torch.float32, device="cuda")
    a = P.project(q, wl.params)
    p2 = W.Params(tol=wl.params.tol, max_iters=120, lam=wl.params.lam, cyclic=True)
    b = P.project(q, p2)
    torch.cuda.synchronize()
    ca, cb = (a[1] & 1).bool(), (b[1] & 1).bool()
    assert ca.float().mean() > 0.99 and cb.float().mean() > 0.99
    assert b[2][cb].float().mean() > a[2][ca].float().mean()
    assert (a[3][ca] < wl.params.tol).all() and (b[3][cb] < wl.params.tol).all()
    both = ca & cb
    assert (a[0][:, both] - b[0][:, both]).abs().max() > 1e-3


def test_humanoid_cyclic_fp32_parity(mcproj):
    """Cyclic projection on the 36-DoF humanoid (warp kernel with masked
    per-constraint steps): the slow, linearly convergent alternating projection
    the stacked form replaces.  Compared with the oracle over 250 sweeps."""
    wl = W.humanoid_workload(n=512)
    wl.params.cyclic = True
    wl.params.max_iters = 250
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    gpu = run(P, q0, wl.params, ld=512)
    el, ora = eligible_mask(O, q0, wl.params)
    st = compare_projection(gpu, ora, wl.params.tol, oracle=O, eligible=el, min_eligible=0.3)
    assert st["conv_oracle"] > 0.25, st


def test_humanoid_cyclic_fp64_plain_parity(mcproj):
    wl = W.humanoid_workload(n=256)
    wl.params.cyclic = True
    wl.params.max_iters = 250
    wl.params.precision = W.PREC_FP64
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    gpu = run(P, wl.q, wl.params, dtype=torch.float64)
    el, ora = eligible_mask(O, wl.q, wl.params)
    st = compare_projection(gpu, ora, wl.params.tol, q_tol=Q_TOL_FP64, oracle=O, eligible=el, min_eligible=0.5)
    assert st["iters_equal"] > 0.99, st


def test_bounded_tsr_rejects_inverted_bounds(mcproj):
    wl = W.arm_task_workload("tsr", n=4)
    c = wl.constraints[0]
    c.B = c.B.copy()
    c.B[0], c.B[6] = 0.1, -0.1
    with pytest.raises(mcproj.MCPError):
        mcproj.Projector(wl.robot, [c])


def test_humanoid_hull_fp32_parity(mcproj):
    """The humanoid with the CoM on its support polygon (distance to the
    polygon, zero inside) instead of at its centre: the warp kernel against
    the oracle; the polygon is resolved alike on both sides."""
    wl = W.humanoid_workload(n=4099, hull=True)
    q0 = f32_exact(wl.q)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    np.testing.assert_allclose(P.constraint_bounds(3)[:8], O.bounds(3)[:8], atol=1e-13)
    gpu = run(P, q0, wl.params, ld=4128)
    selfst = {}
    el, ora = eligible_mask(O, q0, wl.params, stable_iters=True, stats=selfst)
    # inside / edge / vertex is decided on the CoM in the working precision
    # (a nonsmooth residual like the bounded TSR's): points at the 99.9th percentile
    st = compare_projection(gpu, ora, wl.params.tol, oracle=O, eligible=el, min_eligible=0.5, sample_resid=512,
                            stable_only=True, q_quantile=0.999, **self_consistent_bars(selfst))
    assert st["conv_gpu"] > 0.95, st


def test_humanoid_hull_fp64_plain_parity(mcproj):
    wl = W.humanoid_workload(n=512, hull=True)
    wl.params.precision = W.PREC_FP64
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    gpu = run(P, wl.q, wl.params, dtype=torch.float64)
    selfst = {}
    el, ora = eligible_mask(O, wl.q, wl.params, stable_iters=True, stats=selfst)
    compare_projection(gpu, ora, wl.params.tol, q_tol=Q_TOL_FP64, oracle=O, eligible=el, min_eligible=0.7,
                       stable_only=True, **self_consistent_bars(selfst))
