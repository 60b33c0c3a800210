"""The operation-counting build of the oracle, and the kernel-structure flop
model (paper_2604_13323_gb300/flops.py) against it.

The counting build compiles the oracle's own source with a counting scalar
(oracle/count_ops.cpp); what it tallies per evaluation of F, per LM step and
per VJP is the method's arithmetic, with structural zeros and signed unit
factors free (traced straight-line code, Sec. IV-A).  Its tallies are pinned
on cases that can be counted by hand, and it must compute what the oracle
computes.  The benchmark's algorithmic flops use it, with the oracle's own
iteration counts.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_13323_gb300 import flops as FL
from paper_2604_13323_gb300 import workloads as W

ADD, MUL, DIV, SQRT, TRIG, ATAN2 = range(6)


def _flops(c):
    return c[:, ADD] + c[:, MUL] + c[:, DIV]


def test_sphere_evaluation_is_the_hand_count():
    """F = |q| - 1 for q in R^3: q0^2 + q1^2 + q2^2 (3 multiplies, 2 adds), one
    square root, one subtraction."""
    wl = W.sphere_workload(n_pairs=2)
    O = orc.Oracle(wl.robot, wl.constraints)
    q = np.random.default_rng(0).standard_normal((3, 16)) * 1.7
    c = O.count_ops(q, wl.params)["eval"]
    assert (c == np.array([3, 3, 0, 1, 0, 0])).all(), c[:2]


@pytest.mark.parametrize("name", ["arm", "dual", "humanoid"])
def test_evaluation_takes_one_sin_cos_pair_per_revolute_joint(name):
    """Forward kinematics evaluates sin and cos once per revolute joint and
    nothing else does in a residual evaluation without a log map (the arm's
    axis constraint); the pose constraints add one atan2 per log map."""
    wl = {"arm": W.arm_workload(n=64), "dual": W.dual_arm_workload(total=10, n_random=64),
          "humanoid": W.humanoid_workload(n=64)}[name]
    O = orc.Oracle(wl.robot, wl.constraints)
    c = O.count_ops(wl.q[:, :64], wl.params)["eval"]
    n_rev = int((np.asarray(wl.robot.type) == W.REVOLUTE).sum())
    assert (c[:, TRIG] == 2 * n_rev).all()
    n_log = sum(1 for k in wl.constraints if k.kind in (W.C_POSE, W.C_REL_POSE))
    assert (c[:, ATAN2] == n_log).all()


def test_counting_is_free_of_structural_zeros():
    """Multiplying by a structural zero or a signed unit costs nothing: one LM
    step on a linear constraint of a prismatic-only robot (F = A q - b, J = A)
    counts only the products with nonzero, non-unit entries."""
    wl = W.sphere_workload(n_pairs=2)
    O = orc.Oracle(wl.robot, [W.Constraint(W.C_PLANE, frame_a=0)])
    q = np.random.default_rng(1).standard_normal((3, 4))
    c = O.count_ops(q, W.Params(tol=1e-9, max_iters=5, lam=0.0))
    # F = z of the point: one row of J = (0, 0, 1): Gram 1x1 = 1 * 1 (free), sqrt
    # of the pivot, two divisions of the substitutions, J^T y = (0, 0, y) free,
    # the update subtracts one nonzero component
    step = c["step"]
    assert (step[:, SQRT] == 1).all() and (step[:, TRIG] == 0).all()
    assert (_flops(step) <= 4).all(), step


@pytest.mark.parametrize("name", ["arm", "dual", "humanoid"])
def test_flop_model_agrees_with_the_counted_oracle_per_step(name):
    """flops.py counts the structure of the kernels' code; without its sin/cos
    polynomials (special functions in the oracle's count) its LM step is
    within 10 % of the counted oracle's."""
    wl = {"arm": W.arm_workload(n=256), "dual": W.dual_arm_workload(total=10, n_random=256),
          "humanoid": W.humanoid_workload(n=256)}[name]
    O = orc.Oracle(wl.robot, wl.constraints)
    counted = _flops(O.count_ops(wl.q[:, :256], wl.params)["step"]).mean()
    fm = FL.FlopModel(wl.robot, wl.constraints)
    n_rev = int((np.asarray(wl.robot.type) == W.REVOLUTE).sum())
    model = fm.iteration - FL.SINCOS32 * n_rev
    assert abs(model - counted) <= 0.10 * counted, (model, counted)
