"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, a textbook/library routine, an independent formulation, exact
hand-worked values, or invariants.  A plausible mistake in the oracle (a
dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from oracle import oracle as orc
from paper_2604_13323_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _rt(R, t):
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T.reshape(12)


def _h(T12):
    H = np.eye(4)
    H[:3, :] = np.asarray(T12).reshape(3, 4)
    return H


def cartesian_robot(extra_sphere_r=0.0):
    wl = W.sphere_workload(n_pairs=2)
    rb = wl.robot
    rb.sphere = np.array([[0.0, 0.0, 0.0, extra_sphere_r]])
    return rb


def planar_2link(l1, l2):
    """Two revolute joints about world z; all mass at the tip of link 2, so the
    CoM is the tip position."""
    X = np.stack([_rt(np.eye(3), (0, 0, 0)), _rt(np.eye(3), (l1, 0, 0))])
    return W.Robot(parent=np.array([-1, 0], np.int32), type=np.zeros(2, np.int32), X=X,
                   lower=np.full(2, -10.0), upper=np.full(2, 10.0), mass=np.array([0.0, 1.0]),
                   com=np.array([[0.0, 0.0, 0.0], [l2, 0.0, 0.0]]), sphere_link=np.zeros(0, np.int32),
                   sphere=np.zeros((0, 4)), frame_link=np.array([1], np.int32),
                   frame_X=_rt(np.eye(3), (l2, 0, 0))[None])


# ---------------------------------------------------------------------------
# Sphere manifold: the closed form q* = q0 / ||q0|| (Newton on ||q|| - 1 is radial)
# ---------------------------------------------------------------------------
def test_sphere_projection_is_normalisation():
    rb = cartesian_robot()
    o = orc.Oracle(rb, [W.Constraint(W.C_SPHERE, target=np.array([1.0, 0, 0]))])
    rng = np.random.default_rng(0)
    q0 = rng.standard_normal((3, 200)) * rng.uniform(0.05, 3.0, 200)
    out, flags, iters, resid = o.project(q0, tol=1e-12, max_iters=50, lam=0.0)
    expect = q0 / np.linalg.norm(q0, axis=0)
    assert np.all(flags & orc.CONVERGED)
    np.testing.assert_allclose(out, expect, atol=1e-14, rtol=0)
    # lambda = 0: one Newton step is exact, the second residual check passes
    assert np.all(iters == 1)
    # damped steps stay radial, so the limit is the same point
    out2, flags2, iters2, _ = o.project(q0, tol=1e-12, max_iters=50, lam=1e-2)
    assert np.all(flags2 & orc.CONVERGED)
    np.testing.assert_allclose(out2, expect, atol=1e-12, rtol=0)
    assert iters2.max() > 1


def test_sphere_origin_is_flagged():
    rb = cartesian_robot()
    o = orc.Oracle(rb, [W.Constraint(W.C_SPHERE, target=np.array([1.0, 0, 0]))])
    _, flags, _, _ = o.project(np.zeros((3, 1)), tol=1e-8, max_iters=50, lam=0.0)
    assert flags[0] & orc.NONFINITE


# ---------------------------------------------------------------------------
# Linear constraint: prismatic robot + CoM constraint is affine in q, so one
# step with lambda = 0 is the exact orthogonal projection
#     q* = q0 - A^T (A A^T)^{-1} (A q0 - b).
# A and b are derived here from the robot description alone.
# ---------------------------------------------------------------------------
def prismatic_robot(seed, n=5):
    rng = np.random.default_rng(seed)
    X = np.stack([_rt(W.random_rotation(rng), rng.uniform(-0.5, 0.5, 3)) for _ in range(n)])
    parent = np.array([-1] + list(range(n - 1)), np.int32)
    return W.Robot(parent=parent, type=np.ones(n, np.int32), X=X, lower=np.full(n, -9.0), upper=np.full(n, 9.0),
                   mass=rng.uniform(0.5, 2.0, n), com=rng.uniform(-0.3, 0.3, (n, 3)),
                   sphere_link=np.zeros(0, np.int32), sphere=np.zeros((0, 4)),
                   frame_link=np.array([n - 1], np.int32), frame_X=W.IDENTITY12[None].copy())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linear_constraint_one_step_is_orthogonal_projection(seed):
    rb = prismatic_robot(seed)
    n = rb.n_joints
    # independent affine model of the CoM: prismatic joints never rotate, so the
    # rotation of every frame is the product of the fixed X rotations.
    Rw, pw = [], []
    for j in range(n):
        H = _h(rb.X[j]) if j == 0 else np.linalg.multi_dot([_H_joint_chain(rb, j - 1), _h(rb.X[j])])
        Rw.append(H[:3, :3])
        pw.append(H[:3, 3])
    M = rb.mass.sum()
    A = np.zeros((2, n))
    b0 = np.zeros(2)
    for i in range(n):   # link i carries mass m_i at com_i; its position is affine in q_0..q_i
        ci0 = pw[i] + Rw[i] @ rb.com[i]
        b0 += rb.mass[i] * ci0[:2] / M
        for j in range(i + 1):
            A[:, j] += rb.mass[i] * Rw[j][:2, 2] / M
    target = np.array([0.1, -0.2])
    o = orc.Oracle(rb, [W.Constraint(W.C_COM_XY, target=np.array([target[0], target[1], 0.0]))])
    rng = np.random.default_rng(seed + 10)
    q0 = rng.uniform(-1, 1, (n, 16))
    out, flags, iters, _ = o.project(q0, tol=1e-12, max_iters=1, lam=0.0)
    resid = A @ q0 + b0[:, None] - target[:, None]
    expect = q0 - A.T @ np.linalg.solve(A @ A.T, resid)
    np.testing.assert_allclose(out, expect, atol=1e-12, rtol=0)
    assert np.all(flags & orc.CONVERGED)


def _H_joint_chain(rb, j):
    """World pose of joint frame j at q = 0 (only used for prismatic chains)."""
    H = np.eye(4)
    chain = []
    while j >= 0:
        chain.append(j)
        j = rb.parent[j]
    for i in reversed(chain):
        H = H @ _h(rb.X[i])
    return H


# ---------------------------------------------------------------------------
# Planar 2-link analytic IK: Newton on the tip position lands on one of the two
# closed-form solutions (hand-worked values in tests/golden/planar_2link_ik.txt).
# ---------------------------------------------------------------------------
def _golden_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "planar_2link_ik.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_planar_2link_matches_closed_form_ik(row):
    l1, l2, x, y, q1u, q2u, q1d, q2d = row
    rb = planar_2link(l1, l2)
    o = orc.Oracle(rb, [W.Constraint(W.C_COM_XY, target=np.array([x, y, 0.0]))])
    # starts near each solution converge to that solution
    rng = np.random.default_rng(3)
    for sol in ((q1u, q2u), (q1d, q2d)):
        q0 = np.array(sol)[:, None] + rng.uniform(-0.3, 0.3, (2, 8))
        out, flags, _, _ = o.project(q0, tol=1e-13, max_iters=50, lam=0.0)
        assert np.all(flags & orc.CONVERGED)
        err = np.angle(np.exp(1j * (out - np.array(sol)[:, None])))
        assert np.abs(err).max() < 1e-10


# ---------------------------------------------------------------------------
# Forward kinematics: local-frame recursion vs the product-of-exponentials
# formula T(q) = exp([S_1] q_1) ... exp([S_n] q_n) M (screw axes at q = 0).
# ---------------------------------------------------------------------------
def _poe_fk(rb, q, link):
    """Pose of joint frame `link` by the product of exponentials (chain to root)."""
    chain = []
    j = link
    while j >= 0:
        chain.append(j)
        j = rb.parent[j]
    chain.reverse()
    H0 = np.eye(4)
    out = np.eye(4)
    for j in chain:
        H0 = H0 @ _h(rb.X[j])          # joint frame at q = 0
        w = H0[:3, 2]
        p = H0[:3, 3]
        S = np.zeros((4, 4))
        if rb.type[j] == W.REVOLUTE:
            S[:3, :3] = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
            S[:3, 3] = -np.cross(w, p)
        else:
            S[:3, 3] = w
        out = out @ expm(S * q[j])
    return out @ H0


@pytest.mark.parametrize("which", ["arm", "tree0", "tree1", "humanoid"])
def test_fk_matches_product_of_exponentials(which):
    if which == "arm":
        rb = W.dh_arm_robot(W.arm_link_lengths(3))
    elif which == "humanoid":
        rb, _ = W.humanoid_robot(7)
    else:
        rb = W.random_tree_robot(int(which[-1]), n_joints=9)
    o = orc.Oracle(rb)
    rng = np.random.default_rng(5)
    for _ in range(3):
        q = rng.uniform(-2.5, 2.5, rb.n_joints)
        Tj, Tf = o.fk(q)
        for j in range(rb.n_joints):
            np.testing.assert_allclose(_h(Tj[j]), _poe_fk(rb, q, j), atol=1e-12)


def test_fk_one_joint_circle():
    """A single revolute joint moves an offset point on a circle of its radius."""
    X = _rt(np.eye(3), (0.2, -0.1, 0.3))[None]
    rb = W.Robot(parent=np.array([-1], np.int32), type=np.zeros(1, np.int32), X=X, lower=-np.ones(1) * 9,
                 upper=np.ones(1) * 9, mass=np.ones(1), com=np.zeros((1, 3)), sphere_link=np.zeros(0, np.int32),
                 sphere=np.zeros((0, 4)), frame_link=np.array([0], np.int32),
                 frame_X=_rt(np.eye(3), (0.5, 0, 0))[None])
    o = orc.Oracle(rb)
    for q in np.linspace(-3, 3, 13):
        _, Tf = o.fk(np.array([q]))
        p = Tf[0].reshape(3, 4)[:, 3]
        np.testing.assert_allclose(p, [0.2 + 0.5 * math.cos(q), -0.1 + 0.5 * math.sin(q), 0.3], atol=1e-15)


# ---------------------------------------------------------------------------
# SO(3) log map vs scipy's rotation-vector routine; inverse left Jacobian vs
# the textbook left Jacobian and vs finite differences of log(exp(d) exp(phi)).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [0.0, 1e-9, 1e-5, 9.99e-4, 1.001e-3, 0.3, 1.5, 2.3, 0.75 * math.pi - 1e-9,
                                   0.75 * math.pi + 1e-9, 3.0, math.pi - 1e-4, math.pi - 1e-7])
def test_log_map_matches_rotvec(theta):
    rng = np.random.default_rng(int(theta * 1e6) % 1000)
    for _ in range(5):
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        R = Rotation.from_rotvec(theta * axis).as_matrix()
        phi = orc.so3_log(R)
        ref = Rotation.from_matrix(R).as_rotvec()
        if theta > math.pi - 1e-3 and np.dot(phi, ref) < 0:   # both +-pi*axis are logs near pi
            ref = -ref
        np.testing.assert_allclose(phi, ref, atol=1e-9)


def _left_jac(phi):
    th = np.linalg.norm(phi)
    P = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-3:
        return np.eye(3) + 0.5 * P + P @ P / 6.0
    return np.eye(3) + (1 - math.cos(th)) / th ** 2 * P + (th - math.sin(th)) / th ** 3 * P @ P


@pytest.mark.parametrize("th", [1e-6, 5e-3, 0.2, 1.4, 2.9])
def test_left_jacobian_inverse(th):
    rng = np.random.default_rng(11)
    axis = rng.standard_normal(3)
    phi = th * axis / np.linalg.norm(axis)
    Jinv = orc.so3_left_jac_inv(phi)
    np.testing.assert_allclose(Jinv @ _left_jac(phi), np.eye(3), atol=1e-12)
    h = 1e-6
    R = Rotation.from_rotvec(phi)
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (Rotation.from_rotvec(e) * R).as_rotvec() - (Rotation.from_rotvec(-e) * R).as_rotvec()
        np.testing.assert_allclose(fd / (2 * h), Jinv[:, i], atol=2e-8)


# ---------------------------------------------------------------------------
# Residual closed forms
# ---------------------------------------------------------------------------
def test_pose_residual_closed_form_single_joint():
    """One revolute joint about world z: T_err = P^-1 Rz(q) Q^-1; with P = Q = I
    the residual is (0, 0, 0, 0, 0, q) for |q| < pi."""
    X = W.IDENTITY12[None].copy()
    rb = W.Robot(parent=np.array([-1], np.int32), type=np.zeros(1, np.int32), X=X, lower=-np.ones(1) * 9,
                 upper=np.ones(1) * 9, mass=np.ones(1), com=np.zeros((1, 3)), sphere_link=np.zeros(0, np.int32),
                 sphere=np.zeros((0, 4)), frame_link=np.array([0], np.int32), frame_X=W.IDENTITY12[None].copy())
    o = orc.Oracle(rb, [W.Constraint(W.C_POSE, frame_a=0)])
    for q in (-2.0, -0.4, 0.0, 0.7, 2.5):
        np.testing.assert_allclose(o.residual(np.array([q])), [0, 0, 0, 0, 0, q], atol=1e-15)
    # TSR frame translated by (1, 0, 0): the error translation is R(-)... = (-1, 0, 0)
    P = _rt(np.eye(3), (1.0, 0.0, 0.0))
    o2 = orc.Oracle(rb, [W.Constraint(W.C_POSE, frame_a=0, P=P)])
    np.testing.assert_allclose(o2.residual(np.array([0.3])), [-1, 0, 0, 0, 0, 0.3], atol=1e-15)


def test_references_from_q_ref_zero_the_residual():
    wl = W.humanoid_workload(n=4)
    o = orc.Oracle(wl.robot, wl.constraints)
    F = o.residual(wl.extra["q_nom"])
    # feet and hands are exactly at their references; the CoM is generally not
    # at the support centre at the nominal stance
    np.testing.assert_allclose(F[:18], 0.0, atol=1e-14)
    _, Tf = o.fk(wl.extra["q_nom"])
    P, _, target = o.constraint_values(3)
    mid = 0.5 * (Tf[0].reshape(3, 4)[:2, 3] + Tf[1].reshape(3, 4)[:2, 3])
    np.testing.assert_allclose(target[:2], mid, atol=1e-15)
    wl2 = W.dual_arm_workload(total=10)
    o2 = orc.Oracle(wl2.robot, wl2.constraints)
    np.testing.assert_allclose(o2.residual(wl2.extra["q_ref"]), 0.0, atol=1e-14)
    wl3 = W.dual_rod_workload(n=1)
    o3 = orc.Oracle(wl3.robot, wl3.constraints)
    np.testing.assert_allclose(o3.residual(wl3.extra["q_ref"]), 0.0, atol=1e-14)
    for task in ("tray", "peg", "tsr"):
        wl4 = W.arm_task_workload(task, n=1)
        o4 = orc.Oracle(wl4.robot, wl4.constraints)
        # the plane / line / TSR pass through the end effector at q_ref, where
        # the end effector's z-axis is vertical as well
        np.testing.assert_allclose(o4.residual(wl4.extra["q_ref"]), 0.0, atol=1e-14)


def test_axis_align_residual_is_ee_z_axis():
    rb = W.dh_arm_robot(W.arm_link_lengths(3))
    o = orc.Oracle(rb, [W.Constraint(W.C_AXIS_ALIGN, frame_a=0)])
    q = np.random.default_rng(1).uniform(-2, 2, 7)
    T = _poe_fk(rb, q, 6) @ _h(rb.frame_X[0])
    np.testing.assert_allclose(o.residual(q), T[:2, 2], atol=1e-13)


# ---------------------------------------------------------------------------
# CoM invariants
# ---------------------------------------------------------------------------
def test_com_invariants():
    rb, names = W.humanoid_robot(3)
    o = orc.Oracle(rb)
    q = W.humanoid_nominal(names)
    x0, M = o.com(q)
    assert abs(M - rb.mass.sum()) < 1e-12
    t = np.array([0.3, -0.7, 0.25])
    q2 = q.copy()
    q2[:3] += t            # base_x, base_y, base_z are prismatic along world x, y, z
    x1, _ = o.com(q2)
    np.testing.assert_allclose(x1 - x0, t, atol=1e-14)
    # yaw of the whole body about the base z axis rotates the CoM about the base
    q3 = q.copy()
    q3[3] += 0.5
    x3, _ = o.com(q3)
    c, s = math.cos(0.5), math.sin(0.5)
    base = q[:3]
    d0 = x0 - base
    np.testing.assert_allclose(x3 - base, [c * d0[0] - s * d0[1], s * d0[0] + c * d0[1], d0[2]], atol=1e-14)


# ---------------------------------------------------------------------------
# Analytic Jacobians vs central finite differences of the residual.
# ---------------------------------------------------------------------------
def _cases():
    tree = W.random_tree_robot(4, n_joints=10, n_frames=3)
    yield "sphere", cartesian_robot(), [W.Constraint(W.C_SPHERE, target=np.array([1.0, 0, 0]))]
    arm = W.dh_arm_robot(W.arm_link_lengths(3))
    yield "axis", arm, [W.Constraint(W.C_AXIS_ALIGN, frame_a=0)]
    rng = np.random.default_rng(2)
    P = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    Q = _rt(W.random_rotation(rng), rng.uniform(-0.2, 0.2, 3))
    yield "pose", tree, [W.Constraint(W.C_POSE, frame_a=1, P=P, Q=Q)]
    yield "rel", tree, [W.Constraint(W.C_REL_POSE, frame_a=0, frame_b=2, P=P)]
    yield "com", tree, [W.Constraint(W.C_COM_XY, target=np.array([0.1, 0.2, 0]))]
    wl = W.humanoid_workload(n=4)
    yield "humanoid", wl.robot, wl.constraints
    wl2 = W.dual_arm_workload(total=10)
    yield "dual", wl2.robot, wl2.constraints
    yield "plane", tree, [W.Constraint(W.C_PLANE, frame_a=1, P=P)]
    yield "line", tree, [W.Constraint(W.C_LINE, frame_a=2, P=P)]
    yield "dist", tree, [W.Constraint(W.C_DIST, frame_a=0, frame_b=2, target=np.array([0.3, 0, 0]))]
    # bounds: some components pinned to zero (always active), some wide (always
    # inactive), so that no finite difference straddles a bound
    lo = np.array([0.0, -50.0, 0.0, -50.0, 0.0, 0.0])
    yield "tsr", tree, [W.Constraint(W.C_POSE_BOUNDED, frame_a=1, P=P, Q=Q, B=np.concatenate([lo, -lo]))]
    yield "rod", W.dual_rod_workload(n=1).robot, W.dual_rod_workload(n=1).constraints
    poly = np.array([-0.1, -0.1, 0.1, -0.1, 0.1, 0.1, -0.1, 0.1, 0, 0, 0, 0])
    yield "hull", tree, [W.Constraint(W.C_COM_HULL, target=np.array([4.0, 0.0, 0.0]), B=poly)]


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_jacobian_matches_finite_differences(case):
    name, rb, cons = case
    o = orc.Oracle(rb, cons)
    rng = np.random.default_rng(9)
    h = 1e-6
    for _ in range(4):
        if name == "humanoid":
            q = W.humanoid_workload(n=1, seed=int(rng.integers(1 << 30))).q[:, 0]
        else:
            q = rng.uniform(-1.5, 1.5, rb.n_joints)
            if name == "sphere":
                q = q + 0.5 * np.sign(q)
        F, J = o.residual_jacobian(q)
        Jfd = np.zeros_like(J)
        for j in range(rb.n_joints):
            e = np.zeros(rb.n_joints)
            e[j] = h
            Jfd[:, j] = (o.residual(q + e) - o.residual(q - e)) / (2 * h)
        np.testing.assert_allclose(J, Jfd, atol=2e-7 * max(1.0, np.abs(J).max()), rtol=1e-6)


# ---------------------------------------------------------------------------
# Convergence invariant and cyclic/stacked agreement
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["arm", "dual", "humanoid", "tray", "peg", "tsr", "rod", "rod_cyclic",
                                  "tsr_cyclic"])
def test_converged_configs_satisfy_tolerance(name):
    if name == "arm":
        wl = W.arm_workload(n=256)
    elif name == "dual":
        wl = W.dual_arm_workload(total=10, n_random=256)
    elif name in ("tray", "peg", "tsr", "tsr_cyclic"):
        wl = W.arm_task_workload(name.split("_")[0], n=256)
    elif name in ("rod", "rod_cyclic"):
        wl = W.dual_rod_workload(n=256)
    else:
        wl = W.humanoid_workload(n=128)
    o = orc.Oracle(wl.robot, wl.constraints)
    p = wl.params
    out, flags, iters, resid = o.project(wl.q, p.tol, p.max_iters, p.lam, cyclic=name.endswith("cyclic"))
    conv = (flags & orc.CONVERGED) != 0
    assert conv.mean() > 0.8
    for i in np.flatnonzero(conv)[:64]:
        assert np.linalg.norm(o.residual(out[:, i])) < p.tol
        assert abs(np.linalg.norm(o.residual(out[:, i])) - resid[i]) < 1e-15
    assert np.all(iters[conv] <= p.max_iters)
    capped = (flags & orc.CAP) != 0
    assert np.all(iters[capped] == p.max_iters)


def test_one_dof_axis_alignment_brute_force():
    """1 revolute joint about world x: z_ee = (0, -sin q, cos q); the iteration
    is Newton on sin q = 0 and converges to the nearest multiple of pi for
    starts within pi/4 of it (checked on a 1e-3 grid)."""
    X = _rt(np.array([[0, 0, 1.0], [0, 1, 0], [-1, 0, 0]]), (0, 0, 0))[None]   # joint z -> world x
    rb = W.Robot(parent=np.array([-1], np.int32), type=np.zeros(1, np.int32), X=X, lower=-np.ones(1) * 9,
                 upper=np.ones(1) * 9, mass=np.ones(1), com=np.zeros((1, 3)), sphere_link=np.zeros(0, np.int32),
                 sphere=np.zeros((0, 4)),
                 frame_link=np.array([0], np.int32),
                 frame_X=_rt(np.array([[0, 0, -1.0], [0, 1, 0], [1, 0, 0]]), (0, 0, 0))[None])
    o = orc.Oracle(rb, [W.Constraint(W.C_AXIS_ALIGN, frame_a=0)])
    _, Tf = o.fk(np.array([0.3]))
    z = Tf[0].reshape(3, 4)[:, 2]
    np.testing.assert_allclose(z, [0, -math.sin(0.3), math.cos(0.3)], atol=1e-15)
    q0 = np.arange(-0.78, 0.78, 1e-3)[None, :]
    out, flags, _, _ = o.project(q0, tol=1e-12, max_iters=50, lam=1e-12)
    assert np.all(flags & orc.CONVERGED)
    assert np.abs(out).max() < 1e-11


def test_cyclic_equals_stacked_for_one_constraint():
    wl = W.arm_workload(n=64)
    o = orc.Oracle(wl.robot, wl.constraints)
    a = o.project(wl.q, 1e-5, 30, 1e-6, cyclic=False)
    b = o.project(wl.q, 1e-5, 30, 1e-6, cyclic=True)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_cyclic_converges_on_humanoid():
    """Cyclic projection (one LM step per constraint per sweep) is alternating
    projection onto four coupled manifolds: it converges, linearly and far more
    slowly than the stacked step (hundreds of sweeps here)."""
    wl = W.humanoid_workload(n=16)
    o = orc.Oracle(wl.robot, wl.constraints)
    out, flags, iters, _ = o.project(wl.q, 1e-5, 1500, 1e-6, cyclic=True)
    conv = (flags & orc.CONVERGED) != 0
    assert conv.mean() > 0.9
    assert np.median(iters[conv]) > 40
    for i in np.flatnonzero(conv):
        assert np.linalg.norm(o.residual(out[:, i])) < 1e-5


def test_divergence_exit_keeps_last_iterate():
    rb = cartesian_robot()
    o = orc.Oracle(rb, [W.Constraint(W.C_SPHERE, target=np.array([1.0, 0, 0]))])
    q0 = np.array([[3.0], [0.0], [0.0]])     # the Newton step has length 2
    out, flags, iters, _ = o.project(q0, tol=1e-8, max_iters=50, lam=0.0, max_step=1.0)
    assert flags[0] & orc.DIVERGED
    assert iters[0] == 0
    np.testing.assert_array_equal(out, q0)


# ---------------------------------------------------------------------------
# Collision: hand-made tangent and near-tangent cases (strict inequality).
# ---------------------------------------------------------------------------
def test_collision_hand_cases():
    # exactly representable radii/positions: robot sphere r = 1/8, obstacle r = 1/4
    rb = cartesian_robot(extra_sphere_r=0.125)
    obst = W.Obstacles(spheres=np.array([[1.0, 0.0, 0.0, 0.25]]),
                       aabbs=np.array([[-1.0, -1.0, -1.0, -0.5, -0.5, -0.5]]))
    o = orc.Oracle(rb, [], obst)
    eps = 2.0 ** -30
    q = np.array([[0.625 - eps, 0.625 + eps, 0.625, 0.0, -0.75, -0.375 + eps, -0.375 - eps],
                  [0.0, 0.0, 0.0, 0.0, -0.75, -0.625, -0.625],
                  [0.0, 0.0, 0.0, 0.0, -0.75, -0.625, -0.625]])
    hit, margin = o.check(q)
    # outside by eps / penetrating by eps / exactly touching (free: strict <) /
    # far / inside the box / outside a box face by eps / inside the face band
    assert hit.tolist() == [0, 1, 0, 0, 1, 0, 1]
    assert margin[2] == 0.0 and abs(margin[0] - eps) < 1e-15
    # a world-fixed sphere (link -1) does not move with q
    rb2 = cartesian_robot(extra_sphere_r=0.125)
    rb2.sphere_link = np.array([-1], np.int32)
    rb2.sphere = np.array([[1.0, 0.0, 0.0, 0.125]])
    hit2, _ = orc.Oracle(rb2, [], obst).check(np.zeros((3, 2)))
    assert hit2.tolist() == [1, 1]


def test_collision_corner_of_box():
    """Sphere near a box corner: the distance is to the corner, not to a face."""
    rb = cartesian_robot(extra_sphere_r=0.1)
    obst = W.Obstacles(spheres=np.zeros((0, 4)), aabbs=np.array([[0.0, 0.0, 0.0, 1.0, 1.0, 1.0]]))
    o = orc.Oracle(rb, [], obst)
    d = 0.1 / math.sqrt(3)
    q = np.array([[1 + d * 0.99, 1 + d * 1.01], [1 + d * 0.99, 1 + d * 1.01], [1 + d * 0.99, 1 + d * 1.01]])
    hit, _ = o.check(q)
    assert hit.tolist() == [1, 0]


# ---------------------------------------------------------------------------
# VJP: projector identities, the sphere closed form and finite differences of
# the projection map evaluated at a point on the manifold.
# ---------------------------------------------------------------------------
def test_vjp_sphere_closed_form():
    rb = cartesian_robot()
    o = orc.Oracle(rb, [W.Constraint(W.C_SPHERE, target=np.array([1.0, 0, 0]))])
    rng = np.random.default_rng(4)
    q = rng.standard_normal((3, 50))
    q /= np.linalg.norm(q, axis=0)
    g = rng.standard_normal((3, 50))
    v, flags = o.vjp(q, g)
    np.testing.assert_allclose(v, g - (g * q).sum(0) * q, atol=1e-14)
    assert not flags.any()


@pytest.mark.parametrize("name", ["dual", "humanoid"])
def test_vjp_projector_identities(name):
    if name == "dual":
        wl = W.dual_arm_workload(total=10, n_random=4)
    else:
        wl = W.humanoid_workload(n=4)
    o = orc.Oracle(wl.robot, wl.constraints)
    qs, flags, _, _ = o.project(wl.q, 1e-12, 60, 0.0)
    d = wl.dof
    for i in np.flatnonzero(flags & orc.CONVERGED)[:2]:
        q = np.repeat(qs[:, i:i + 1], d, axis=1)
        P, _ = o.vjp(q, np.eye(d))          # column j = P e_j
        np.testing.assert_allclose(P @ P, P, atol=1e-10)
        np.testing.assert_allclose(P, P.T, atol=1e-10)
        _, J = o.residual_jacobian(qs[:, i])
        np.testing.assert_allclose(P @ J.T, 0.0, atol=1e-10)
        assert abs(np.trace(P) - (d - wl.k)) < 1e-9


def test_vjp_matches_finite_differences_of_projection():
    """d Pi / d q at q* (lambda = 0, tight tol) contracted with g equals the VJP."""
    wl = W.dual_arm_workload(total=10, n_random=3)
    o = orc.Oracle(wl.robot, wl.constraints)
    qs, flags, _, _ = o.project(wl.q, 1e-13, 80, 0.0)
    rng = np.random.default_rng(8)
    h = 1e-4
    for i in np.flatnonzero(flags & orc.CONVERGED)[:2]:
        q = qs[:, i]
        g = rng.standard_normal(14)
        cols = []
        for j in range(14):
            e = np.zeros(14)
            e[j] = h
            pp = o.project(np.stack([q + e, q - e], 1), 1e-13, 80, 0.0)[0]
            cols.append((pp[:, 0] - pp[:, 1]) / (2 * h))
        D = np.stack(cols, 1)
        v, _ = o.vjp(q[:, None], g[:, None])
        ref = g @ D
        assert np.linalg.norm(v[:, 0] - ref) / np.linalg.norm(ref) < 1e-4


# ---------------------------------------------------------------------------
# Residual values at arbitrary q vs an independent evaluation: product-of-
# exponentials kinematics and scipy's rotation vector as the SO(3) log.
# ---------------------------------------------------------------------------
def _frame_poe(rb, q, f):
    return _poe_fk(rb, q, rb.frame_link[f]) @ _h(rb.frame_X[f])


def _err6(T):
    return np.concatenate([T[:3, 3], Rotation.from_matrix(T[:3, :3]).as_rotvec()])


def test_residual_values_match_independent_evaluation():
    tree = W.random_tree_robot(6, n_joints=10, n_frames=3)
    rng = np.random.default_rng(12)
    P = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    Q = _rt(W.random_rotation(rng), rng.uniform(-0.2, 0.2, 3))
    Tref = _rt(W.random_rotation(rng), rng.uniform(-0.5, 0.5, 3))
    cons = [W.Constraint(W.C_POSE, frame_a=1, P=P, Q=Q), W.Constraint(W.C_REL_POSE, frame_a=0, frame_b=2, P=Tref),
            W.Constraint(W.C_COM_XY, target=np.array([0.3, -0.1, 0.0])), W.Constraint(W.C_AXIS_ALIGN, frame_a=2)]
    o = orc.Oracle(tree, cons)
    checked = 0
    for _ in range(40):
        q = rng.uniform(-2, 2, tree.n_joints)
        F = o.residual(q)
        pose = np.linalg.inv(_h(P)) @ _frame_poe(tree, q, 1) @ np.linalg.inv(_h(Q))
        rel = np.linalg.inv(_h(Tref)) @ np.linalg.inv(_frame_poe(tree, q, 0)) @ _frame_poe(tree, q, 2)
        if max(np.linalg.norm(_err6(pose)[3:]), np.linalg.norm(_err6(rel)[3:])) > math.pi - 1e-3:
            continue          # the log is two-valued at pi
        com = sum(tree.mass[i] * (_poe_fk(tree, q, i) @ np.append(tree.com[i], 1.0))[:3]
                  for i in range(tree.n_joints)) / tree.mass.sum()
        expect = np.concatenate([_err6(pose), _err6(rel), com[:2] - [0.3, -0.1], _frame_poe(tree, q, 2)[:2, 2]])
        np.testing.assert_allclose(F, expect, atol=1e-11)
        checked += 1
    assert checked > 30


# ---------------------------------------------------------------------------
# Task constraints beyond B^w = 0 (Sec. II bounded TSRs, Sec. III task
# constraints, Sec. V-C closed linkages): closed forms on Cartesian points,
# where one Newton step from any start is the Euclidean projection.
# ---------------------------------------------------------------------------
def _two_points():
    a = cartesian_robot()
    return W._merge_robots(a, cartesian_robot())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plane_and_line_one_step_are_orthogonal_projections(seed):
    rng = np.random.default_rng(40 + seed)
    R = W.random_rotation(rng)
    c = rng.uniform(-1, 1, 3)
    P = _rt(R, c)
    n, dl = R[:, 2], R[:, 2]
    rb = cartesian_robot()
    p0 = rng.uniform(-1.5, 1.5, (3, 16))
    op = orc.Oracle(rb, [W.Constraint(W.C_PLANE, frame_a=0, P=P)])
    # the residual is the signed distance to the plane
    np.testing.assert_allclose(op.residual(p0[:, 0]), [n @ (p0[:, 0] - c)], atol=1e-14)
    out, fl, it, _ = op.project(p0, 1e-12, 1, 0.0)
    expect = p0 - np.outer(n, n @ (p0 - c[:, None]))
    np.testing.assert_allclose(out, expect, atol=1e-13)
    ol = orc.Oracle(rb, [W.Constraint(W.C_LINE, frame_a=0, P=P)])
    out, fl, it, _ = ol.project(p0, 1e-12, 1, 0.0)
    expect = c[:, None] + np.outer(dl, dl @ (p0 - c[:, None]))
    np.testing.assert_allclose(out, expect, atol=1e-13)
    # the distance to the line is the norm of the residual
    r = ol.residual(p0[:, 1])
    np.testing.assert_allclose(np.linalg.norm(r), np.linalg.norm(np.cross(p0[:, 1] - c, dl)), atol=1e-14)


def test_distance_constraint_one_step_moves_both_points_symmetrically():
    """F = |b - a| - L with J = [-u^T, u^T]: the minimum-norm step moves a and b
    by F/2 each along u = (b - a)/|b - a|, which lands exactly on |b - a| = L."""
    rb = _two_points()
    rng = np.random.default_rng(44)
    o = orc.Oracle(rb, [W.Constraint(W.C_DIST, frame_a=0, frame_b=1, target=np.array([0.7, 0, 0]))])
    q0 = rng.uniform(-1, 1, (6, 32))
    out, fl, it, res = o.project(q0, 1e-12, 1, 0.0)
    a, b = q0[:3], q0[3:]
    e = b - a
    nrm = np.linalg.norm(e, axis=0)
    u = e / nrm
    F = nrm - 0.7
    np.testing.assert_allclose(out[:3], a + u * F / 2, atol=1e-14)
    np.testing.assert_allclose(out[3:], b - u * F / 2, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(out[3:] - out[:3], axis=0), 0.7, atol=1e-14)


def test_bounded_tsr_zero_bounds_is_the_pose_constraint():
    tree = W.random_tree_robot(4, n_joints=10, n_frames=3)
    rng = np.random.default_rng(45)
    P = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    Q = _rt(W.random_rotation(rng), rng.uniform(-0.2, 0.2, 3))
    a = orc.Oracle(tree, [W.Constraint(W.C_POSE, frame_a=1, P=P, Q=Q)])
    b = orc.Oracle(tree, [W.Constraint(W.C_POSE_BOUNDED, frame_a=1, P=P, Q=Q, B=np.zeros(12))])
    for _ in range(8):
        q = rng.uniform(-1.5, 1.5, tree.n_joints)
        Fa, Ja = a.residual_jacobian(q)
        Fb, Jb = b.residual_jacobian(q)
        np.testing.assert_array_equal(Fa, Fb)
        np.testing.assert_array_equal(Ja, Jb)


def test_bounded_tsr_projects_a_point_onto_its_box():
    """Translation bounds on a Cartesian point: the TSR set is a box and the
    step moves only the violated coordinates, onto the box faces (clamp)."""
    rb = cartesian_robot()
    rng = np.random.default_rng(46)
    R = W.random_rotation(rng)
    c = rng.uniform(-0.5, 0.5, 3)
    half = np.array([0.2, 0.1, 0.3])
    inf = np.full(3, np.inf)
    B = np.concatenate([-half, -inf, half, inf])
    o = orc.Oracle(rb, [W.Constraint(W.C_POSE_BOUNDED, frame_a=0, P=_rt(R, c), B=B)])
    p0 = rng.uniform(-1.2, 1.2, (3, 64))
    local = R.T @ (p0 - c[:, None])
    # inactive rows carry lambda only: lambda = 1e-14 leaves the active step exact to ~1e-14
    out, fl, it, _ = o.project(p0, 1e-12, 1, 1e-14)
    expect = c[:, None] + R @ np.clip(local, -half[:, None], half[:, None])
    np.testing.assert_allclose(out, expect, atol=1e-12)
    inside = (np.abs(local) <= half[:, None]).all(axis=0)
    assert inside.any() and (~inside).any()
    np.testing.assert_array_equal(out[:, inside], p0[:, inside])


def test_bounded_tsr_yaw_interval():
    """One revolute joint about z with the TSR's yaw bounded to [-0.2, 0.3]: the
    valid set is that interval and a start outside lands on its nearer end."""
    rb = W.Robot(parent=np.array([-1], np.int32), type=np.zeros(1, np.int32), X=_rt(np.eye(3), 0)[None],
                 lower=np.full(1, -3.0), upper=np.full(1, 3.0), mass=np.ones(1), com=np.zeros((1, 3)),
                 sphere_link=np.zeros(0, np.int32), sphere=np.zeros((0, 4)), frame_link=np.array([0], np.int32),
                 frame_X=_rt(np.eye(3), (0.4, 0, 0))[None])
    B = np.array([-np.inf] * 5 + [-0.2] + [np.inf] * 5 + [0.3])
    B[0:3], B[6:9] = -1.0, 1.0           # translation bounds wide enough for the 0.4 m offset
    o = orc.Oracle(rb, [W.Constraint(W.C_POSE_BOUNDED, frame_a=0, B=B)])
    qs = np.array([[-1.0, -0.5, -0.1, 0.0, 0.25, 0.6, 1.4]])
    out, fl, it, _ = o.project(qs, 1e-12, 5, 1e-14)
    expect = np.clip(qs, -0.2, 0.3)
    np.testing.assert_allclose(out, expect, atol=1e-12)


def test_cyclic_sweep_equals_stacked_step_on_decoupled_linear_constraints():
    """Two planes, each on its own Cartesian point: J is block diagonal, so one
    cyclic sweep (a step per constraint) and one stacked step coincide, and both
    land on the closed-form projections."""
    rb = _two_points()
    rng = np.random.default_rng(47)
    Pa = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    Pb = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    cons = [W.Constraint(W.C_PLANE, frame_a=0, P=Pa), W.Constraint(W.C_PLANE, frame_a=1, P=Pb)]
    o = orc.Oracle(rb, cons)
    q0 = rng.uniform(-1, 1, (6, 16))
    s = o.project(q0, 1e-12, 1, 0.0, cyclic=False)[0]
    c = o.project(q0, 1e-12, 1, 0.0, cyclic=True)[0]
    np.testing.assert_allclose(s, c, atol=1e-14)
    na, ca = Pa.reshape(3, 4)[:, 2], Pa.reshape(3, 4)[:, 3]
    np.testing.assert_allclose(c[:3], q0[:3] - np.outer(na, na @ (q0[:3] - ca[:, None])), atol=1e-13)


def test_cyclic_sweep_is_sequential_on_coupled_constraints():
    """Two planes on the same point: a sweep projects onto plane a, then from
    there onto plane b (alternating projections), which is not the stacked
    step; iterated, it converges to the intersection line."""
    rb = cartesian_robot()
    rng = np.random.default_rng(48)
    Pa = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    Pb = _rt(W.random_rotation(rng), rng.uniform(-1, 1, 3))
    o = orc.Oracle(rb, [W.Constraint(W.C_PLANE, frame_a=0, P=Pa), W.Constraint(W.C_PLANE, frame_a=0, P=Pb)])
    q0 = rng.uniform(-1, 1, (3, 8))
    na, ca = Pa.reshape(3, 4)[:, 2], Pa.reshape(3, 4)[:, 3]
    nb, cb = Pb.reshape(3, 4)[:, 2], Pb.reshape(3, 4)[:, 3]
    x = q0 - np.outer(na, na @ (q0 - ca[:, None]))
    x = x - np.outer(nb, nb @ (x - cb[:, None]))
    np.testing.assert_allclose(o.project(q0, 1e-12, 1, 0.0, cyclic=True)[0], x, atol=1e-13)
    out, fl, it, _ = o.project(q0, 1e-10, 500, 0.0, cyclic=True)
    assert (fl & orc.CONVERGED).all()
    np.testing.assert_allclose(na @ (out - ca[:, None]), 0.0, atol=1e-10)
    np.testing.assert_allclose(nb @ (out - cb[:, None]), 0.0, atol=1e-10)


# ---------------------------------------------------------------------------
# ParallelConstrainedExtend (Algorithm 2) on the unit sphere: with lambda = 0
# one Newton step on ||q|| - 1 is the radial projection q / ||q||, so every
# particle converges after one step (the lowest index wins), each projected
# point is a normalised chord point, and a bisection midpoint is the exact
# angular bisector of its gap.
# ---------------------------------------------------------------------------
def _sphere_extend_setup(n=8):
    wl = W.sphere_workload(n_pairs=2)
    rb = wl.robot
    cons = wl.constraints
    p = W.Params(tol=1e-12, max_iters=20, lam=0.0)
    return rb, cons, p, n


def _unit(v):
    return v / np.linalg.norm(v)


def _expected(qs, qp, n, r, delta):
    """(status, points) from the geometry of the arc: the n interpolated
    points sit at angles atan2(t sin th, (1 - t) + t cos th), t = k / (n + 1),
    along the great circle from q_s to q_proj; a chord longer than r / n is a
    GAP exit after 1 + n points; otherwise a gap of angle phi needs 2^L - 1
    bisection midpoints, L the least level with 2 sin(phi / 2^(L + 1)) <= delta."""
    ang = [0.0]
    th = math.acos(np.clip(qs @ qp, -1, 1))
    for k in range(1, n + 1):
        t = k / (n + 1)
        ang.append(math.atan2(t * math.sin(th), (1 - t) + t * math.cos(th)))
    ang.append(th)
    gaps = [b - a for a, b in zip(ang[:-1], ang[1:])]
    if max(2 * math.sin(g / 2) for g in gaps) > r / n:
        return orc.EXT_GAP, 1 + n
    total = 1 + n
    for phi in gaps:
        L = 0
        while 2 * math.sin(phi / 2 ** (L + 1)) > delta:
            L += 1
        total += 2 ** L - 1
    return orc.EXT_OK, total


def test_extend_on_sphere_closed_form():
    rb, cons, p, n = _sphere_extend_setup()
    o = orc.Oracle(rb, cons)
    rng = np.random.default_rng(60)
    m = 24
    qs = np.stack([_unit(rng.standard_normal(3)) for _ in range(m)], 1)
    qt = np.stack([_unit(rng.standard_normal(3)) for _ in range(m)], 1) * 1.3
    eps = 0.03 * rng.standard_normal((n, m))
    r, delta = 0.5, 0.03
    qp, st, npts, win = o.extend(qs, qt, eps, p, r, delta)
    seen = set()
    for i in range(m):
        v = qt[:, i] - qs[:, i]
        dist = min(np.linalg.norm(v), r)
        v = v / np.linalg.norm(v)
        expect = _unit(qs[:, i] + (dist + eps[0, i]) * v)
        assert win[i] == 0
        np.testing.assert_allclose(qp[:, i], expect, atol=1e-14)
        status, points = _expected(qs[:, i], expect, n, r, delta)
        assert st[i] == status and npts[i] == points, (i, st[i], status, npts[i], points)
        seen.add(int(st[i]))
    assert seen == {orc.EXT_OK, orc.EXT_GAP}


def test_extend_exits():
    rb, cons, p, n = _sphere_extend_setup()
    qs = np.array([[1.0], [0.0], [0.0]])
    qt = np.array([[0.0], [1.0], [0.0]])
    eps = np.zeros((n, 1))
    # q_t = q_s
    assert orc.Oracle(rb, cons).extend(qs, qs, eps, p, 0.5, 0.05)[1][0] == orc.EXT_DEGENERATE
    # every particle's first step exceeds MaxDistance
    p_div = W.Params(tol=1e-12, max_iters=20, lam=0.0, max_step=1e-6)
    assert orc.Oracle(rb, cons).extend(qs, qt, eps, p_div, 0.5, 0.05)[1][0] == orc.EXT_NO_PROJECTION
    # the winning particle lands more than 2 dist from q_s
    far = np.full((n, 1), 1.5)
    assert orc.Oracle(rb, cons).extend(qs, qt, far, p, 0.2, 0.05)[1][0] == orc.EXT_TOO_FAR
    # an obstacle on q_proj, then one on the arc between q_s and q_proj
    dist = 0.5
    qproj = _unit(qs[:, 0] + dist * _unit(qt[:, 0] - qs[:, 0]))
    hit = W.Obstacles(spheres=np.array([[*qproj, 0.01]]), aabbs=np.zeros((0, 6)))
    assert orc.Oracle(rb, cons, hit).extend(qs, qt, eps, p, dist, 0.05)[1][0] == orc.EXT_PROJ_COLLISION
    mid = _unit(qs[:, 0] + qproj)
    hit2 = W.Obstacles(spheres=np.array([[*mid, 0.01]]), aabbs=np.zeros((0, 6)))
    assert orc.Oracle(rb, cons, hit2).extend(qs, qt, eps, p, dist, 0.05)[1][0] == orc.EXT_INTERP_COLLISION
    # no resolution within the depth cap
    assert orc.Oracle(rb, cons).extend(qs, qt, eps, p, dist, 1e-4, max_depth=2)[1][0] == orc.EXT_RESOLUTION


# ---------------------------------------------------------------------------
# Outer form of the LM step, (J^T J + lambda I)^{-1} J^T F (Alg. 2), and the
# step scale alpha.
# ---------------------------------------------------------------------------
def test_outer_step_is_least_squares_step():
    """With lambda = 0 and J of full column rank the outer step is the
    least-squares solution of J dq = F (numpy's lstsq)."""
    rb = cartesian_robot()
    rng = np.random.default_rng(70)
    cons = [W.Constraint(W.C_PLANE, frame_a=0, P=_rt(W.random_rotation(rng), rng.uniform(-1, 1, 3)))
            for _ in range(4)]
    o = orc.Oracle(rb, cons)
    q0 = rng.uniform(-1, 1, (3, 8))
    out = o.project(q0, 1e-13, 1, 0.0, outer=True)[0]
    for i in range(8):
        F, J = o.residual_jacobian(q0[:, i])
        np.testing.assert_allclose(out[:, i], q0[:, i] - np.linalg.lstsq(J, F, rcond=None)[0], atol=1e-13)


def test_outer_form_solves_consistent_overdetermined_system():
    """Four planes through one point, a Cartesian point (k = 4 > d = 3): the
    outer step lands on the common point in one step; the inner form's
    4 x 4 J J^T is singular at lambda = 0."""
    rb = cartesian_robot()
    rng = np.random.default_rng(71)
    c = rng.uniform(-0.5, 0.5, 3)
    cons = [W.Constraint(W.C_PLANE, frame_a=0, P=_rt(W.random_rotation(rng), c)) for _ in range(4)]
    o = orc.Oracle(rb, cons)
    q0 = rng.uniform(-1, 1, (3, 8))
    out, fl, it, _ = o.project(q0, 1e-10, 5, 0.0, outer=True)
    assert (fl & orc.CONVERGED).all() and (it == 1).all()
    np.testing.assert_allclose(out, np.repeat(c[:, None], 8, 1), atol=1e-12)
    assert (o.project(q0, 1e-10, 5, 0.0, outer=False)[1] & orc.NONFINITE).all()


def test_inner_and_outer_steps_agree_with_damping():
    """J^T (J J^T + lambda I)^{-1} = (J^T J + lambda I)^{-1} J^T for lambda > 0:
    one step of either form from the same start, on the 7-DoF arm."""
    wl = W.arm_workload(n=32)
    o = orc.Oracle(wl.robot, wl.constraints)
    a = o.project(wl.q, 1e-13, 1, 1e-3, outer=False)[0]
    b = o.project(wl.q, 1e-13, 1, 1e-3, outer=True)[0]
    np.testing.assert_allclose(a, b, atol=1e-9)


def test_step_scale_alpha():
    """On the unit sphere one full Newton step is the radial projection; with
    alpha the point moves that fraction of the way: q - alpha (|q| - 1) q / |q|."""
    wl = W.sphere_workload(n_pairs=2)
    o = orc.Oracle(wl.robot, wl.constraints)
    rng = np.random.default_rng(72)
    q0 = rng.uniform(-1.5, 1.5, (3, 16))
    nq = np.linalg.norm(q0, axis=0)
    for alpha in (0.5, 0.8):
        out = o.project(q0, 1e-13, 1, 0.0, alpha=alpha)[0]
        np.testing.assert_allclose(out, q0 - alpha * (nq - 1) * q0 / nq, atol=1e-14)


# ---------------------------------------------------------------------------
# CoM support-hull constraint (Sec. V-C): the CoM's xy distance to a convex
# polygon, zero inside.
# ---------------------------------------------------------------------------
def test_com_hull_residual_is_distance_to_polygon():
    """planar 2-link with all mass at the tip: the CoM is the tip, so the
    residual is the vector from the polygon's nearest point to the tip; checked
    against a brute-force nearest point on a densely sampled boundary."""
    rb = planar_2link(0.7, 0.5)
    square = np.array([0.2, -0.3, 0.8, -0.3, 0.8, 0.3, 0.2, 0.3, 0, 0, 0, 0])
    o = orc.Oracle(rb, [W.Constraint(W.C_COM_HULL, target=np.array([4.0, 0.0, 0.0]), B=square)])
    V = square[:8].reshape(4, 2)
    t = np.linspace(0, 1, 20001)[:, None]
    boundary = np.concatenate([V[i] + t * (V[(i + 1) % 4] - V[i]) for i in range(4)])
    rng = np.random.default_rng(90)
    inside_seen = outside_seen = 0
    for _ in range(60):
        q = rng.uniform(-3, 3, 2)
        tip = np.array([0.7 * math.cos(q[0]) + 0.5 * math.cos(q[0] + q[1]),
                        0.7 * math.sin(q[0]) + 0.5 * math.sin(q[0] + q[1])])
        F = o.residual(q)
        inside = (0.2 <= tip[0] <= 0.8) and (-0.3 <= tip[1] <= 0.3)
        if inside:
            inside_seen += 1
            np.testing.assert_array_equal(F, [0.0, 0.0])
        else:
            outside_seen += 1
            near = boundary[np.argmin(np.linalg.norm(boundary - tip, axis=1))]
            np.testing.assert_allclose(F, tip - near, atol=1e-4)
    assert inside_seen > 3 and outside_seen > 20


def test_com_hull_reference_box_and_humanoid_hull_projection():
    wl = W.humanoid_workload(n=64, hull=True)
    o = orc.Oracle(wl.robot, wl.constraints)
    _, Tf = o.fk(wl.extra["q_nom"])
    fa, fb = Tf[0].reshape(3, 4)[:, 3], Tf[1].reshape(3, 4)[:, 3]
    lo, hi = np.minimum(fa, fb)[:2] - 0.08, np.maximum(fa, fb)[:2] + 0.08
    B = o.bounds(3)
    np.testing.assert_allclose(B[:8], [lo[0], lo[1], hi[0], lo[1], hi[0], hi[1], lo[0], hi[1]], atol=1e-14)
    p = wl.params
    out, fl, it, res = o.project(wl.q, p.tol, p.max_iters, p.lam)
    conv = (fl & orc.CONVERGED) != 0
    assert conv.mean() > 0.9
    for i in np.flatnonzero(conv)[:16]:
        assert np.linalg.norm(o.residual(out[:, i])) < p.tol
