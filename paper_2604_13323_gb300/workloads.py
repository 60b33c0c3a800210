"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module holds *data* only: robot descriptions (kinematic trees of 1-DoF
joints), constraint descriptors, obstacle sets and batches of start
configurations.  It contains none of the projection arithmetic (no forward
kinematics, residuals, Jacobians or Newton steps); both sides compute those
independently from what is generated here.

The robots stand in for the paper's Panda / KUKA IIWA / Digit models (Sec. V),
which are not available.  Each workload mirrors the shape of one of the
paper's problem classes:

* ``sphere``    -- a point in R^3 on the unit sphere (the textbook manifold),
                   geodesics between random pairs interpolated at step 0.05.
* ``arm``       -- a 7-DoF serial (IIWA-like DH) arm with the end-effector
                   z-axis kept parallel to world z (the "upright mug" TSR of
                   Sec. II, two equations).
* ``dual_arm``  -- two copies of that arm, relative end-effector pose fixed
                   (the bimanual constraint, Eq. 2), uneven geodesic segments.
* ``humanoid``  -- a 36-DoF tree (6-DoF floating base, two 6-DoF legs, two
                   7-DoF arms, 4-DoF torso/neck) with both feet fixed (Eq. 1),
                   the hands in a fixed relative pose (Eq. 2) and the CoM xy at
                   the support-polygon centre (Sec. V-C), 20 equations.

Robot format (all arrays are numpy, row-major):
    parent[j]   int32, parent joint (< j), -1 = world
    type[j]     int32, 0 = revolute about the joint's local z, 1 = prismatic along it
    X[j]        float64[12], fixed 3x4 transform parent-joint frame -> this joint
                frame, applied before the joint motion:
                T_j = T_parent(j) * X_j * Jnt(q_j)
    lower/upper joint limits (reported only, never enforced)
    mass[j], com[j] (link j is rigidly attached to joint frame j)
    sphere_link[s], sphere[s] = (x, y, z, r) in that joint frame (-1 = world)
    frame_link[f], frame_X[f] = 3x4 offset of a task frame (end effector, foot, hand)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

REVOLUTE = 0
PRISMATIC = 1

C_SPHERE = 0      # F = ||q|| - r                       (k = 1)
C_AXIS_ALIGN = 1  # frame z-axis parallel to world z    (k = 2)
C_POSE = 2        # TSR pose error, Eq. 1, B^w = 0      (k = 6)
C_REL_POSE = 3    # relative pose error, Eq. 2          (k = 6)
C_COM_XY = 4      # centre-of-mass xy at a target point (k = 2)
C_PLANE = 5       # frame origin on the xy-plane of P   (k = 1)
C_LINE = 6        # frame origin on the z-axis of P     (k = 2)
C_DIST = 7        # |x_b - x_a| = L, closed linkage     (k = 1)
C_POSE_BOUNDED = 8  # TSR pose error outside bounds B^w (k = 6)
C_COM_HULL = 9    # CoM xy distance to the support polygon, zero inside (k = 2)

CONSTRAINT_DIM = {C_SPHERE: 1, C_AXIS_ALIGN: 2, C_POSE: 6, C_REL_POSE: 6, C_COM_XY: 2, C_PLANE: 1, C_LINE: 2,
                  C_DIST: 1, C_POSE_BOUNDED: 6, C_COM_HULL: 2}

# Precision selector of the projection entry point.
PREC_FP32 = 0   # FP32 Newton with FP64 acceptance
PREC_FP64 = 1   # plain FP64 throughout

# Exact signed-permutation rotations that carry the local z axis onto x / y / z.
_R_AXIS = {
    "x": np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]]),
    "y": np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]]),
    "z": np.eye(3),
}
# Rx(+pi/2) and Rx(-pi/2) written out exactly (DH twist angles).
_RX_PLUS = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])
_RX_MINUS = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]])


def _rt(R, t) -> np.ndarray:
    """Pack a rotation and a translation into a row-major 3x4 array of 12."""
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T.reshape(12)


IDENTITY12 = _rt(np.eye(3), np.zeros(3))


@dataclasses.dataclass
class Robot:
    parent: np.ndarray
    type: np.ndarray
    X: np.ndarray
    lower: np.ndarray
    upper: np.ndarray
    mass: np.ndarray
    com: np.ndarray
    sphere_link: np.ndarray
    sphere: np.ndarray
    frame_link: np.ndarray
    frame_X: np.ndarray

    @property
    def n_joints(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_link.shape[0])

    @property
    def n_frames(self) -> int:
        return int(self.frame_link.shape[0])


@dataclasses.dataclass
class Constraint:
    """One stacked constraint.

    kind    one of C_*
    frame_a / frame_b   task-frame indices (POSE: a; REL_POSE: a = left, b = right;
                        COM_XY reference: midpoint of a and b)
    P       3x4: POSE, POSE_BOUNDED -> T_w^0 (TSR frame in world); REL_POSE -> T_ref;
            PLANE / LINE -> task frame whose xy-plane / z-axis holds frame a's origin
    Q       3x4: POSE, POSE_BOUNDED -> T_e^w (end-effector offset in the TSR frame)
    target  SPHERE -> (radius, -, -); COM_XY -> (cx, cy, -); DIST -> (L, -, -);
            COM_HULL -> (number of polygon vertices, margin, -)
    B       POSE_BOUNDED: 12 bounds of [t; log R], lower[6] then upper[6];
            COM_HULL: polygon vertices x0, y0, x1, y1, ... counter-clockwise (<= 6)
    q_ref   if given, P (POSE, POSE_BOUNDED, REL_POSE), the origin of P (PLANE,
            LINE), L (DIST), the CoM target (COM_XY) or the support polygon
            (COM_HULL: the xy box around frames a and b grown by the margin)
            is derived from the robot's pose at q_ref when the constraint is
            loaded
    """
    kind: int
    frame_a: int = -1
    frame_b: int = -1
    P: np.ndarray = dataclasses.field(default_factory=lambda: IDENTITY12.copy())
    Q: np.ndarray = dataclasses.field(default_factory=lambda: IDENTITY12.copy())
    target: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    q_ref: np.ndarray | None = None
    B: np.ndarray | None = None

    @property
    def dim(self) -> int:
        return CONSTRAINT_DIM[self.kind]


@dataclasses.dataclass
class Params:
    tol: float = 1e-5
    max_iters: int = 30
    lam: float = 1e-6
    max_step: float = 0.0       # <= 0: divergence exit disabled
    pivot_fp64: float = 1e-7    # FP32 Cholesky pivot below this -> FP64 re-solve
    precision: int = PREC_FP32
    cyclic: bool = False        # one LM step per constraint in order (Sec. IV-C) instead of stacked
    alpha: float = 1.0          # step scale of getDescentStep
    outer: bool = False         # outer form (J^T J + lambda I)^{-1} J^T F instead of the inner one


@dataclasses.dataclass
class Obstacles:
    spheres: np.ndarray   # [n, 4] centre xyz, radius
    aabbs: np.ndarray     # [m, 6] min xyz, max xyz


@dataclasses.dataclass
class Segments:
    """Uneven interpolation segments: point t of segment s is start[:, s] + t * delta[:, s]."""
    start: np.ndarray     # [d, S] float64
    delta: np.ndarray     # [d, S] float64
    length: np.ndarray    # [S] int32, number of points (t = 0 .. length-1)

    @property
    def total(self) -> int:
        return int(self.length.sum())


@dataclasses.dataclass
class Workload:
    name: str
    robot: Robot
    constraints: list
    obstacles: Obstacles
    params: Params
    q: np.ndarray | None = None          # [d, n] float64 start configurations
    segments: Segments | None = None
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def dof(self) -> int:
        return self.robot.n_joints

    @property
    def k(self) -> int:
        return sum(c.dim for c in self.constraints)


def _spheres_along(seg_a, seg_b, count, r_lo, r_hi, rng):
    """`count` spheres evenly spaced on the segment a->b (body coordinates)."""
    a = np.asarray(seg_a, float)
    b = np.asarray(seg_b, float)
    out = np.zeros((count, 4))
    for i in range(count):
        t = (i + 0.5) / count
        out[i, :3] = a + t * (b - a)
        out[i, 3] = rng.uniform(r_lo, r_hi)
    return out


# --------------------------------------------------------------------------
# 7-DoF DH arm (standard DH: Rz(theta) Tz(d) Tx(a) Rx(alpha), a = 0,
# d_i = L_i ~ U(0.1, 0.4), alpha alternating +-pi/2, alpha_7 = 0).
# --------------------------------------------------------------------------
ARM_SPHERES_PER_LINK = (9, 9, 9, 9, 8, 8, 8)   # 60 link spheres


def arm_link_lengths(seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.1, 0.4, size=7)


def dh_arm_robot(L, base=(0.0, 0.0, 0.0), rng=None, n_spheres=ARM_SPHERES_PER_LINK,
                 limit=2.8) -> Robot:
    """Serial 7-joint arm in the tree format.  Joint i's X carries the DH
    offset of joint i-1: Tz(L_{i-1}) Rx(alpha_{i-1})."""
    rng = np.random.default_rng(0) if rng is None else rng
    n = len(L)
    twists = [_RX_PLUS if i % 2 == 0 else _RX_MINUS for i in range(n - 1)] + [np.eye(3)]
    parent = np.arange(-1, n - 1, dtype=np.int32)
    typ = np.zeros(n, np.int32)
    X = np.zeros((n, 12))
    X[0] = _rt(np.eye(3), base)
    for i in range(1, n):
        X[i] = _rt(twists[i - 1], (0.0, 0.0, L[i - 1]))
    spheres, links = [], []
    for i in range(n):
        s = _spheres_along((0, 0, 0), (0, 0, L[i]), n_spheres[i], 0.03, 0.08, rng)
        spheres.append(s)
        links += [i] * n_spheres[i]
    mass = rng.uniform(1.0, 3.0, size=n)
    com = np.zeros((n, 3))
    com[:, 2] = np.asarray(L) / 2
    frame_X = _rt(twists[n - 1], (0.0, 0.0, L[n - 1]))[None, :]
    return Robot(parent=parent, type=typ, X=X, lower=np.full(n, -limit), upper=np.full(n, limit),
                 mass=mass, com=com, sphere_link=np.asarray(links, np.int32),
                 sphere=np.concatenate(spheres), frame_link=np.asarray([n - 1], np.int32),
                 frame_X=frame_X)


def _merge_robots(a: Robot, b: Robot) -> Robot:
    """Two independent trees side by side (b's joints re-indexed after a's)."""
    na = a.n_joints
    pb = b.parent.copy()
    pb[pb >= 0] += na
    sl = b.sphere_link.copy()
    sl[sl >= 0] += na
    fl = b.frame_link.copy()
    fl[fl >= 0] += na
    cat = np.concatenate
    return Robot(parent=cat([a.parent, pb]).astype(np.int32), type=cat([a.type, b.type]).astype(np.int32),
                 X=cat([a.X, b.X]), lower=cat([a.lower, b.lower]), upper=cat([a.upper, b.upper]),
                 mass=cat([a.mass, b.mass]), com=cat([a.com, b.com]),
                 sphere_link=cat([a.sphere_link, sl]).astype(np.int32), sphere=cat([a.sphere, b.sphere]),
                 frame_link=cat([a.frame_link, fl]).astype(np.int32), frame_X=cat([a.frame_X, b.frame_X]))


def _sphere_obstacles(rng, n, lo, hi, r_lo=0.05, r_hi=0.2):
    c = rng.uniform(lo, hi, size=(n, 3))
    r = rng.uniform(r_lo, r_hi, size=(n, 1))
    return np.concatenate([c, r], axis=1)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def sphere_workload(seed: int = 1000, n_pairs: int = 1024, step: float = 0.05,
                    n_obstacles: int = 10) -> Workload:
    """Point q in R^3 on the unit sphere; F(q) = ||q|| - 1.

    The point is modelled as a Cartesian robot (three prismatic joints along
    x, y, z) carrying one sphere of radius 0, so that the collision check of a
    configuration is the check of the point itself.  Each start/goal pair is
    interpolated in ambient space with ceil(|b - a| / step) + 1 evenly spaced
    points (spacing <= step), endpoints included."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n_pairs, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = rng.standard_normal((n_pairs, 3))
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    dist = np.linalg.norm(b - a, axis=1)
    length = (np.ceil(dist / step) + 1).astype(np.int32)
    delta = (b - a) / (length - 1)[:, None]
    X = np.stack([_rt(_R_AXIS["x"], 0), _rt(_R_AXIS["x"].T @ _R_AXIS["y"], 0),
                  _rt(_R_AXIS["y"].T @ _R_AXIS["z"], 0)])
    robot = Robot(parent=np.array([-1, 0, 1], np.int32), type=np.full(3, PRISMATIC, np.int32), X=X,
                  lower=np.full(3, -2.0), upper=np.full(3, 2.0), mass=np.zeros(3), com=np.zeros((3, 3)),
                  sphere_link=np.array([2], np.int32), sphere=np.zeros((1, 4)),
                  frame_link=np.array([2], np.int32), frame_X=IDENTITY12[None, :].copy())
    obst = Obstacles(spheres=_sphere_obstacles(np.random.default_rng(seed + 1), n_obstacles, -1.5, 1.5),
                     aabbs=np.zeros((0, 6)))
    seg = Segments(start=a.T.copy(), delta=delta.T.copy(), length=length)
    wl = Workload(name="sphere", robot=robot, constraints=[Constraint(C_SPHERE, target=np.array([1.0, 0, 0]))],
                  obstacles=obst, params=Params(tol=1e-8, max_iters=50, lam=0.0, precision=PREC_FP64),
                  segments=seg)
    wl.q = segment_points(seg)
    return wl


def segment_points(seg: Segments) -> np.ndarray:
    """Materialise every interpolated point (used by tests and the oracle side)."""
    d = seg.start.shape[0]
    out = np.zeros((d, seg.total))
    off = 0
    for s in range(seg.length.shape[0]):
        t = np.arange(seg.length[s])
        out[:, off:off + seg.length[s]] = seg.start[:, s:s + 1] + t[None, :] * seg.delta[:, s:s + 1]
        off += seg.length[s]
    return out


def arm_workload(seed: int = 1001, n: int = 65536, n_obstacles: int = 64, batch_seed: int | None = None) -> Workload:
    """7-DoF DH arm, end-effector z-axis parallel to world z (2 equations).
    `batch_seed` (default: seed) draws the start configurations only."""
    rng = np.random.default_rng(seed if batch_seed is None else batch_seed)
    L = arm_link_lengths(seed + 2)
    robot = dh_arm_robot(L, rng=np.random.default_rng(seed + 3))
    q = rng.uniform(-2.8, 2.8, size=(7, n))
    # a 1.5 m cube of obstacles in front of the arm's base
    obst = Obstacles(spheres=_sphere_obstacles(np.random.default_rng(seed + 1), n_obstacles,
                                               (0.2, -0.75, 0.0), (1.7, 0.75, 1.5)),
                     aabbs=np.zeros((0, 6)))
    return Workload(name="arm", robot=robot, constraints=[Constraint(C_AXIS_ALIGN, frame_a=0)],
                    obstacles=obst, params=Params(tol=1e-5, max_iters=30, lam=1e-6), q=q)


def arm_task_workload(task: str, seed: int = 1007, n: int = 65536, n_obstacles: int = 64,
                      batch_seed: int | None = None) -> Workload:
    """The arm of `arm_workload` under a task constraint through its
    end-effector pose at a seeded q_ref (so the manifold is not empty):

    * ``tray``: the end effector on the horizontal plane through its q_ref
      position and its z-axis vertical (PLANE + AXIS_ALIGN, 3 equations);
    * ``peg``: the end effector on the vertical line through its q_ref
      position and its z-axis vertical (LINE + AXIS_ALIGN, 4 equations);
    * ``tsr``: a bounded TSR around the q_ref pose, +-5 cm in x and y,
      +-2 cm in z, +-0.1 rad about x and y, +-0.6 rad about z (6 equations).

    For tray and peg, q_ref has q_2 = q_4 = 0 and q_5 = -(q_1 + q_3): with the
    chain's alternating +-pi/2 twists, joints 1, 3 and 5 then turn about one
    common horizontal axis by a total of zero, so the end effector's z-axis
    is vertical at q_ref and q_ref lies on the manifold.  Starts are
    q_ref + N(0, 0.3^2) (configurations near a task, as the extension steps
    of a planner produce)."""
    rng = np.random.default_rng(seed)
    q_ref = rng.uniform(-1.5, 1.5, 7)
    if task in ("tray", "peg"):
        q_ref[2] = q_ref[4] = 0.0
        q_ref[5] = -(q_ref[1] + q_ref[3])
    base = arm_workload(n=1, n_obstacles=n_obstacles)
    brng = np.random.default_rng(seed + 10 if batch_seed is None else batch_seed)
    q = q_ref[:, None] + 0.3 * brng.standard_normal((7, n))
    if task == "tray":
        cons = [Constraint(C_PLANE, frame_a=0, q_ref=q_ref), Constraint(C_AXIS_ALIGN, frame_a=0)]
    elif task == "peg":
        cons = [Constraint(C_LINE, frame_a=0, q_ref=q_ref), Constraint(C_AXIS_ALIGN, frame_a=0)]
    elif task == "tsr":
        hi = np.array([0.05, 0.05, 0.02, 0.1, 0.1, 0.6])
        cons = [Constraint(C_POSE_BOUNDED, frame_a=0, q_ref=q_ref, B=np.concatenate([-hi, hi]))]
    else:
        raise ValueError(task)
    wl = Workload(name=f"arm_{task}", robot=base.robot, constraints=cons, obstacles=base.obstacles,
                  params=Params(tol=1e-5, max_iters=30, lam=1e-6), q=q)
    wl.extra["q_ref"] = q_ref
    return wl


def dual_arm_robot(seed: int = 1002) -> Robot:
    L = arm_link_lengths(1001 + 2)    # two copies of the arm workload's chain
    left = dh_arm_robot(L, base=(0.0, 0.3, 0.0), rng=np.random.default_rng(seed + 3))
    right = dh_arm_robot(L, base=(0.0, -0.3, 0.0), rng=np.random.default_rng(seed + 4))
    return _merge_robots(left, right)


def dual_arm_workload(seed: int = 1002, total: int = 262144, len_lo: int = 2, len_hi: int = 200,
                      step: float = 0.05, n_obstacles: int = 128, n_random: int = 0,
                      batch_seed: int | None = None) -> Workload:
    """Two 7-DoF arms 0.6 m apart; relative EE pose fixed (Eq. 2, 6 equations).

    The reference relative pose is the one the arms have at a seeded
    configuration q_ref, so the manifold is non-empty.  Segments: lengths
    U{len_lo..len_hi} drawn until their sum reaches `total`; raw starts are
    q_ref plus N(0, 0.2^2) noise and raw directions are uniform on S^13.  The
    starts are projected and the directions made tangent before use (see
    `prepare_segments` callers); `extra['raw_start']` / `extra['raw_dir']`
    hold the raw values.  `n_random` > 0 also provides a plain batch of that
    many configurations q_ref + N(0, 0.3^2) in `q`."""
    rng = np.random.default_rng(seed)
    robot = dual_arm_robot(seed)
    q_ref = rng.uniform(-1.2, 1.2, size=14)
    if batch_seed is not None:   # the robot and its reference stay; segments and batch are redrawn
        rng = np.random.default_rng(batch_seed)
    lengths = []
    acc = 0
    while acc < total:
        ln = int(rng.integers(len_lo, len_hi + 1))
        lengths.append(ln)
        acc += ln
    S = len(lengths)
    raw_start = q_ref[:, None] + 0.2 * rng.standard_normal((14, S))
    raw_dir = rng.standard_normal((14, S))
    raw_dir /= np.linalg.norm(raw_dir, axis=0, keepdims=True)
    obst = Obstacles(spheres=_sphere_obstacles(np.random.default_rng(seed + 1), n_obstacles,
                                               (0.2, -1.05, 0.0), (1.7, 1.05, 1.5)),
                     aabbs=np.zeros((0, 6)))
    cons = [Constraint(C_REL_POSE, frame_a=0, frame_b=1, q_ref=q_ref)]
    wl = Workload(name="dual_arm", robot=robot, constraints=cons, obstacles=obst,
                  params=Params(tol=1e-5, max_iters=30, lam=1e-6, pivot_fp64=1e-7))
    wl.extra.update(raw_start=raw_start, raw_dir=raw_dir, lengths=np.asarray(lengths, np.int32),
                    step=step, q_ref=q_ref)
    if n_random:
        wl.q = q_ref[:, None] + 0.3 * rng.standard_normal((14, n_random))
    return wl


def dual_rod_workload(seed: int = 1009, n: int = 65536, n_obstacles: int = 128, sigma: float = 0.3,
                      batch_seed: int | None = None) -> Workload:
    """The dual arm carrying a rigid rod on a table: the distance between the
    two end effectors fixed (a closed linkage, DIST) and each end effector on
    the horizontal plane through its position at a seeded q_ref (PLANE,
    PLANE): 3 equations in 3 stacked constraints.  Starts q_ref + N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    robot = dual_arm_robot()
    q_ref = rng.uniform(-1.2, 1.2, 14)
    brng = rng if batch_seed is None else np.random.default_rng(batch_seed)
    q = q_ref[:, None] + sigma * brng.standard_normal((14, n))
    cons = [Constraint(C_DIST, frame_a=0, frame_b=1, q_ref=q_ref), Constraint(C_PLANE, frame_a=0, q_ref=q_ref),
            Constraint(C_PLANE, frame_a=1, q_ref=q_ref)]
    obst = Obstacles(spheres=_sphere_obstacles(np.random.default_rng(1002 + 1), n_obstacles,
                                               (0.2, -1.05, 0.0), (1.7, 1.05, 1.5)),
                     aabbs=np.zeros((0, 6)))
    wl = Workload(name="dual_rod", robot=robot, constraints=cons, obstacles=obst,
                  params=Params(tol=1e-5, max_iters=30, lam=1e-6, pivot_fp64=1e-7), q=q)
    wl.extra["q_ref"] = q_ref
    return wl


def extend_workload(seed: int = 1010, n_ext: int = 4096, n: int = 8, r: float = 0.3, delta: float = 0.02,
                    sigma: float = 0.05, n_obstacles: int = 32, batch_seed: int | None = None) -> Workload:
    """Batched ParallelConstrainedExtend (Alg. 2) on the dual-arm closed chain
    of `dual_arm_workload` (relative end-effector pose fixed at its q_ref):
    n_ext extensions, each from a start on the manifold towards a random
    target, with n particles and n interpolated points, range r, resolution
    delta and particle offsets eps ~ N(0, sigma^2) along the extension
    direction (the random numbers of Alg. 2, drawn here and passed to both
    sides).  `extra['raw_start']` holds q_ref + N(0, 0.2^2) starts that are
    projected before use; targets are q_ref + U(-1, 1)^14.  MaxDistance 1.0;
    obstacles: spheres 1 .. n_obstacles of the dual-arm scene (its first
    sphere sits where the right arm is at q_ref, which would put most starts
    in collision)."""
    base = dual_arm_workload(total=10)
    q_ref = base.extra["q_ref"]
    rng = np.random.default_rng(seed if batch_seed is None else batch_seed)
    raw_start = q_ref[:, None] + 0.2 * rng.standard_normal((14, n_ext))
    target = q_ref[:, None] + rng.uniform(-1.0, 1.0, size=(14, n_ext))
    eps = sigma * rng.standard_normal((n, n_ext))
    obst = Obstacles(spheres=base.obstacles.spheres[1:1 + n_obstacles].copy(), aabbs=np.zeros((0, 6)))
    wl = Workload(name="extend", robot=base.robot, constraints=base.constraints, obstacles=obst,
                  params=Params(tol=1e-5, max_iters=30, lam=1e-6, pivot_fp64=1e-7, max_step=1.0))
    wl.extra.update(raw_start=raw_start, target=target, eps=eps, r=r, delta=delta, n=n, q_ref=q_ref)
    return wl


def make_segments(start: np.ndarray, direction: np.ndarray, lengths: np.ndarray, step: float) -> Segments:
    """Segments from (projected) starts and (unit) directions."""
    return Segments(start=np.ascontiguousarray(start, dtype=np.float64),
                    delta=np.ascontiguousarray(direction * step, dtype=np.float64),
                    length=np.asarray(lengths, np.int32))


# --------------------------------------------------------------------------
# 36-DoF humanoid-like tree
# --------------------------------------------------------------------------
def _humanoid_plan(rng):
    """Joint list: (name, parent name, offset in parent body frame, axis, type),
    plus body sphere segments and masses.  Body frames are axis-aligned at
    q = 0; the joint frame of joint j is its body frame rotated by R_axis(j)."""
    Lth, Lsh = rng.uniform(0.35, 0.45, 2)
    Ltor = rng.uniform(0.35, 0.45)
    Lup, Lfo = rng.uniform(0.25, 0.30), rng.uniform(0.22, 0.28)
    J = []   # name, parent, offset, axis, type
    J += [("base_x", None, (0, 0, 0), "x", PRISMATIC), ("base_y", "base_x", (0, 0, 0), "y", PRISMATIC),
          ("base_z", "base_y", (0, 0, 0), "z", PRISMATIC), ("base_yaw", "base_z", (0, 0, 0), "z", REVOLUTE),
          ("base_pitch", "base_yaw", (0, 0, 0), "y", REVOLUTE), ("pelvis", "base_pitch", (0, 0, 0), "x", REVOLUTE)]
    for side, sy in (("l", 1.0), ("r", -1.0)):
        J += [(f"{side}_hip_yaw", "pelvis", (0, 0.09 * sy, -0.05), "z", REVOLUTE),
              (f"{side}_hip_roll", f"{side}_hip_yaw", (0, 0, -0.04), "x", REVOLUTE),
              (f"{side}_hip_pitch", f"{side}_hip_roll", (0, 0, -0.04), "y", REVOLUTE),
              (f"{side}_knee", f"{side}_hip_pitch", (0, 0, -Lth), "y", REVOLUTE),
              (f"{side}_ankle_pitch", f"{side}_knee", (0, 0, -Lsh), "y", REVOLUTE),
              (f"{side}_ankle_roll", f"{side}_ankle_pitch", (0, 0, 0), "x", REVOLUTE)]
    J += [("waist_yaw", "pelvis", (0, 0, 0.12), "z", REVOLUTE), ("torso", "waist_yaw", (0, 0, 0.05), "y", REVOLUTE),
          ("neck_yaw", "torso", (0, 0, Ltor + 0.05), "z", REVOLUTE), ("head", "neck_yaw", (0, 0, 0.05), "y", REVOLUTE)]
    for side, sy in (("l", 1.0), ("r", -1.0)):
        J += [(f"{side}_sh_pitch", "torso", (0, 0.2 * sy, Ltor), "y", REVOLUTE),
              (f"{side}_sh_roll", f"{side}_sh_pitch", (0, 0.05 * sy, 0), "x", REVOLUTE),
              (f"{side}_sh_yaw", f"{side}_sh_roll", (0, 0, -0.05), "z", REVOLUTE),
              (f"{side}_elbow", f"{side}_sh_yaw", (0, 0, -Lup), "y", REVOLUTE),
              (f"{side}_wr_yaw", f"{side}_elbow", (0, 0, -Lfo), "z", REVOLUTE),
              (f"{side}_wr_pitch", f"{side}_wr_yaw", (0, 0, 0), "y", REVOLUTE),
              (f"{side}_wr_roll", f"{side}_wr_pitch", (0, 0, 0), "x", REVOLUTE)]
    # body segments: name -> (a, b, n_spheres, r_lo, r_hi, mass)
    B = {"pelvis": ((0, -0.14, 0), (0, 0.14, 0), 14, 0.06, 0.09, 10.0),
         "torso": ((0, 0, 0), (0, 0, Ltor), 18, 0.08, 0.12, 15.0),
         "head": ((0, 0, 0), (0, 0, 0.2), 6, 0.06, 0.09, 4.0),
         "waist_yaw": ((0, 0, 0), (0, 0, 0.05), 0, 0, 0, 1.0),
         "neck_yaw": ((0, 0, 0), (0, 0, 0.05), 0, 0, 0, 0.5)}
    for side in ("l", "r"):
        B.update({f"{side}_hip_yaw": ((0, 0, 0), (0, 0, -0.04), 0, 0, 0, 1.0),
                  f"{side}_hip_roll": ((0, 0, 0), (0, 0, -0.04), 3, 0.05, 0.07, 1.0),
                  f"{side}_hip_pitch": ((0, 0, 0), (0, 0, -Lth), 10, 0.05, 0.08, 6.0),
                  f"{side}_knee": ((0, 0, 0), (0, 0, -Lsh), 10, 0.04, 0.07, 3.0),
                  f"{side}_ankle_pitch": ((0, 0, 0), (0, 0, -0.02), 0, 0, 0, 0.3),
                  f"{side}_ankle_roll": ((-0.05, 0, -0.06), (0.12, 0, -0.06), 6, 0.03, 0.05, 1.0),
                  f"{side}_sh_pitch": ((0, 0, 0), (0, 0.05, 0), 0, 0, 0, 0.5),
                  f"{side}_sh_roll": ((0, 0, 0), (0, 0, -0.05), 3, 0.05, 0.07, 0.5),
                  f"{side}_sh_yaw": ((0, 0, 0), (0, 0, -Lup), 8, 0.04, 0.06, 2.0),
                  f"{side}_elbow": ((0, 0, 0), (0, 0, -Lfo), 8, 0.035, 0.05, 1.5),
                  f"{side}_wr_yaw": ((0, 0, 0), (0, 0, 0), 0, 0, 0, 0.2),
                  f"{side}_wr_pitch": ((0, 0, 0), (0, 0, 0), 0, 0, 0, 0.2),
                  f"{side}_wr_roll": ((0, 0, 0), (0, 0, -0.12), 8, 0.03, 0.05, 0.5)})
    return J, B


HUMANOID_FRAMES = ("l_foot", "r_foot", "l_hand", "r_hand")


def humanoid_robot(seed: int = 1005) -> tuple[Robot, list]:
    rng = np.random.default_rng(seed)
    plan, bodies = _humanoid_plan(rng)
    names = [p[0] for p in plan]
    idx = {nm: i for i, nm in enumerate(names)}
    n = len(plan)
    parent = np.full(n, -1, np.int32)
    typ = np.zeros(n, np.int32)
    X = np.zeros((n, 12))
    axis = {}
    for j, (nm, par, off, ax, tp) in enumerate(plan):
        axis[nm] = ax
        Rp = _R_AXIS[axis[par]] if par is not None else np.eye(3)
        parent[j] = idx[par] if par is not None else -1
        typ[j] = tp
        X[j] = _rt(Rp.T @ _R_AXIS[ax], Rp.T @ np.asarray(off, float))
    spheres, slinks = [], []
    mass = np.zeros(n)
    com = np.zeros((n, 3))
    for nm, (a, b, ns, rlo, rhi, m) in bodies.items():
        j = idx[nm]
        Rj = _R_AXIS[axis[nm]]
        if ns:
            s = _spheres_along(a, b, ns, rlo, rhi, rng)
            s[:, :3] = s[:, :3] @ Rj        # body -> joint-frame coordinates (R^T c)
            spheres.append(s)
            slinks += [j] * ns
        mass[j] = m * rng.uniform(0.8, 1.2)
        com[j] = Rj.T @ (0.5 * (np.asarray(a, float) + np.asarray(b, float)))
    frames = [("l_ankle_roll", (0.03, 0, -0.06)), ("r_ankle_roll", (0.03, 0, -0.06)),
              ("l_wr_roll", (0, 0, -0.1)), ("r_wr_roll", (0, 0, -0.1))]
    frame_link = np.asarray([idx[f[0]] for f in frames], np.int32)
    frame_X = np.stack([_rt(_R_AXIS[axis[f[0]]].T, _R_AXIS[axis[f[0]]].T @ np.asarray(f[1], float))
                        for f in frames])
    lower = np.where(typ == PRISMATIC, -5.0, -2.8)
    robot = Robot(parent=parent, type=typ, X=X, lower=lower, upper=-lower, mass=mass, com=com,
                  sphere_link=np.asarray(slinks, np.int32), sphere=np.concatenate(spheres),
                  frame_link=frame_link, frame_X=frame_X)
    return robot, names


def humanoid_nominal(names) -> np.ndarray:
    q = np.zeros(len(names))
    val = {"base_z": 1.0, "l_hip_pitch": -0.3, "r_hip_pitch": -0.3, "l_knee": 0.6, "r_knee": 0.6,
           "l_ankle_pitch": -0.3, "r_ankle_pitch": -0.3, "l_sh_pitch": -1.2, "r_sh_pitch": -1.2,
           "l_sh_roll": 0.25, "r_sh_roll": -0.25, "l_elbow": -0.6, "r_elbow": -0.6}
    for i, nm in enumerate(names):
        q[i] = val.get(nm, 0.0)
    return q


def humanoid_workload(seed: int = 1003, n: int = 1048576, n_obstacles: int = 200,
                      batch_seed: int | None = None, hull: bool = False) -> Workload:
    """36-DoF tree; feet fixed in 6-D pose (2 x Eq. 1), hands in a fixed relative
    pose (Eq. 2), CoM xy at the support-polygon centre: 20 equations.  All
    references are taken at the nominal stance q_nom; the support-polygon
    centre is the midpoint of the two foot frames there.  With `hull`, the
    CoM constraint is the distance to the support polygon instead (zero
    inside), the polygon being the xy box around the feet at q_nom grown by
    0.08 m."""
    robot, names = humanoid_robot(seed + 2)
    q_nom = humanoid_nominal(names)
    rng = np.random.default_rng(seed if batch_seed is None else batch_seed)
    sigma = np.where(robot.type == PRISMATIC, 0.05, 0.3)
    q = q_nom[:, None] + sigma[:, None] * rng.standard_normal((robot.n_joints, n))
    cons = [Constraint(C_POSE, frame_a=0, q_ref=q_nom), Constraint(C_POSE, frame_a=1, q_ref=q_nom),
            Constraint(C_REL_POSE, frame_a=2, frame_b=3, q_ref=q_nom),
            Constraint(C_COM_XY, frame_a=0, frame_b=1, q_ref=q_nom)]
    if hull:
        cons[3] = Constraint(C_COM_HULL, frame_a=0, frame_b=1, q_ref=q_nom, target=np.array([4.0, 0.08, 0.0]))
    orng = np.random.default_rng(seed + 1)
    sph = _sphere_obstacles(orng, n_obstacles, (0.5, -2.0, 0.0), (2.5, 2.0, 2.2), 0.05, 0.15)
    # a shelf in front of the robot: two side panels, three boards, a back panel
    x0, x1, y0, y1 = 0.75, 1.1, -0.6, 0.6
    aabbs = np.array([[x0, y0 - 0.03, 0.0, x1, y0, 1.8], [x0, y1, 0.0, x1, y1 + 0.03, 1.8],
                      [x0, y0, 0.4, x1, y1, 0.43], [x0, y0, 0.9, x1, y1, 0.93],
                      [x0, y0, 1.4, x1, y1, 1.43], [x1, y0, 0.0, x1 + 0.03, y1, 1.8]])
    wl = Workload(name="humanoid", robot=robot, constraints=cons,
                  obstacles=Obstacles(spheres=sph, aabbs=aabbs),
                  params=Params(tol=1e-5, max_iters=40, lam=1e-6), q=q)
    wl.extra.update(q_nom=q_nom, names=names)
    return wl


def adjoint_workload(seed: int = 1004, n: int = 65536) -> Workload:
    """Dual-arm manifold; `q` holds raw configurations (projected before use)
    and `extra['g']` upstream gradients g ~ N(0, 1)."""
    wl = dual_arm_workload(seed=1002, total=0, n_random=0)
    rng = np.random.default_rng(seed)
    q_ref = wl.extra["q_ref"]
    wl.q = q_ref[:, None] + 0.3 * rng.standard_normal((14, n))
    wl.extra["g"] = rng.standard_normal((14, n))
    wl.name = "adjoint"
    return wl


def path_workload(seed: int = 1006, n_paths: int = 4096, n_way: int = 64) -> dict:
    """Raw material for path shortening on the dual-arm manifold: per path two
    raw endpoint configurations and N(0, 0.05^2) waypoint noise.  Endpoints
    are projected, waypoints linearly interpolated, noised and projected by
    the caller."""
    wl = dual_arm_workload(seed=1002, total=0)
    rng = np.random.default_rng(seed)
    q_ref = wl.extra["q_ref"]
    qa = q_ref[:, None] + 0.3 * rng.standard_normal((14, n_paths))
    qb = q_ref[:, None] + 0.3 * rng.standard_normal((14, n_paths))
    noise = 0.05 * rng.standard_normal((14, n_paths, n_way))
    noise[:, :, 0] = 0.0
    noise[:, :, -1] = 0.0
    return {"workload": wl, "qa": qa, "qb": qb, "noise": noise, "n_paths": n_paths, "n_way": n_way}


def random_tree_robot(seed: int, n_joints: int = 9, n_frames: int = 3, prismatic_frac: float = 0.2) -> Robot:
    """A random kinematic tree with generic (non-axis-aligned) fixed
    transforms, for testing FK / Jacobians / projection on arbitrary trees."""
    rng = np.random.default_rng(seed)
    parent = np.full(n_joints, -1, np.int32)
    for j in range(1, n_joints):
        parent[j] = rng.integers(-1, j) if rng.uniform() < 0.15 else rng.integers(max(0, j - 3), j)
    typ = (rng.uniform(size=n_joints) < prismatic_frac).astype(np.int32)
    X = np.zeros((n_joints, 12))
    for j in range(n_joints):
        X[j] = _rt(random_rotation(rng), rng.uniform(-0.3, 0.3, 3))
    ns = 2 * n_joints
    frame_link = rng.integers(0, n_joints, n_frames).astype(np.int32)
    frame_X = np.stack([_rt(random_rotation(rng), rng.uniform(-0.2, 0.2, 3)) for _ in range(n_frames)])
    return Robot(parent=parent, type=typ, X=X, lower=np.full(n_joints, -3.0), upper=np.full(n_joints, 3.0),
                 mass=rng.uniform(0.5, 2.0, n_joints), com=rng.uniform(-0.1, 0.1, (n_joints, 3)),
                 sphere_link=rng.integers(-1, n_joints, ns).astype(np.int32),
                 sphere=np.concatenate([rng.uniform(-0.2, 0.2, (ns, 3)), rng.uniform(0.02, 0.1, (ns, 1))], 1),
                 frame_link=frame_link, frame_X=frame_X)


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    w, x, y, z = rng.standard_normal(4) / 1.0
    nrm = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


WORKLOADS = {"sphere": sphere_workload, "arm": arm_workload, "dual_arm": dual_arm_workload,
             "humanoid": humanoid_workload}
