"""Algorithmic floating-point operation counts of the projection path.

The count follows the structure-aware algorithm the kernels implement (the
GPU counterpart of the paper's traced straight-line code, Sec. IV-A): fixed
joint offsets whose rotation is a signed permutation cost nothing, structurally
zero translation components are skipped, Jacobian entries that are zero by the
tree structure (a joint that is not above a frame) are neither formed nor
multiplied.  An add or a multiply counts 1, a fused multiply-add 2.  Square
roots, reciprocal square roots and atan2 are special-function work and are not
counted.  sin/cos are the FMA polynomials of the kernels (FP32: 27 flops;
FP64 table-driven: 24 flops).

Per configuration:
    fp32 = iters * iteration + (evaluation only, for the final residual test)
    fp64 = acceptance (FK + residual in FP64), once
with `iters` the number of Newton steps the configuration took.  In the
cyclic form (Sec. IV-C) an iteration is one sweep: the stopping test on the
stacked F plus one full step (FK, residual, Jacobian, solve) per constraint.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

SINCOS32 = 27
SINCOS64 = 24
ROT_UPDATE = 18          # R_pre * Rz(q): two columns, 3 x (mul + fma)
TRANS_PER_AXIS = 6       # one nonzero translation component: 3 fma
MUL33 = 45               # dense 3x3 product: 9 x (mul + 2 fma)
MULV = 15                # 3x3 times vector
LOG_MAP = 22
BETA = 10


def _rot_is_perm(R):
    R = np.asarray(R)
    return all(np.count_nonzero(R[:, k]) == 1 and abs(R[np.flatnonzero(R[:, k])[0], k]) == 1 for k in range(3))


def _ancestors(parent, link):
    out = set()
    while link >= 0:
        out.add(int(link))
        link = parent[link]
    return out


class FlopModel:
    def __init__(self, robot, constraints, cyclic: bool = False):
        self.rb = robot
        self.cons = list(constraints)
        self.d = robot.n_joints
        self.k = sum(c.dim for c in self.cons)
        kinds = [c.kind for c in self.cons]
        self.needs_fk = any(k != W.C_SPHERE for k in kinds)
        self.needs_pos = any(k in (W.C_POSE, W.C_REL_POSE, W.C_COM_XY) for k in kinds)
        self._fk32 = self._fk(SINCOS32) if self.needs_fk else 0
        self._fk64 = self._fk(SINCOS64) if self.needs_fk else 0
        self._res = self._residual(with_j=False)
        self._res_j = self._residual(with_j=True)
        self._jac, nz = self._jacobian()
        K = self.k
        gram = 0
        for a in range(K):
            for b in range(a + 1):
                gram += 2 * int(np.sum(nz[a] & nz[b]))
        chol = 0
        for j in range(K):
            chol += 2 * j + 1                    # pivot
            chol += (K - j - 1) * (2 * j + 1)    # column below the pivot
        chol += 2 * sum(2 * i + 1 for i in range(K))   # forward + back substitution
        jty = 2 * int(nz.sum())
        # the refinement step of the FP32 kernels is not part of the method and is not counted
        self.iteration = self._fk32 + self._res_j + 2 * K + self._jac + gram + chol + jty + 3 * self.d
        self.evaluation = self._fk32 + self._res + 2 * K
        self.acceptance = self._fk64 + self._res + 2 * K
        if cyclic and len(self.cons) > 1:
            self.iteration = self.evaluation + 3 * self.d + sum(
                FlopModel(robot, [c]).iteration for c in self.cons)
        # sin / cos evaluations per forward kinematics (special functions: the
        # algorithmic counts below leave their polynomial flops out)
        self.n_sincos = int(sum(1 for j in range(self.d) if robot.type[j] == W.REVOLUTE)) if self.needs_fk else 0
        n_fk_step = 1 + (len(self.cons) if cyclic and len(self.cons) > 1 else 0)
        self.iteration_alg = self.iteration - SINCOS32 * self.n_sincos * n_fk_step
        self.evaluation_alg = self.evaluation - SINCOS32 * self.n_sincos
        self.acceptance_alg = self.acceptance - SINCOS64 * self.n_sincos

    def _fk(self, sincos):
        rb = self.rb
        X = np.asarray(rb.X).reshape(-1, 3, 4)
        total = 0
        for j in range(self.d):
            root = rb.parent[j] < 0
            perm = _rot_is_perm(X[j, :, :3])
            if not root and not perm:
                total += MUL33
            if self.needs_pos and not root:
                total += TRANS_PER_AXIS * int(np.count_nonzero(X[j, :, 3]))
            if rb.type[j] == W.REVOLUTE:
                total += sincos + (0 if (root and perm) else ROT_UPDATE)
            elif self.needs_pos:
                total += TRANS_PER_AXIS
        F = np.asarray(rb.frame_X).reshape(-1, 3, 4)
        for f in range(rb.n_frames):
            if not _rot_is_perm(F[f, :, :3]):
                total += MUL33
            if self.needs_pos:
                total += TRANS_PER_AXIS * int(np.count_nonzero(F[f, :, 3]))
        return total

    def _residual(self, with_j):
        total = 0
        for c in self.cons:
            if c.kind == W.C_SPHERE:
                total += 2 * self.d + 2
            elif c.kind in (W.C_POSE, W.C_POSE_BOUNDED):
                total += 2 * MUL33 + 18 + MULV + 3 + LOG_MAP + (BETA if with_j else 0)
                if c.kind == W.C_POSE_BOUNDED:
                    total += 6          # one subtraction per component outside its bounds
            elif c.kind == W.C_PLANE:
                total += 6
            elif c.kind == W.C_LINE:
                total += 12
            elif c.kind == W.C_DIST:
                total += 3 + 5 + 1 + (3 if with_j else 0)
            elif c.kind == W.C_REL_POSE:
                total += 2 * MUL33 + 3 + MULV + 3 + LOG_MAP + (BETA if with_j else 0)
            elif c.kind == W.C_COM_XY:
                total += 24 * self.d + 4
                if with_j:
                    total += 3 * sum(1 for j in range(self.d) if self.rb.parent[j] >= 0)
        return total

    def _jacobian(self):
        rb = self.rb
        K, D = self.k, self.d
        nz = np.zeros((K, D), bool)
        total = 0
        r0 = 0
        for c in self.cons:
            kd = c.dim
            if c.kind == W.C_SPHERE:
                nz[r0, :] = True
                total += D
            elif c.kind == W.C_COM_XY:
                nz[r0:r0 + 2, :] = True
                total += sum(17 if rb.type[j] == W.REVOLUTE else 3 for j in range(D))
            elif c.kind in (W.C_PLANE, W.C_LINE, W.C_DIST):
                la = _ancestors(rb.parent, rb.frame_link[c.frame_a])
                lb = _ancestors(rb.parent, rb.frame_link[c.frame_b]) if c.kind == W.C_DIST else set()
                for j in range(D):
                    s = (j in lb) - (j in la) if c.kind == W.C_DIST else (1 if j in la else 0)
                    if s == 0:
                        continue
                    rev = rb.type[j] == W.REVOLUTE
                    nz[r0:r0 + kd, j] = True
                    total += (12 if rev else 0) + 5 * kd   # point velocity + one dot product per row
            else:
                la = _ancestors(rb.parent, rb.frame_link[c.frame_a])
                lb = _ancestors(rb.parent, rb.frame_link[c.frame_b]) if c.kind == W.C_REL_POSE else set()
                for j in range(D):
                    s = (1 if j in la else 0) if c.kind != W.C_REL_POSE else (j in lb) - (j in la)
                    if s == 0:
                        continue
                    rev = rb.type[j] == W.REVOLUTE
                    if c.kind == W.C_AXIS_ALIGN:
                        if rev:
                            nz[r0:r0 + 2, j] = True
                            total += 6
                    else:
                        nz[r0:r0 + 3, j] = True
                        total += 12 + MULV if rev else MULV
                        if rev:
                            nz[r0 + 3:r0 + 6, j] = True
                            total += MULV + 30
            r0 += kd
        return total, nz

    def projection(self, iters, sincos=True):
        """(FP32 flops, FP64 flops) of projecting configurations that took
        `iters` steps; without the sin/cos polynomials if not `sincos`."""
        it = np.asarray(iters, dtype=np.float64)
        n = it.size
        if sincos:
            return float(it.sum()) * self.iteration + n * self.evaluation, n * self.acceptance
        return float(it.sum()) * self.iteration_alg + n * self.evaluation_alg, n * self.acceptance_alg

    def fk_positions(self):
        """FP32 flops of the forward kinematics with translations (collision check)."""
        saved = self.needs_pos
        self.needs_pos = True
        v = self._fk(SINCOS32)
        self.needs_pos = saved
        return v


def collision_pair_flops() -> int:
    """Sphere-sphere test: 3 sub, |d|^2 (mul + 2 fma), r_s + r_o, its square."""
    return 3 + 5 + 1 + 1
