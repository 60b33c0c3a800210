"""ctypes wrapper of the FP64 CPU oracle (mcp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by
the benchmark's CPU-baseline leg.  The product path never imports it.  It
does not import the CUDA package either: robots, constraints and obstacles are
duck-typed objects with the attributes of the seeded input generators.

Numbering (kinds, flags, layouts) follows the paper's problem statement as
restated in mcp_oracle.c; it is written out here independently of the CUDA
library's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CONVERGED, CAP, DIVERGED, NONFINITE, OUT_OF_LIMITS = 1, 2, 4, 8, 64
SPHERE, AXIS_ALIGN, POSE, REL_POSE, COM_XY = 0, 1, 2, 3, 4
PLANE, LINE, DIST, POSE_BOUNDED, COM_HULL = 5, 6, 7, 8, 9
DIM = {SPHERE: 1, AXIS_ALIGN: 2, POSE: 6, REL_POSE: 6, COM_XY: 2, PLANE: 1, LINE: 2, DIST: 1, POSE_BOUNDED: 6,
       COM_HULL: 2}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class _Robot(ctypes.Structure):
    _fields_ = [("nj", ctypes.c_int32), ("parent", _ip), ("type", _ip), ("X", _dp), ("lower", _dp),
                ("upper", _dp), ("mass", _dp), ("com", _dp), ("ns", ctypes.c_int32), ("sphere_link", _ip),
                ("sphere", _dp), ("nf", ctypes.c_int32), ("frame_link", _ip), ("frame_X", _dp)]


class _Constraint(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("fa", ctypes.c_int32), ("fb", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("P", ctypes.c_double * 12), ("Q", ctypes.c_double * 12), ("target", ctypes.c_double * 4),
                ("B", ctypes.c_double * 12)]


class _ExtParams(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("delta", ctypes.c_double), ("n", ctypes.c_int32),
                ("max_depth", ctypes.c_int32)]


# ParallelConstrainedExtend status codes (mcp_oracle.c)
EXT_OK, EXT_DEGENERATE, EXT_NO_PROJECTION, EXT_PROJ_COLLISION, EXT_TOO_FAR, EXT_INTERP_FAIL, EXT_GAP, \
    EXT_INTERP_COLLISION, EXT_RESOLUTION = range(9)


class _Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("cyclic", ctypes.c_int32),
                ("lam", ctypes.c_double), ("alpha", ctypes.c_double), ("max_step", ctypes.c_double),
                ("outer", ctypes.c_int32), ("pad", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm",
                                   "-pthread"])
            os.replace(tmp, _LIB)
    return _LIB


_COUNT_SRC = os.path.join(_HERE, "count_ops.cpp")
_COUNT_LIB = os.path.join(_OUT_DIR, "liboracle_count.so")
_count_lib = None


def build_count(force: bool = False) -> str:
    """Compile the operation-counting build of the oracle (g++, the oracle's
    C source included with `double` replaced by a counting wrapper)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_COUNT_SRC))
        if force or not os.path.exists(_COUNT_LIB) or os.path.getmtime(_COUNT_LIB) < newest:
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _COUNT_LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-o", tmp, _COUNT_SRC, "-lm",
                                   "-pthread"])
            os.replace(tmp, _COUNT_LIB)
    return _COUNT_LIB


def _load_count():
    global _count_lib
    if _count_lib is None:
        lib = ctypes.CDLL(build_count())
        P = ctypes.POINTER
        lib.oc_count.argtypes = [P(_Robot), P(_Constraint), ctypes.c_int, P(_Params), ctypes.c_int64, ctypes.c_int64,
                                 _dp, _dp, ctypes.POINTER(ctypes.c_uint64)]
        _count_lib = lib
    return _count_lib


# operation classes of the counting build: flops (add, mul, div) and special functions
OP_NAMES = ("add", "mul", "div", "sqrt", "sincos", "atan2")


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.or_fk.argtypes = [P(_Robot), _dp, _dp, _dp]
        lib.or_joint_axes.argtypes = [P(_Robot), _dp, _dp, _dp]
        lib.or_com.argtypes = [P(_Robot), _dp, _dp]
        lib.or_com.restype = ctypes.c_double
        lib.or_residual_jacobian.argtypes = [P(_Robot), P(_Constraint), ctypes.c_int, _dp, _dp, _dp]
        lib.or_residual_jacobian.restype = ctypes.c_int
        lib.or_so3_log.argtypes = [_dp, _dp]
        lib.or_so3_left_jac_inv.argtypes = [_dp, _dp]
        lib.or_resolve_reference.argtypes = [P(_Robot), P(_Constraint), _dp]
        lib.or_project.argtypes = [P(_Robot), P(_Constraint), ctypes.c_int, P(_Params), ctypes.c_int64,
                                   ctypes.c_int64, _dp, _dp, _u8p, _ip, _dp, ctypes.c_int]
        lib.or_check.argtypes = [P(_Robot), ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int64, ctypes.c_int64,
                                 _dp, _u8p, _dp, ctypes.c_int]
        lib.or_vjp.argtypes = [P(_Robot), P(_Constraint), ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _dp, _dp,
                               _dp, _u8p, ctypes.c_int]
        lib.or_extend.argtypes = [P(_Robot), P(_Constraint), ctypes.c_int, P(_Params), P(_ExtParams), ctypes.c_int,
                                  _dp, ctypes.c_int, _dp, ctypes.c_int64, ctypes.c_int64, _dp, _dp, _dp,
                                  ctypes.c_int64, _dp, _u8p, _ip, _ip, ctypes.c_int]
        lib.or_path_length_grad.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp]
        lib.or_shorten.argtypes = [P(_Robot), P(_Constraint), ctypes.c_int, P(_Params), ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_int64, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _u8p,
                                   _dp, _dp, ctypes.c_int]
        lib.or_shorten.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


class Oracle:
    """FP64 reference for one robot, constraint stack and obstacle set."""

    def __init__(self, robot, constraints=(), obstacles=None):
        lib = _load()
        self._keep = []
        keep = self._keep.append

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep(a)
            return a

        nj = int(np.asarray(robot.parent).shape[0])
        self.d = nj
        r = _Robot()
        r.nj = nj
        r.parent = _ptr(arr(robot.parent, np.int32), _ip)
        r.type = _ptr(arr(robot.type, np.int32), _ip)
        r.X = _ptr(arr(np.asarray(robot.X).reshape(nj, 12), np.float64))
        r.lower = _ptr(arr(robot.lower, np.float64))
        r.upper = _ptr(arr(robot.upper, np.float64))
        r.mass = _ptr(arr(robot.mass, np.float64))
        r.com = _ptr(arr(np.asarray(robot.com).reshape(nj, 3), np.float64))
        ns = int(np.asarray(robot.sphere_link).shape[0])
        r.ns = ns
        r.sphere_link = _ptr(arr(robot.sphere_link, np.int32), _ip)
        r.sphere = _ptr(arr(np.asarray(robot.sphere).reshape(max(ns, 1) if ns else 0, 4) if ns else
                            np.zeros((1, 4)), np.float64))
        nf = int(np.asarray(robot.frame_link).shape[0])
        r.nf = nf
        r.frame_link = _ptr(arr(robot.frame_link if nf else np.zeros(1), np.int32), _ip)
        r.frame_X = _ptr(arr(np.asarray(robot.frame_X).reshape(nf, 12) if nf else np.zeros((1, 12)), np.float64))
        self._robot = r
        self.nc = len(constraints)
        self._cons = (_Constraint * max(1, self.nc))()
        self.k = 0
        for i, c in enumerate(constraints):
            cc = self._cons[i]
            cc.kind, cc.fa, cc.fb = int(c.kind), int(c.frame_a), int(c.frame_b)
            for t in range(12):
                cc.P[t] = float(c.P[t])
                cc.Q[t] = float(c.Q[t])
            for t in range(3):
                cc.target[t] = float(c.target[t])
            B = getattr(c, "B", None)
            for t in range(12):   # unbounded unless given
                cc.B[t] = float(B[t]) if B is not None else (-np.inf if t < 6 else np.inf)
            cc.target[3] = 0.0
            if getattr(c, "q_ref", None) is not None:
                lib.or_resolve_reference(ctypes.byref(r), ctypes.byref(cc), _ptr(_f64(c.q_ref)))
            self.k += DIM[int(c.kind)]
        if obstacles is not None:
            self._obs = _f64(np.asarray(obstacles.spheres).reshape(-1, 4))
            self._box = _f64(np.asarray(obstacles.aabbs).reshape(-1, 6))
        else:
            self._obs = np.zeros((0, 4))
            self._box = np.zeros((0, 6))

    # ---- references resolved at construction ----
    def constraint_values(self, i):
        c = self._cons[i]
        return np.array(c.P[:]), np.array(c.Q[:]), np.array(c.target[:3])

    def bounds(self, i):
        c = self._cons[i]
        return np.array(c.B[:])

    # ---- single-configuration helpers ----
    def fk(self, q):
        q = _f64(q)
        Tj = np.zeros((self.d, 12))
        nf = self._robot.nf
        Tf = np.zeros((max(nf, 1), 12))
        _load().or_fk(ctypes.byref(self._robot), _ptr(q), _ptr(Tj), _ptr(Tf))
        return Tj, Tf[:nf]

    def joint_axes(self, q):
        q = _f64(q)
        z = np.zeros((self.d, 3))
        o = np.zeros((self.d, 3))
        _load().or_joint_axes(ctypes.byref(self._robot), _ptr(q), _ptr(z), _ptr(o))
        return z, o

    def com(self, q):
        x = np.zeros(3)
        M = _load().or_com(ctypes.byref(self._robot), _ptr(_f64(q)), _ptr(x))
        return x, M

    def residual(self, q):
        F = np.zeros(max(self.k, 1))
        _load().or_residual_jacobian(ctypes.byref(self._robot), self._cons, self.nc, _ptr(_f64(q)), _ptr(F), None)
        return F[:self.k]

    def residual_jacobian(self, q):
        F = np.zeros(max(self.k, 1))
        J = np.zeros((max(self.k, 1), self.d))
        _load().or_residual_jacobian(ctypes.byref(self._robot), self._cons, self.nc, _ptr(_f64(q)), _ptr(F),
                                     _ptr(J))
        return F[:self.k], J[:self.k]

    # ---- batched (SoA [d, n]) ----
    def project(self, q, tol, max_iters, lam, max_step=0.0, alpha=1.0, cyclic=False, outer=False, threads=None):
        q = _f64(q)
        d, n = q.shape
        out = np.empty_like(q)
        flags = np.zeros(n, np.uint8)
        iters = np.zeros(n, np.int32)
        resid = np.zeros(n)
        p = _Params(tol=tol, max_iters=max_iters, cyclic=int(bool(cyclic)), lam=lam, alpha=alpha,
                    max_step=max_step, outer=int(bool(outer)))
        _load().or_project(ctypes.byref(self._robot), self._cons, self.nc, ctypes.byref(p), n, n, _ptr(q),
                           _ptr(out), _ptr(flags, _u8p), _ptr(iters, _ip), _ptr(resid),
                           threads or default_threads())
        return out, flags, iters, resid

    def project_params(self, q, params, **kw):
        kw.setdefault("alpha", getattr(params, "alpha", 1.0))
        kw.setdefault("outer", getattr(params, "outer", False))
        kw.setdefault("cyclic", getattr(params, "cyclic", False))
        return self.project(q, params.tol, params.max_iters, params.lam, max_step=params.max_step, **kw)

    def extend(self, q_s, q_t, eps, params, r, delta, max_depth=6, threads=None):
        """ParallelConstrainedExtend (Alg. 2) of each column of q_s towards the
        same column of q_t; eps [n, n_ext] are the particle offsets along the
        extension direction.  Returns (q_proj, status, n_points, winner)."""
        q_s, q_t, eps = _f64(q_s), _f64(q_t), _f64(eps)
        d, m = q_s.shape
        n = eps.shape[0]
        q_proj = np.empty_like(q_s)
        status = np.zeros(m, np.uint8)
        n_points = np.zeros(m, np.int32)
        winner = np.zeros(m, np.int32)
        p = _Params(tol=params.tol, max_iters=params.max_iters, cyclic=int(bool(getattr(params, "cyclic", False))),
                    lam=params.lam, alpha=getattr(params, "alpha", 1.0), max_step=params.max_step,
                    outer=int(bool(getattr(params, "outer", False))))
        ep = _ExtParams(r=r, delta=delta, n=n, max_depth=max_depth)
        _load().or_extend(ctypes.byref(self._robot), self._cons, self.nc, ctypes.byref(p), ctypes.byref(ep),
                          self._obs.shape[0], _ptr(self._obs), self._box.shape[0], _ptr(self._box), m, m,
                          _ptr(q_s), _ptr(q_t), _ptr(eps), m, _ptr(q_proj), _ptr(status, _u8p), _ptr(n_points, _ip),
                          _ptr(winner, _ip), threads or default_threads())
        return q_proj, status, n_points, winner

    def check(self, q, threads=None):
        q = _f64(q)
        d, n = q.shape
        hit = np.zeros(n, np.uint8)
        margin = np.zeros(n)
        _load().or_check(ctypes.byref(self._robot), self._obs.shape[0], _ptr(self._obs), self._box.shape[0],
                         _ptr(self._box), n, n, _ptr(q), _ptr(hit, _u8p), _ptr(margin), threads or default_threads())
        return hit, margin

    def shorten(self, Q, n_paths, n_way, params, steps, eta=0.1, max_step=0.05, threads=None):
        """Gradient path shortening on the manifold (FP64): `steps` descent
        steps (project every waypoint, length gradient at the projections, its
        VJP through the projection, clipped step of the interior waypoints),
        then a final projection.  Q: [d, n_paths * n_way] waypoints.  Returns
        (Q_final, flags, resid, lengths [n_paths, 2] before / after)."""
        Q = _f64(Q)
        d, ld = Q.shape
        out = np.empty_like(Q)
        flags = np.zeros(ld, np.uint8)
        resid = np.zeros(ld)
        lengths = np.zeros((n_paths, 2))
        p = _Params(tol=params.tol, max_iters=params.max_iters, cyclic=int(bool(getattr(params, "cyclic", False))),
                    lam=params.lam, alpha=getattr(params, "alpha", 1.0), max_step=params.max_step,
                    outer=int(bool(getattr(params, "outer", False))))
        if _load().or_shorten(ctypes.byref(self._robot), self._cons, self.nc, ctypes.byref(p), n_paths, n_way, ld,
                              _ptr(Q), steps, eta, max_step, _ptr(out), _ptr(flags, _u8p), _ptr(resid),
                              _ptr(lengths), threads or default_threads()):
            raise MemoryError("oracle path shortening: scratch allocation failed")
        return out, flags, resid, lengths

    def count_ops(self, q, params, g=None):
        """Operations the method performs per configuration (the counting
        build of this oracle; structural zeros and signed unit factors are
        free, as in traced straight-line code).  Returns a dict of arrays
        [n, 6] (columns OP_NAMES): 'eval' = one evaluation of the stacked F,
        'step' = one LM step (F and J, Gram, Cholesky, solves, J^T y,
        update), 'vjp' = one VJP at q with upstream gradient g."""
        q = _f64(q)
        d, n = q.shape
        g = _f64(g) if g is not None else np.zeros_like(q)
        out = np.zeros((n, 18), np.uint64)
        p = _Params(tol=params.tol, max_iters=params.max_iters, cyclic=int(bool(getattr(params, "cyclic", False))),
                    lam=params.lam, alpha=getattr(params, "alpha", 1.0), max_step=params.max_step,
                    outer=int(bool(getattr(params, "outer", False))))
        _load_count().oc_count(ctypes.byref(self._robot), self._cons, self.nc, ctypes.byref(p), n, n, _ptr(q),
                               _ptr(g), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        out = out.astype(np.int64)
        return {"eval": out[:, 0:6], "step": out[:, 6:12], "vjp": out[:, 12:18]}

    def vjp(self, q, g, threads=None):
        q = _f64(q)
        g = _f64(g)
        d, n = q.shape
        v = np.zeros_like(q)
        flags = np.zeros(n, np.uint8)
        _load().or_vjp(ctypes.byref(self._robot), self._cons, self.nc, n, n, _ptr(q), _ptr(g), _ptr(v),
                       _ptr(flags, _u8p), threads or default_threads())
        return v, flags


def path_length_grad(Q, n_paths, n_way):
    """Lengths [n_paths] and gradient [d, n] of waypoint paths (SoA, path p in
    columns p * n_way ..): L = sum of |q_{w+1} - q_w|."""
    Q = _f64(Q)
    d, ld = Q.shape
    L = np.zeros(n_paths)
    G = np.zeros_like(Q)
    _load().or_path_length_grad(d, n_paths, n_way, ld, _ptr(Q), _ptr(L), _ptr(G))
    return L, G


def so3_log(R3x3):
    T = np.zeros(12)
    T.reshape(3, 4)[:, :3] = R3x3
    phi = np.zeros(3)
    _load().or_so3_log(_ptr(T), _ptr(phi))
    return phi


def so3_left_jac_inv(phi):
    M = np.zeros(9)
    _load().or_so3_left_jac_inv(_ptr(_f64(phi)), _ptr(M))
    return M.reshape(3, 3)
