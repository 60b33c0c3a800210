"""Thin ctypes binding of libmcproj.so (include/mcproj.h).

Argument marshalling only: every step of the projection, collision check and
VJP runs in the library's CUDA kernels.  PyTorch provides device memory and
streams.  There is no CPU fallback: if the library is missing or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmcproj.so")

MCP_OK, MCP_ERR_ARG, MCP_ERR_STATE, MCP_ERR_CUDA, MCP_ERR_OOM, MCP_ERR_UNSUPPORTED = range(6)
F_CONVERGED, F_CAP, F_DIVERGED, F_NONFINITE, F_FP64_RESOLVE, F_ACCEPT_FAIL, F_OUT_OF_LIMITS = 1, 2, 4, 8, 16, 32, 64
# ParallelConstrainedExtend outcomes (MCP_EXT_*)
EXT_OK, EXT_DEGENERATE, EXT_NO_PROJECTION, EXT_PROJ_COLLISION, EXT_TOO_FAR, EXT_INTERP_FAIL, EXT_GAP, \
    EXT_INTERP_COLLISION, EXT_RESOLUTION = range(9)
# constraint kinds (mcp_ckind) and their equation counts
C_SPHERE, C_AXIS_ALIGN, C_POSE, C_REL_POSE, C_COM_XY, C_PLANE, C_LINE, C_DIST, C_POSE_BOUNDED, C_COM_HULL = range(10)
C_DIM = {C_SPHERE: 1, C_AXIS_ALIGN: 2, C_POSE: 6, C_REL_POSE: 6, C_COM_XY: 2, C_PLANE: 1, C_LINE: 2, C_DIST: 1,
         C_POSE_BOUNDED: 6, C_COM_HULL: 2}
PREC_FP32, PREC_FP64 = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class RobotDesc(ctypes.Structure):
    _fields_ = [("n_joints", ctypes.c_int32), ("parent", _ip), ("type", _ip), ("X", _dp), ("lower", _dp),
                ("upper", _dp), ("mass", _dp), ("com", _dp), ("n_spheres", ctypes.c_int32), ("sphere_link", _ip),
                ("sphere", _dp), ("n_frames", ctypes.c_int32), ("frame_link", _ip), ("frame_X", _dp)]


class ConstraintDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("frame_a", ctypes.c_int32), ("frame_b", ctypes.c_int32),
                ("P", ctypes.c_double * 12), ("Q", ctypes.c_double * 12), ("target", ctypes.c_double * 3),
                ("q_ref", _dp), ("B", ctypes.c_double * 12)]


class ExtendParams(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("delta", ctypes.c_double), ("n", ctypes.c_int32),
                ("max_depth", ctypes.c_int32)]


class ProjectParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("lam", ctypes.c_double), ("max_step", ctypes.c_double), ("pivot_fp64", ctypes.c_double),
                ("cyclic", ctypes.c_int32), ("outer", ctypes.c_int32), ("alpha", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libmcproj.so (built by paper_2604_13323_gb300.build); the default
    library is loaded once per process, another path (the bounds-checked
    build) is opened beside it."""
    global _lib
    if path == LIB_PATH and _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -m paper_2604_13323_gb300.build` "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    ctx_pp = P(ctypes.c_void_p)
    sig = {
        "mcp_create": ([ctypes.c_int, ctx_pp], ctypes.c_int),
        "mcp_destroy": ([_vp], None),
        "mcp_last_error": ([_vp], ctypes.c_char_p),
        "mcp_launch_count": ([_vp], ctypes.c_int64),
        "mcp_load_robot": ([_vp, P(RobotDesc)], ctypes.c_int),
        "mcp_load_constraints": ([_vp, P(ConstraintDesc), ctypes.c_int32], ctypes.c_int),
        "mcp_load_obstacles": ([_vp, _dp, ctypes.c_int32, _dp, ctypes.c_int32], ctypes.c_int),
        "mcp_get_constraint": ([_vp, ctypes.c_int32, _dp, _dp, _dp, _dp], ctypes.c_int),
        "mcp_project_batch": ([_vp, P(ProjectParams), ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp],
                              ctypes.c_int),
        "mcp_project_check_batch": ([_vp, P(ProjectParams), ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp, _vp], ctypes.c_int),
        "mcp_project_segments": ([_vp, P(ProjectParams), ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp,
                                  ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "mcp_check_batch": ([_vp, ctypes.c_int64, ctypes.c_int64, _vp, ctypes.c_int32, _vp, _vp, _vp], ctypes.c_int),
        "mcp_project_vjp": ([_vp, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "mcp_path_length_grad": ([_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp],
                                 ctypes.c_int),
        "mcp_autotune": ([_vp, P(ProjectParams), ctypes.c_int64, ctypes.c_int64, _vp, _ip, _ip, _ip, _ip, _ip, _vp],
                         ctypes.c_int),
        "mcp_set_tuning": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
                           ctypes.c_int),
        "mcp_extend_batch": ([_vp, P(ProjectParams), P(ExtendParams), ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp,
                              ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "mcp_path_step": ([_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _vp, _vp, ctypes.c_float,
                           ctypes.c_float, _vp], ctypes.c_int),
        "mcp_project_segments_noalloc": ([_vp, P(ProjectParams), ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp,
                                          ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "mcp_fma_probe": ([_vp, ctypes.c_int32, ctypes.c_int64, _vp, P(ctypes.c_int64), _vp], ctypes.c_int),
        "mcp_alloc_count": ([], ctypes.c_int64),
        "mcp_bounds_status": ([_vp, P(ctypes.c_int32), P(ctypes.c_uint32), ctypes.c_int32], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path == LIB_PATH:
        _lib = lib
    return lib


EXPORTED = ("mcp_create", "mcp_destroy", "mcp_last_error", "mcp_launch_count", "mcp_load_robot",
            "mcp_load_constraints", "mcp_load_obstacles", "mcp_get_constraint", "mcp_project_batch",
            "mcp_project_check_batch", "mcp_project_segments", "mcp_check_batch", "mcp_project_vjp",
            "mcp_path_length_grad", "mcp_autotune", "mcp_set_tuning", "mcp_project_segments_noalloc",
            "mcp_path_step", "mcp_extend_batch", "mcp_fma_probe", "mcp_alloc_count", "mcp_bounds_status")


def alloc_count() -> int:
    """Device allocations the library has made in this process (all contexts)."""
    return int(load_library().mcp_alloc_count())


class MCPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mcproj error {status}: {msg}")
        self.status = status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Projector:
    """One library context bound to a robot, a constraint stack and obstacles.

    All batch arguments are torch CUDA tensors laid out structure-of-arrays,
    shape [d, ld] (row j = joint j), contiguous, float32 for the FP32 path and
    float64 for the plain FP64 path.
    """

    def __init__(self, robot, constraints=(), obstacles=None, device: int = 0, lib=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("mcproj needs a CUDA device; there is no CPU fallback")
        self.lib = lib if lib is not None else load_library()
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.mcp_create(device, ctypes.byref(h))
        if st != MCP_OK:
            raise MCPError(st, "mcp_create failed")
        self.h = h
        self._keep = []
        self.dof = int(np.asarray(robot.parent).shape[0])
        self.load_robot(robot)
        self.k = 0
        if constraints:
            self.load_constraints(constraints)
        if obstacles is not None:
            self.load_obstacles(obstacles)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mcp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != MCP_OK:
            raise MCPError(st, self.lib.mcp_last_error(self.h).decode())

    def _arr(self, a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        self._keep.append(a)
        return a

    def load_robot(self, rb):
        nj = int(np.asarray(rb.parent).shape[0])
        d = RobotDesc()
        d.n_joints = nj
        d.parent = self._arr(rb.parent, np.int32).ctypes.data_as(_ip)
        d.type = self._arr(rb.type, np.int32).ctypes.data_as(_ip)
        d.X = self._arr(np.asarray(rb.X).reshape(nj, 12), np.float64).ctypes.data_as(_dp)
        d.lower = self._arr(rb.lower, np.float64).ctypes.data_as(_dp)
        d.upper = self._arr(rb.upper, np.float64).ctypes.data_as(_dp)
        d.mass = self._arr(rb.mass, np.float64).ctypes.data_as(_dp)
        d.com = self._arr(np.asarray(rb.com).reshape(nj, 3), np.float64).ctypes.data_as(_dp)
        ns = int(np.asarray(rb.sphere_link).shape[0])
        d.n_spheres = ns
        d.sphere_link = self._arr(rb.sphere_link if ns else np.zeros(1), np.int32).ctypes.data_as(_ip)
        d.sphere = self._arr(np.asarray(rb.sphere).reshape(-1, 4) if ns else np.zeros((1, 4)),
                             np.float64).ctypes.data_as(_dp)
        nf = int(np.asarray(rb.frame_link).shape[0])
        d.n_frames = nf
        d.frame_link = self._arr(rb.frame_link if nf else np.zeros(1), np.int32).ctypes.data_as(_ip)
        d.frame_X = self._arr(np.asarray(rb.frame_X).reshape(-1, 12) if nf else np.zeros((1, 12)),
                              np.float64).ctypes.data_as(_dp)
        self._check(self.lib.mcp_load_robot(self.h, ctypes.byref(d)))
        self.dof = nj

    def load_constraints(self, constraints):
        n = len(constraints)
        arr = (ConstraintDesc * max(n, 1))()
        k = 0
        for i, c in enumerate(constraints):
            arr[i].kind, arr[i].frame_a, arr[i].frame_b = int(c.kind), int(c.frame_a), int(c.frame_b)
            for t in range(12):
                arr[i].P[t] = float(c.P[t])
                arr[i].Q[t] = float(c.Q[t])
            for t in range(3):
                arr[i].target[t] = float(c.target[t])
            if getattr(c, "q_ref", None) is not None:
                arr[i].q_ref = self._arr(c.q_ref, np.float64).ctypes.data_as(_dp)
            B = getattr(c, "B", None)
            for t in range(12):   # unbounded unless given
                arr[i].B[t] = float(B[t]) if B is not None else (-np.inf if t < 6 else np.inf)
            k += C_DIM[int(c.kind)]
        self._check(self.lib.mcp_load_constraints(self.h, arr, n))
        self.k = k

    def load_obstacles(self, obstacles):
        sph = self._arr(np.asarray(obstacles.spheres).reshape(-1, 4), np.float64)
        box = self._arr(np.asarray(obstacles.aabbs).reshape(-1, 6), np.float64)
        self._check(self.lib.mcp_load_obstacles(self.h, sph.ctypes.data_as(_dp), sph.shape[0],
                                                box.ctypes.data_as(_dp), box.shape[0]))

    def constraint(self, i):
        P = np.zeros(12)
        Q = np.zeros(12)
        t = np.zeros(3)
        self._check(self.lib.mcp_get_constraint(self.h, i, P.ctypes.data_as(_dp), Q.ctypes.data_as(_dp),
                                                t.ctypes.data_as(_dp), None))
        return P, Q, t

    def constraint_bounds(self, i):
        """B of constraint i (TSR bounds or support-polygon vertices) after q_ref handling."""
        B = np.zeros(12)
        self._check(self.lib.mcp_get_constraint(self.h, i, None, None, None, B.ctypes.data_as(_dp)))
        return B

    def bounds_status(self, reset=False):
        """(enabled, first source line out of range or 0) of the bounds-check
        mode (enabled only in the -DMCP_CHECK_BOUNDS build)."""
        en, line = ctypes.c_int32(), ctypes.c_uint32()
        self._check(self.lib.mcp_bounds_status(self.h, ctypes.byref(en), ctypes.byref(line), int(bool(reset))))
        return en.value, line.value

    @property
    def launches(self) -> int:
        return int(self.lib.mcp_launch_count(self.h))

    @staticmethod
    def params(p) -> ProjectParams:
        return ProjectParams(tol=p.tol, max_iters=p.max_iters, precision=p.precision, lam=p.lam,
                             max_step=p.max_step, pivot_fp64=p.pivot_fp64,
                             cyclic=int(bool(getattr(p, "cyclic", False))), outer=int(bool(getattr(p, "outer", False))),
                             alpha=float(getattr(p, "alpha", 1.0)))

    # ---- batched entry points (torch CUDA tensors) ----
    def project(self, q, params, out=None, flags=None, iters=None, resid=None, n=None, stream=None):
        import torch
        d, ld = q.shape
        n = ld if n is None else n
        out = torch.empty_like(q) if out is None else out
        flags = torch.empty(ld, dtype=torch.uint8, device=q.device) if flags is None else flags
        iters = torch.empty(ld, dtype=torch.uint8, device=q.device) if iters is None else iters
        resid = torch.empty(ld, dtype=torch.float64, device=q.device) if resid is None else resid
        pp = self.params(params)
        self._check(self.lib.mcp_project_batch(self.h, ctypes.byref(pp), n, ld, _ptr(q), _ptr(out), _ptr(flags),
                                               _ptr(iters), _ptr(resid), _stream(stream)))
        return out, flags, iters, resid

    def project_check(self, q, params, out=None, flags=None, iters=None, resid=None, hit=None, pairs=None, n=None,
                      stream=None):
        """Projection, then the collision verdict of every output (fused where
        the kernels allow): (q*, flags, iters, resid, in_collision)."""
        import torch
        d, ld = q.shape
        n = ld if n is None else n
        out = torch.empty_like(q) if out is None else out
        flags = torch.empty(ld, dtype=torch.uint8, device=q.device) if flags is None else flags
        iters = torch.empty(ld, dtype=torch.uint8, device=q.device) if iters is None else iters
        resid = torch.empty(ld, dtype=torch.float64, device=q.device) if resid is None else resid
        hit = torch.empty(ld, dtype=torch.uint8, device=q.device) if hit is None else hit
        pp = self.params(params)
        self._check(self.lib.mcp_project_check_batch(self.h, ctypes.byref(pp), n, ld, _ptr(q), _ptr(out), _ptr(flags),
                                                     _ptr(iters), _ptr(resid), _ptr(hit), _ptr(pairs),
                                                     _stream(stream)))
        return out, flags, iters, resid, hit

    def extend(self, q_s, q_t, eps, params, r, delta, max_depth=6, steps=None, out=None, stream=None):
        """ParallelConstrainedExtend (Alg. 2) of every column of q_s towards the
        same column of q_t ([d, n_ext] float32 CUDA tensors); eps [n, n_ext] the
        particle offsets; `steps` (int32 [n_ext]) optionally receives the Newton
        steps of each extension.  Returns (q_proj, status, n_points, winner)."""
        import torch
        d, m = q_s.shape
        n = eps.shape[0]
        if out is None:
            out = (torch.empty_like(q_s), torch.empty(m, dtype=torch.uint8, device=q_s.device),
                   torch.empty(m, dtype=torch.int32, device=q_s.device),
                   torch.empty(m, dtype=torch.int32, device=q_s.device))
        q_proj, status, n_points, winner = out
        pp = self.params(params)
        ep = ExtendParams(r=r, delta=delta, n=n, max_depth=max_depth)
        self._check(self.lib.mcp_extend_batch(self.h, ctypes.byref(pp), ctypes.byref(ep), m, m, _ptr(q_s), _ptr(q_t),
                                              _ptr(eps), eps.shape[1], _ptr(q_proj), _ptr(status), _ptr(n_points),
                                              _ptr(winner), _ptr(steps), _stream(stream)))
        return q_proj, status, n_points, winner

    def project_segments(self, start, delta, length, params, total=None, out=None, flags=None, iters=None,
                         resid=None, stream=None):
        import torch
        d, ld_seg = start.shape
        n_seg = length.shape[0]
        total = int(length.sum().item()) if total is None else total
        out = torch.empty((d, total), dtype=start.dtype, device=start.device) if out is None else out
        ld_out = out.shape[1]
        flags = torch.empty(ld_out, dtype=torch.uint8, device=start.device) if flags is None else flags
        iters = torch.empty(ld_out, dtype=torch.uint8, device=start.device) if iters is None else iters
        resid = torch.empty(ld_out, dtype=torch.float64, device=start.device) if resid is None else resid
        pp = self.params(params)
        self._check(self.lib.mcp_project_segments(self.h, ctypes.byref(pp), n_seg, ld_seg, _ptr(start), _ptr(delta),
                                                  _ptr(length), total, ld_out, _ptr(out), _ptr(flags), _ptr(iters),
                                                  _ptr(resid), _stream(stream)))
        return out, flags, iters, resid

    def check(self, q, out=None, n=None, pairs=None, stream=None):
        """Collision verdicts (uint8); `pairs` (int32 tensor [ld]) optionally
        receives the sphere-obstacle pairs evaluated per configuration."""
        import torch
        d, ld = q.shape
        n = ld if n is None else n
        out = torch.empty(ld, dtype=torch.uint8, device=q.device) if out is None else out
        prec = PREC_FP64 if q.dtype == torch.float64 else PREC_FP32
        self._check(self.lib.mcp_check_batch(self.h, n, ld, _ptr(q), prec, _ptr(out), _ptr(pairs), _stream(stream)))
        return out

    def vjp(self, q_star, g, out=None, flags=None, stream=None):
        import torch
        d, ld = q_star.shape
        out = torch.empty_like(g) if out is None else out
        flags = torch.empty(ld, dtype=torch.uint8, device=g.device) if flags is None else flags
        self._check(self.lib.mcp_project_vjp(self.h, ld, ld, _ptr(q_star), _ptr(g), _ptr(out), _ptr(flags),
                                             _stream(stream)))
        return out, flags

    def path_step(self, Q, D, n_paths, n_way, eta, max_step=0.0, stream=None):
        """In place: interior waypoints of Q move by -clip(eta * D)."""
        d, ld = Q.shape
        self._check(self.lib.mcp_path_step(self.h, n_paths, n_way, ld, _ptr(Q), _ptr(D), float(eta), float(max_step),
                                           _stream(stream)))
        return Q

    def autotune(self, q_sample, params, stream=None):
        """Times the persistent kernel's launch shapes on q_sample ([d, n] float32
        CUDA tensor) and keeps the fastest; returns (threads/block, blocks/SM,
        chunk, fuse_check, threads/configuration)."""
        d, n = q_sample.shape
        t, b, c, f, k = (ctypes.c_int32() for _ in range(5))
        pp = self.params(params)
        self._check(self.lib.mcp_autotune(self.h, ctypes.byref(pp), n, n, _ptr(q_sample), ctypes.byref(t),
                                          ctypes.byref(b), ctypes.byref(c), ctypes.byref(f), ctypes.byref(k),
                                          _stream(stream)))
        return t.value, b.value, c.value, f.value, k.value

    def fma_probe(self, fp64=False, iters=None, reps=5, stream=None):
        """Measured FMA throughput of this device (TFLOP/s): the best of `reps`
        timed launches of the library's FMA-chain probe."""
        import torch
        dev = torch.device("cuda", self.device)
        iters = iters or ((1 << 12) if fp64 else (1 << 16))
        out = torch.empty(1, dtype=torch.float64 if fp64 else torch.float32, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        flops = ctypes.c_int64()
        best = float("inf")
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            self._check(self.lib.mcp_fma_probe(self.h, 1 if fp64 else 0, iters, _ptr(out), ctypes.byref(flops),
                                               _stream(st)))
            e1.record(st)
            e1.synchronize()
            if r:   # the first launch warms up
                best = min(best, e0.elapsed_time(e1))
        return flops.value / (best * 1e-3) / 1e12

    def set_tuning(self, tpb, blocks_per_sm, chunk, fuse_check=0, threads_per_config=1):
        self._check(self.lib.mcp_set_tuning(self.h, int(tpb), int(blocks_per_sm), int(chunk), int(fuse_check),
                                            int(threads_per_config)))

    def path_length_grad(self, Q, n_paths, n_way, length=None, grad=None, stream=None):
        import torch
        d, ld = Q.shape
        length = torch.empty(n_paths, dtype=torch.float32, device=Q.device) if length is None else length
        grad = torch.empty_like(Q) if grad is None else grad
        self._check(self.lib.mcp_path_length_grad(self.h, n_paths, n_way, ld, _ptr(Q), _ptr(length), _ptr(grad),
                                                  _stream(stream)))
        return length, grad
