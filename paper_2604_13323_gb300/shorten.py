"""Differentiable projection and path shortening on the manifold.

`ProjectFn` wraps the library's projection as a torch.autograd.Function: the
forward is the batched projection kernel (Alg. 2 ParallelProject), the
backward the VJP kernel g - J^T (J J^T)^{-1} J g at the projected
configurations (the implicit-function-theorem adjoint; the paper makes its
log map differentiable for gradient-based optimisation, Sec. IV-A).
`PathLengthFn` is the total length sum_i |q_{i+1} - q_i| of waypoint paths,
with its gradient from the path-length kernel.

`shorten_paths` runs gradient descent on the length of many paths at once:
each step projects the waypoints, back-propagates the length through the
projection (a tangent-space gradient), moves interior waypoints with the path
step kernel and projects again in the next step.  Every numeric step runs in
the library's kernels; torch only holds the tensors and the autograd graph.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import mcproj


class ProjectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, projector, params):
        out, flags, iters, resid = projector.project(q.detach().contiguous(), params)
        ctx.projector = projector
        ctx.save_for_backward(out)
        ctx.flags = flags
        ctx.resid = resid
        return out

    @staticmethod
    def backward(ctx, g):
        (q_star,) = ctx.saved_tensors
        v, _ = ctx.projector.vjp(q_star, g.contiguous())
        return v, None, None


class PathLengthFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, projector, n_paths, n_way):
        length, grad = projector.path_length_grad(Q.detach().contiguous(), n_paths, n_way)
        ctx.save_for_backward(grad)
        ctx.n_way = n_way
        return length

    @staticmethod
    def backward(ctx, g_len):
        (grad,) = ctx.saved_tensors
        return grad * g_len.repeat_interleave(ctx.n_way)[None, :], None, None, None


def initial_paths(projector, qa, qb, noise, params):
    """Linear interpolation between projected endpoints plus waypoint noise,
    projected.  qa, qb: [d, n_paths]; noise: [d, n_paths, n_way] (zero at the
    endpoints).  Returns Q [d, n_paths * n_way] on the device."""
    d, n_paths, n_way = noise.shape
    dev = torch.device("cuda", projector.device)
    a = projector.project(torch.tensor(qa, dtype=torch.float32, device=dev), params)[0]
    b = projector.project(torch.tensor(qb, dtype=torch.float32, device=dev), params)[0]
    t = torch.linspace(0.0, 1.0, n_way, device=dev)
    Q = a[:, :, None] + (b - a)[:, :, None] * t[None, None, :] + torch.tensor(noise, dtype=torch.float32, device=dev)
    Q = Q.reshape(d, n_paths * n_way).contiguous()
    return projector.project(Q, params)[0]


def shorten_paths(projector, Q, n_paths, n_way, params, steps=100, eta=0.1, max_step=0.05):
    """Gradient descent on the total path length, on the manifold.  Returns
    (Q, stats) with the per-path lengths before and after and the final
    residuals and flags."""
    Q = Q.contiguous()
    L0 = PathLengthFn.apply(Q, projector, n_paths, n_way).detach().clone()
    Qs = Q
    for _ in range(steps):
        Qv = Q.detach().requires_grad_(True)
        Qs = ProjectFn.apply(Qv, projector, params)
        L = PathLengthFn.apply(Qs, projector, n_paths, n_way)
        L.sum().backward()
        with torch.no_grad():
            Q = Qs.detach().clone()
            projector.path_step(Q, Qv.grad.contiguous(), n_paths, n_way, eta, max_step)
    Qf, flags, _, resid = projector.project(Q, params)
    L1 = PathLengthFn.apply(Qf, projector, n_paths, n_way).detach()
    torch.cuda.synchronize()
    red = ((L0 - L1) / L0).cpu().numpy()
    conv = (flags.cpu().numpy() & mcproj.F_CONVERGED) != 0
    return Qf, {"mean_length_reduction": float(red.mean()), "min_length_reduction": float(red.min()),
                "max_resid": float(resid.cpu().numpy().max()), "converged_fraction": float(conv.mean()),
                "mean_length_before": float(L0.mean()), "mean_length_after": float(L1.mean())}


def shorten_paths_graph(projector, Q, n_paths, n_way, params, steps=100, eta=0.1, max_step=0.05):
    """The descent of `shorten_paths` without autograd: one step (project the
    waypoints, path-length gradient at the projections, its VJP through the
    projection, the clipped step) captured once as a CUDA graph and replayed,
    so that the host issues one launch per step instead of a Python loop of
    kernel calls.  The same kernels run in the same order on the same data:
    the results equal `shorten_paths`'s."""
    dev = Q.device
    d, n = Q.shape
    Qw = Q.detach().contiguous().clone()
    out = torch.empty_like(Qw)
    flags = torch.empty(n, dtype=torch.uint8, device=dev)
    iters = torch.empty(n, dtype=torch.uint8, device=dev)
    resid = torch.empty(n, dtype=torch.float64, device=dev)
    length = torch.empty(n_paths, dtype=torch.float32, device=dev)
    grad = torch.empty_like(Qw)
    v = torch.empty_like(Qw)
    vf = torch.empty(n, dtype=torch.uint8, device=dev)
    L0 = projector.path_length_grad(Qw, n_paths, n_way)[0].clone()
    side = torch.cuda.Stream(dev)

    def one_step():
        st = torch.cuda.current_stream(dev)
        projector.project(Qw, params, out=out, flags=flags, iters=iters, resid=resid, stream=st)
        projector.path_length_grad(out, n_paths, n_way, length=length, grad=grad, stream=st)
        projector.vjp(out, grad, out=v, flags=vf, stream=st)
        Qw.copy_(out)
        projector.path_step(Qw, v, n_paths, n_way, eta, max_step, stream=st)

    side.wait_stream(torch.cuda.current_stream(dev))
    if steps > 0:
        Qstart = Qw.clone()
        with torch.cuda.stream(side):
            one_step()                       # warm-up outside the capture
            Qw.copy_(Qstart)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                one_step()
            Qw.copy_(Qstart)
            for _ in range(steps):
                graph.replay()
    torch.cuda.current_stream(dev).wait_stream(side)
    Qf, fl, _, rs = projector.project(Qw, params)
    L1 = projector.path_length_grad(Qf, n_paths, n_way)[0]
    torch.cuda.synchronize()
    red = ((L0 - L1) / L0).cpu().numpy()
    conv = (fl.cpu().numpy() & mcproj.F_CONVERGED) != 0
    return Qf, {"mean_length_reduction": float(red.mean()), "min_length_reduction": float(red.min()),
                "max_resid": float(rs.cpu().numpy().max()), "converged_fraction": float(conv.mean()),
                "mean_length_before": float(L0.mean()), "mean_length_after": float(L1.mean())}


def main():  # pragma: no cover - run on a GPU
    import argparse
    import time

    from . import build, workloads as W
    ap = argparse.ArgumentParser(description="path shortening on the dual-arm manifold")
    ap.add_argument("--paths", type=int, default=4096)
    ap.add_argument("--waypoints", type=int, default=64)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--eta", type=float, default=0.1)
    ap.add_argument("--max-step", type=float, default=0.05)
    args = ap.parse_args()
    build.build()
    pw = W.path_workload(n_paths=args.paths, n_way=args.waypoints)
    wl = pw["workload"]
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    Q = initial_paths(P, pw["qa"], pw["qb"], pw["noise"], wl.params)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Qf, st = shorten_paths(P, Q, args.paths, args.waypoints, wl.params, args.steps, args.eta, args.max_step)
    torch.cuda.synchronize()
    st["seconds"] = time.perf_counter() - t0
    st["collision_fraction"] = float(P.check(Qf).float().mean().item())
    st.update(paths=args.paths, waypoints=args.waypoints, steps=args.steps, eta=args.eta, max_step=args.max_step)
    print(json.dumps(st))


if __name__ == "__main__":  # pragma: no cover
    main()
