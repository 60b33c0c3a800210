#!/usr/bin/env python3
"""Benchmark: converged projections/sec at ||F|| <= 1e-5 on one GB300.

A step is one pass of the whole hot path over one batch: projection (FP32
Newton/LM steps with FP64 acceptance, Alg. 2 ParallelProject) followed by the
sphere collision check of every projected configuration (CollisionFree).
The default workload is the largest configuration that fits one GPU: the
36-DoF humanoid (feet fixed in 6-D, hands in a fixed relative pose, centre of
mass over the feet: 20 equations), 1,048,576 configurations, tol 1e-5, cap
40, lambda 1e-6; 150 link spheres against 200 obstacle spheres and 6 boxes.
Its line also carries:
  * vs_plain_fp64: the plain per-configuration FP64 kernel projecting the same
    configurations, and the ratio of the projection kernels' throughputs;
  * sub_records: the 7-DoF arm (65,536), the dual-arm uneven segments
    (262,240 points in one persistent launch), the VJP (65,536) and path
    shortening (4,096 x 64 x 100), each with its own value and roofline;
  * cpu_baseline: the FP64 oracle on the host cores, and under it the
    whole-batch parity of the GPU's outputs against the oracle and the
    oracle-counted algorithmic flops the roofline divides.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload humanoid|arm|dual_segments|...] [--precision fp32|fp64]

Prints one JSON line (rank 0).  Under torchrun each rank projects its own
seeded batch of the same size (independent problems, no collective on the
data path); value is the sum over ranks divided by the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged projections/sec at ||F||<=1e-5 (batched FP32 vs plain FP64, 1 GB300)"
UNIT = "projections/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from one ncu capture of the kernel built from this source
# (profiles/ gives the command and the full capture summary).  Keyed by
# (workload, kernel); an entry is removed whenever its kernel changes.
MEASURED_TRAFFIC = {
    ("arm7_axis_65536", "k_project_f32+check"): 2003456,                  # read 2.00 MB, write 0
    ("humanoid36_1048576", "k_project_group"): 238427136 + 132679936,     # read 238.4 MB, write 132.7 MB
}
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="humanoid", choices=["arm", "dual_arm", "dual_segments", "sphere", "humanoid",
                                                          "arm_tray", "arm_peg", "arm_tsr", "dual_rod", "extend",
                                                          "humanoid_hull", "vjp", "shorten"])
    ap.add_argument("--cyclic", action="store_true",
                    help="cyclic getDescentStep (one LM step per constraint per sweep) instead of the stacked step")
    ap.add_argument("--cap", type=int, default=0, help="iteration cap (default: the workload's)")
    ap.add_argument("--launch", default="",
                    help="tpb,blocks_per_sm,chunk,fuse_check[,threads_per_config] instead of autotuning "
                         "(profiler runs)")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="use only the first N configurations (small cases for profilers; not a bench line)")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: split ONE batch over the ranks (contiguous ranges, or whole segments "
                         "balanced by length) and gather the outputs on the host (strong scaling); default: "
                         "one batch per rank (replicas, weak scaling)")
    ap.add_argument("--no-sub", action="store_true",
                    help="the headline workload only (no arm / dual-arm / VJP / shortening sub-records)")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the oracle's whole-batch parity and flop count (the CPU baseline still runs)")
    ap.add_argument("--profile", action="store_true",
                    help="fixed launch count for profilers: no time-padded warm-up, no CPU baseline, no e2e pass")
    return ap.parse_args()


def make_workload(name, rank):
    """(workload, batch q [d, n] or None, name, segments or None)."""
    from paper_2604_13323_gb300 import workloads as W
    if name == "arm":
        wl = W.arm_workload(n=65536, batch_seed=1001 + 1000 * rank)
        return wl, wl.q, "arm7_axis_65536", None
    if name == "sphere":
        wl = W.sphere_workload(seed=1000 + 1000 * rank)   # the point robot has no geometry to keep
        return wl, W.segment_points(wl.segments), "sphere_geodesics_1024_pairs", wl.segments
    if name == "humanoid":
        wl = W.humanoid_workload(batch_seed=1003 + 1000 * rank)
        return wl, wl.q, "humanoid36_1048576", None
    if name == "humanoid_hull":
        wl = W.humanoid_workload(batch_seed=1003 + 1000 * rank, hull=True)
        return wl, wl.q, "humanoid36_hull_1048576", None
    if name in ("arm_tray", "arm_peg", "arm_tsr"):
        wl = W.arm_task_workload(name[4:], batch_seed=None if rank == 0 else 1007 + 1000 * rank)
        return wl, wl.q, f"arm7_{name[4:]}_65536", None
    if name == "dual_rod":
        wl = W.dual_rod_workload(batch_seed=None if rank == 0 else 1009 + 1000 * rank)
        return wl, wl.q, "dual14_rod_65536", None
    if name == "dual_segments":
        wl = W.dual_arm_workload(batch_seed=None if rank == 0 else 1002 + 1000 * rank)
        return wl, None, f"dual14_rel_segments_{int(wl.extra['lengths'].sum())}", "raw"
    wl = W.dual_arm_workload(total=10, n_random=262144, batch_seed=None if rank == 0 else 1002 + 1000 * rank)
    return wl, wl.q, "dual14_rel_262144", None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def aggregate_replicas(ms, converged, world, device):
    """Whole-job numbers of independent replicas: the slowest rank's step time
    and the sum of converged projections over ranks (the only cross-rank
    exchange; the data path itself has no collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    c = torch.tensor([converged], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def apply_overrides(wl, name, args):
    """--cyclic / --cap on the workload's parameters; the workload name says so."""
    if args.cyclic:
        wl.params.cyclic = True
        name += "_cyclic"
    if args.cap:
        wl.params.max_iters = args.cap
        name += f"_cap{args.cap}"
    return name


def oracle_leg(wl, q, gpu=None, budget_s=10.0, whole_batch=True, reps=8):
    """The benchmark's CPU-baseline leg, the one place it runs the FP64 oracle.

    1. cpu_baseline: the oracle as it stands (projection + collision check,
       all host cores) on contiguous chunks of the batch for ~budget_s.
    2. parity (untimed, with the GPU's outputs `gpu` = (q [d, n], flags,
       iters, hit)): the oracle projects the WHOLE batch, plus 8 perturbed
       copies of it (8 unit roundoffs of FP32) that tell which starts have a
       result determined to the 1e-4 rad point bar; reported over all of it:
       flag agreement, equal step counts, the largest point error where the
       result is determined, the share of converged outputs (both sides)
       beyond 1e-4, collision verdicts outside the 1e-5 m contact band.
    3. algorithmic flops: the operation-counting build of the oracle on a
       sample of 256 configurations gives the flops of one evaluation of F and
       of one LM step; with the ORACLE's step counts over the whole batch
       (extra GPU steps earn nothing): FP32 = sum(iters) x step + n x eval,
       FP64 = n x eval (the acceptance).  sin / cos / sqrt / atan2 are
       special functions, counted apart.
    Returns (cpu_baseline, parity or None, flops or None)."""
    from oracle import oracle as orc
    from oracle import parity as par
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    threads = orc.default_threads()
    p = wl.params
    chunk = 4096
    done = conv = 0
    t0 = time.perf_counter()
    off = 0
    while time.perf_counter() - t0 < budget_s:
        sl = q[:, off:off + chunk]
        out, fl, it, r = O.project(sl, p.tol, p.max_iters, p.lam, max_step=p.max_step, cyclic=p.cyclic,
                                   threads=threads)
        O.check(out, threads=threads)
        conv += int(((fl & orc.CONVERGED) != 0).sum())
        done += sl.shape[1]
        off = (off + chunk) % q.shape[1]
    dt = time.perf_counter() - t0
    cpu = {"value": conv / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{done} configurations (contiguous chunks of {chunk} of the bench batch), "
                     f"projection + collision check, FP64, {dt:.1f} s wall"}
    if not whole_batch or gpu is None:
        return cpu, None, None
    t1 = time.perf_counter()
    n = q.shape[1]
    selfst = {}
    el, (qo, fo, io, ro) = par.eligible_mask(O, q, p.tol, p.max_iters, p.lam, max_step=p.max_step,
                                             cyclic=p.cyclic, reps=reps, stats=selfst)
    qg, fg, ig, hg = gpu
    cg, co = (fg & orc.CONVERGED) != 0, (fo & orc.CONVERGED) != 0
    both = cg & co
    same = both & (ig.astype(np.int64) == io)
    err = np.abs(qg.astype(np.float64) - qo).max(axis=0)
    cmp_ = same & el
    hit_o, margin = O.check(qg.astype(np.float64), threads=threads)
    band = margin >= 1e-5
    parity = {"configs": int(n), "scope": "whole batch", "eligible": float(el.mean()),
              "eligibility": f"oracle result moves <= 1e-4 under {reps} perturbations of 8 FP32 unit roundoffs",
              "flag_agree": float((cg == co).mean()),
              "flag_agree_eligible": float((cg == co)[el].mean()) if el.any() else 1.0,
              "oracle_self_flip_rate": selfst.get("self_flip_rate"),
              "iters_equal": float(same.sum() / max(1, both.sum())),
              "compared": int(cmp_.sum()),
              "q_err_max_eligible": float(err[cmp_].max()) if cmp_.any() else 0.0,
              "q_err_p999_eligible": float(np.quantile(err[cmp_], 0.999)) if cmp_.any() else 0.0,
              "eligible_beyond_1e-4": int((err[cmp_] > 1e-4).sum()),
              "converged_beyond_1e-4": float((err[both] > 1e-4).mean()) if both.any() else 0.0,
              "hit_agree_outside_band": float(((hg != 0) == (hit_o != 0))[band].mean()) if band.any() else 1.0,
              "hit_excluded_band": int((~band).sum()),
              "wall_s": round(time.perf_counter() - t1, 1)}
    idx = np.linspace(0, n - 1, min(n, 256)).astype(np.int64)
    cnt = O.count_ops(q[:, idx], p)
    ev = cnt["eval"].mean(axis=0)
    st = cnt["step"].mean(axis=0)
    eval_f, step_f = float(ev[:3].sum()), float(st[:3].sum())
    flops = {"fp32": float(io.sum()) * step_f + n * eval_f, "fp64": n * eval_f,
             "per_step": step_f, "per_eval": eval_f, "oracle_mean_iters": float(io.mean()),
             "special_per_step": dict(zip(orc.OP_NAMES[3:], [float(v) for v in st[3:]])),
             "source": "operation-counting build of the oracle (256 sampled configurations) x the oracle's "
                       "step counts over the whole batch"}
    return cpu, parity, flops


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "extend":
        return run_reference_extend(args)
    if args.workload == "vjp":
        return run_reference_vjp(args)
    if args.workload == "shorten":
        return run_reference_shorten(args)
    wl, q, wname, segs = make_workload(args.workload, 0)
    wname = apply_overrides(wl, wname, args)
    from oracle import oracle as orc
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    threads = orc.default_threads()
    p = wl.params
    if q is None:   # segments: the starts projected by the oracle (setup), then the points on them
        from paper_2604_13323_gb300 import workloads as W
        ex = wl.extra
        starts = O.project(ex["raw_start"], p.tol, p.max_iters, p.lam, threads=threads)[0]
        q = W.segment_points(W.Segments(start=starts, delta=ex["raw_dir"] * ex["step"], length=ex["lengths"]))
    sample = min(q.shape[1], 8192)
    times, convs = [], []
    for s in range(args.warmup + args.steps):
        sl = q[:, (s * sample) % q.shape[1]:][:, :sample]
        t0 = time.perf_counter()
        out, fl, _, _ = O.project(sl, p.tol, p.max_iters, p.lam, max_step=p.max_step, cyclic=p.cyclic,
                                  threads=threads)
        O.check(out, threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            convs.append(int(((fl & orc.CONVERGED) != 0).sum()))
    total = sum(times)
    value = sum(convs) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "batch_per_step": sample, "dof": wl.dof, "k": wl.k, "tol": p.tol,
                       "cap": p.max_iters},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} configurations per step, projection + collision check"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_vjp(args):
    """Reference arm of the VJP workload: the oracle's FP64 VJP at the
    oracle-projected configurations (setup), 8192 per step."""
    from oracle import oracle as orc
    from paper_2604_13323_gb300 import workloads as W
    wl = W.dual_arm_workload(total=10, n_random=VJP_N, batch_seed=1011)
    p = wl.params
    O = orc.Oracle(wl.robot, wl.constraints)
    threads = orc.default_threads()
    q_star = O.project(wl.q, p.tol, p.max_iters, p.lam, threads=threads)[0]
    g = np.random.default_rng(1012).standard_normal((14, VJP_N))
    sample = 8192
    times = []
    for s in range(args.warmup + args.steps):
        sl = slice((s * sample) % VJP_N, (s * sample) % VJP_N + sample)
        t0 = time.perf_counter()
        O.vjp(q_star[:, sl], g[:, sl], threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = sample * len(times) / total
    unit = "VJPs/s"
    line = {"impl": "reference", "metric": "vector-Jacobian products/sec at q* (dual-arm closed chain, 1 GB300)",
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dual14_rel_vjp_{VJP_N}", "vjps_per_step": sample},
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} VJPs per step"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_initial_paths(O, pw, p, threads):
    """The shortening workload's initial waypoints, built by the oracle the
    way the GPU driver builds them: projected endpoints, linear interpolation
    plus the seeded noise, projected."""
    qa = O.project_params(pw["qa"], p, threads=threads)[0]
    qb = O.project_params(pw["qb"], p, threads=threads)[0]
    t = np.linspace(0.0, 1.0, pw["n_way"])
    Q = (qa[:, :, None] + (qb - qa)[:, :, None] * t[None, None, :] + pw["noise"]).reshape(qa.shape[0], -1)
    return O.project_params(Q, p, threads=threads)[0]


def run_reference_shorten(args):
    """Reference arm of the path-shortening workload: the oracle's FP64
    descent (project, length gradient, VJP, clipped step; SHORTEN_STEPS steps)
    on the host cores, SHORTEN_REF_PATHS paths of WAYPOINTS waypoints per
    step (their initial waypoints built by the oracle, untimed)."""
    from oracle import oracle as orc
    from paper_2604_13323_gb300 import workloads as W
    pw = W.path_workload(n_paths=PATHS, n_way=WAYPOINTS)
    wl = pw["workload"]
    p = wl.params
    O = orc.Oracle(wl.robot, wl.constraints)
    threads = orc.default_threads()
    nb = SHORTEN_REF_PATHS
    times, red = [], []
    for s_ in range(args.warmup + args.steps):
        sl = slice((s_ * nb) % PATHS, (s_ * nb) % PATHS + nb)
        sub = {"qa": pw["qa"][:, sl], "qb": pw["qb"][:, sl], "noise": pw["noise"][:, sl], "n_way": WAYPOINTS}
        Q0 = oracle_initial_paths(O, sub, p, threads)
        t0 = time.perf_counter()
        _, _, _, L = O.shorten(Q0, nb, WAYPOINTS, p, SHORTEN_STEPS, 0.1, 0.05, threads=threads)
        dt = time.perf_counter() - t0
        if s_ >= args.warmup:
            times.append(dt)
            red.append(float(np.mean(1.0 - L[:, 1] / L[:, 0])))
    total = sum(times)
    units = nb * WAYPOINTS * SHORTEN_STEPS
    value = units * len(times) / total
    unit = "waypoint-steps/s"
    line = {"impl": "reference", "metric": "path-shortening waypoint steps/sec on the manifold (dual arm, 1 GB300)",
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dual14_rel_shorten_{PATHS}x{WAYPOINTS}x{SHORTEN_STEPS}",
                       "paths_per_step": nb, "mean_length_reduction": float(np.mean(red))},
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": f"{nb} paths x {WAYPOINTS} waypoints x {SHORTEN_STEPS} descent steps per step"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_extend(args):
    """Reference arm of the extend workload: the oracle's Alg. 2 on the host
    cores, 1024 extensions per step."""
    from oracle import oracle as orc
    from paper_2604_13323_gb300 import workloads as W
    wl = W.extend_workload(n_ext=EXT_N)
    ex, p = wl.extra, wl.params
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    threads = orc.default_threads()
    qs = O.project(ex["raw_start"], p.tol, p.max_iters, p.lam, threads=threads)[0]
    sample = 1024
    times, pts = [], []
    for s in range(args.warmup + args.steps):
        sl = slice((s * sample) % EXT_N, (s * sample) % EXT_N + sample)
        t0 = time.perf_counter()
        res = O.extend(qs[:, sl], ex["target"][:, sl], ex["eps"][:, sl], p, ex["r"], ex["delta"], threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pts.append(int(res[2].sum()))
    total = sum(times)
    value = sum(pts) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"dual14_rel_extend_{EXT_N}", "extensions_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} extensions per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def init_dist():
    """(world, rank, local rank, device) of this process; NCCL process group
    for the replica aggregation under torchrun."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    return world, rank, local, torch.device("cuda", local)


def measured_peaks(local):
    """FP32 and FP64 FMA throughput of this GPU, measured with the library's
    FMA-chain probe (TFLOP/s), for the roofline's denominators."""
    from paper_2604_13323_gb300 import mcproj
    from paper_2604_13323_gb300 import workloads as W
    P = mcproj.Projector(W.sphere_workload(n_pairs=2).robot, device=local)
    try:
        return {"fp32_fma": P.fma_probe(fp64=False), "fp64_fma": P.fma_probe(fp64=True),
                "source": "mcp_fma_probe: 8 blocks of 256 threads per SM, 8 independent FMA chains per thread, "
                          "best of 5 launches, CUDA events"}
    finally:
        P.close()


def run_ours(args):
    """The step on the requested workload; for the default (the humanoid, the
    largest configuration that fits one GPU) the line also carries the arm,
    the dual-arm segments, the VJP and path shortening as sub-records."""
    import torch.distributed as dist
    world, rank, local, dev = init_dist()
    from paper_2604_13323_gb300 import build as B
    B.build()
    peaks = None if args.profile else measured_peaks(local)
    env = {"world": world, "rank": rank, "local": local, "dev": dev, "peaks": peaks}
    line = measure_batch(args, args.workload, env)
    if line is not None and args.workload == "humanoid" and not (args.profile or args.batch or args.no_sub):
        subs = {}
        for w in ("arm", "dual_segments"):
            subs[w] = compact(measure_batch(args, w, env, sub=True))
        for w in ("vjp", "shorten"):
            subs[w] = compact(run_adjoint(args, env, w, sub=True))
        line["sub_records"] = subs
    if line is not None and rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def compact(line):
    """The parts of a workload's line kept as a sub-record of the headline."""
    if line is None:
        return None
    keep = {k: line[k] for k in ("metric", "value", "unit", "ms_per_step", "dtype") if k in line}
    keep["workload"] = line["config"]["workload"]
    r = line.get("roofline") or {}
    keep["roofline"] = {k: r[k] for k in ("kernel", "bound", "achieved", "peak", "frac", "fp64_frac",
                                          "mixed_bound_frac") if k in r}
    for k in ("vs_plain_fp64", "e2e"):
        if line.get(k):
            keep[k] = line[k]
    for k in ("mean_length_reduction", "max_resid"):
        if k in line.get("config", {}):
            keep[k] = line["config"][k]
    return keep


def measure_batch(args, name, env, sub=False):
    """One workload of the batch / segment projection: warm-up, the timed
    steps (projection + collision check), the plain FP64 kernel on the same
    configurations, end to end through the C ABI with host buffers, the
    oracle leg (CPU baseline, whole-batch parity, counted flops) and the
    roofline.  `sub`: a sub-record (no e2e, no oracle leg).  Returns the line
    (rank 0) or None."""
    import torch
    world, rank, local, dev = env["world"], env["rank"], env["local"], env["dev"]
    from paper_2604_13323_gb300 import flops as FL
    from paper_2604_13323_gb300 import mcproj
    from paper_2604_13323_gb300 import workloads as W

    sharded = bool(args.shard) and world > 1
    # replicas: each rank its own seeded batch; --shard: every rank the same
    # batch, of which it projects its contiguous part
    wl, q_np, wname, segs = make_workload(name, 0 if sharded else rank)
    wname = apply_overrides(wl, wname, args)
    shard_info = None
    if sharded:
        from paper_2604_13323_gb300 import shard as SHD
        if segs is None:
            rr = SHD.batch_ranges(q_np.shape[1], world)
            a_, b_ = rr[rank]
            q_np = q_np[:, a_:b_]
            shard_info = {"partition": "contiguous configuration ranges", "ranges": rr,
                          "total": int(rr[-1][1])}
        else:
            lens = wl.extra["lengths"]
            sr = SHD.segment_ranges(lens, world)
            a_, b_ = sr[rank]
            for key in ("raw_start", "raw_dir"):
                wl.extra[key] = np.ascontiguousarray(wl.extra[key][:, a_:b_])
            wl.extra["lengths"] = np.ascontiguousarray(lens[a_:b_])
            pr = SHD.point_ranges(lens, sr)
            shard_info = {"partition": "runs of whole segments balanced by their lengths", "ranges": pr,
                          "segment_ranges": sr, "total": int(pr[-1][1])}
    if args.batch and q_np is not None:
        q_np = q_np[:, :args.batch]
        wname += f"_first{args.batch}"
    if args.precision == "fp64":
        wl.params.precision = W.PREC_FP64
    elif args.precision == "fp32":
        wl.params.precision = W.PREC_FP32
    fp64 = wl.params.precision == W.PREC_FP64
    dt = torch.float64 if fp64 else torch.float32
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles, device=local)
    stream = torch.cuda.current_stream(dev)
    seg_args = None
    if segs is not None:
        if segs == "raw":   # starts projected on the device (setup, untimed); ambient unit directions
            st0 = torch.tensor(wl.extra["raw_start"], dtype=dt, device=dev)
            starts = P.project(st0, wl.params)[0]
            delta = torch.tensor(wl.extra["raw_dir"] * wl.extra["step"], dtype=dt, device=dev)
            length = torch.tensor(wl.extra["lengths"], dtype=torch.int32, device=dev)
        else:
            starts = torch.tensor(segs.start, dtype=dt, device=dev)
            delta = torch.tensor(segs.delta, dtype=dt, device=dev)
            length = torch.tensor(segs.length, dtype=torch.int32, device=dev)
        n = int(length.sum().item())
        d = starts.shape[0]
        seg_args = (starts, delta, length)
        # the same points, materialised on the host, for the CPU baseline
        cpu_q = W.segment_points(W.Segments(start=starts.double().cpu().numpy(), delta=delta.double().cpu().numpy(),
                                            length=length.cpu().numpy()))
        q_np = None
    else:
        d, n = q_np.shape
        cpu_q = q_np
    q_in = torch.tensor(q_np, dtype=dt, device=dev) if q_np is not None else None
    q_out = torch.empty((d, n), dtype=dt, device=dev)
    flags = torch.empty(n, dtype=torch.uint8, device=dev)
    iters = torch.empty(n, dtype=torch.uint8, device=dev)
    resid = torch.empty(n, dtype=torch.float64, device=dev)
    hit = torch.empty(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    fused = seg_args is None   # a plain batch: projection and check in one call

    def step(ev=None, separate=False):
        if ev:
            ev[0].record(stream)
        if seg_args is not None:
            P.project_segments(*seg_args, wl.params, total=n, out=q_out, flags=flags, iters=iters, resid=resid,
                               stream=stream)
        elif fused and not separate:
            P.project_check(q_in, wl.params, out=q_out, flags=flags, iters=iters, resid=resid, hit=hit,
                            stream=stream)
            if ev:
                ev[1].record(stream)
                ev[2].record(stream)
            return
        else:
            P.project(q_in, wl.params, out=q_out, flags=flags, iters=iters, resid=resid, stream=stream)
        if ev:
            ev[1].record(stream)
        P.check(q_out, out=hit, stream=stream)
        if ev:
            ev[2].record(stream)

    # launch shape: the library's autotuner over threads per block, resident
    # blocks per SM and claim size, on this batch (setup, untimed)
    tuning = None
    if not fp64 and not name.startswith("humanoid"):
        if args.launch:   # a fixed shape (profiler runs reproduce the tuned one)
            vals = [int(v) for v in args.launch.split(",")]
            P.set_tuning(*vals)
        else:   # segments: tuned on a batch of all their materialised points (the same persistent kernel)
            sample = q_in if seg_args is None else torch.tensor(cpu_q, dtype=dt, device=dev)
            vals = P.autotune(sample, wl.params)
        tuning = dict(zip(("tpb", "blocks_per_sm", "chunk", "fuse_check", "threads_per_config"), vals))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    with sampler:
        # warm-up: at least W steps and at least ~1.5 s of back-to-back load, so
        # that the clock sampler sees the GPU under load around the timed steps
        t0 = time.perf_counter()
        w = 0
        while w < args.warmup or (not args.profile and time.perf_counter() - t0 < 1.5):
            flush.zero_()
            step()
            w += 1
            if w % 64 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches0 = P.launches
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.zero_()          # L2 flush between timed steps (outside the events)
            step(evs[s])
        torch.cuda.synchronize()
    launches = P.launches - launches0
    # the same step as two calls (projection, then check), for comparison only
    sep_ms = None
    if fused and not args.profile:
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        for s_ in range(args.steps):
            flush.zero_()
            step(sev[s_], separate=True)
        torch.cuda.synchronize()
        sep_ms = {"project": sum(e[0].elapsed_time(e[1]) for e in sev) / args.steps,
                  "check": sum(e[1].elapsed_time(e[2]) for e in sev) / args.steps}
    if world > 1:
        dist.barrier()
    pairs = torch.zeros(n, dtype=torch.int32, device=dev)
    P.check(q_out, out=hit, pairs=pairs, stream=stream)   # untimed: counts the pairs the timed kernel tested
    torch.cuda.synchronize()
    pairs_total = float(pairs.double().sum().item())
    t_proj = [e[0].elapsed_time(e[1]) for e in evs]
    t_check = [e[1].elapsed_time(e[2]) for e in evs]
    t_step = [e[0].elapsed_time(e[2]) for e in evs]
    ms = sum(t_step) / len(t_step)
    fl_np = flags.cpu().numpy()
    rs_np = resid.cpu().numpy()
    it_np = iters.cpu().numpy()
    conv = int((((fl_np & mcproj.F_CONVERGED) != 0) & (rs_np <= wl.params.tol)).sum())
    ms_max, c_total = aggregate_replicas(ms, conv, world, dev)
    value = c_total / (ms_max * 1e-3)

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its inputs from pinned host memory, projects and checks
    # them, and copies the outputs back.  Two buffer sets on two streams form a
    # pipeline: the copies of one step overlap the kernel of the previous one,
    # while the kernels themselves stay serialised (an event chain), so that no
    # two steps compute at the same time.  Time from the first copy-in to the
    # last copy-out, divided by the steps.
    if seg_args is not None:   # the step's inputs are the segment descriptions
        host_in = [t.cpu().pin_memory() for t in seg_args]
    else:
        host_in = [torch.tensor(q_np, dtype=dt).pin_memory()]
    NB = 2
    streams = [torch.cuda.Stream(dev) for _ in range(NB)]
    bufs = []
    for _ in range(NB):
        bufs.append({
            "in": [torch.empty_like(t, device=dev) for t in host_in],
            "q": torch.empty((d, n), dtype=dt, device=dev), "fl": torch.empty(n, dtype=torch.uint8, device=dev),
            "it": torch.empty(n, dtype=torch.uint8, device=dev), "rs": torch.empty(n, dtype=torch.float64, device=dev),
            "hit": torch.empty(n, dtype=torch.uint8, device=dev),
            "q_h": torch.empty((d, n), dtype=dt).pin_memory(), "fl_h": torch.empty(n, dtype=torch.uint8).pin_memory(),
            "hit_h": torch.empty(n, dtype=torch.uint8).pin_memory()})

    def e2e_step(b, after):
        """One step on buffer set b; its kernel waits for the event `after`."""
        st, B = streams[b], bufs[b]
        with torch.cuda.stream(st):
            for hi, di in zip(host_in, B["in"]):
                di.copy_(hi, non_blocking=True)
            if after is not None:
                st.wait_event(after)
            if seg_args is not None:
                P.project_segments(*B["in"], wl.params, total=n, out=B["q"], flags=B["fl"], iters=B["it"],
                                   resid=B["rs"], stream=st)
                P.check(B["q"], out=B["hit"], stream=st)
            else:
                P.project_check(B["in"][0], wl.params, out=B["q"], flags=B["fl"], iters=B["it"], resid=B["rs"],
                                hit=B["hit"], stream=st)
            done = torch.cuda.Event()
            done.record(st)
            B["q_h"].copy_(B["q"], non_blocking=True)
            B["fl_h"].copy_(B["fl"], non_blocking=True)
            B["hit_h"].copy_(B["hit"], non_blocking=True)
        return done

    e2e_ms = []
    if not (args.profile or sub):
        last = None
        for s_ in range(args.warmup):
            last = e2e_step(s_ % NB, last)
        torch.cuda.synchronize()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = [torch.cuda.Event(enable_timing=True) for _ in range(NB)]
        e_start.record(streams[0])
        streams[1].wait_event(e_start)
        last = None
        for s_ in range(args.steps):
            last = e2e_step(s_ % NB, last)
        for b in range(NB):
            e_end[b].record(streams[b])
        torch.cuda.synchronize()
        e2e_ms = [max(e_start.elapsed_time(e) for e in e_end) / args.steps]
        # the same steps one at a time on one stream (copies not hidden), for reference
        ser = []
        for s_ in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(streams[0])
            e2e_step(0, None)
            e1.record(streams[0])
            torch.cuda.synchronize()
            if s_ >= args.warmup:
                ser.append(e0.elapsed_time(e1))
        serial_ms = sum(ser) / len(ser)
    out_last = bufs[(args.steps - 1) % NB]
    conv_e2e = int(((out_last["fl_h"].numpy() & mcproj.F_CONVERGED) != 0).sum())
    e2e_ms_max, e2e_c = aggregate_replicas(sum(e2e_ms) / max(1, len(e2e_ms)), conv_e2e, world, dev)
    e2e = {"value": e2e_c / (e2e_ms_max * 1e-3) if e2e_ms else None, "unit": UNIT,
           "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in host_in),
           "d2h_bytes_per_step": out_last["q_h"].numel() * out_last["q_h"].element_size() + 2 * n,
           "pipeline": "2 buffer sets on 2 streams: copies overlap the previous step's kernel; kernels serialised"}
    if e2e_ms:
        ser_max, _ = aggregate_replicas(serial_ms, conv_e2e, world, dev)
        e2e["serial_value"] = e2e_c / (ser_max * 1e-3)
        e2e["serial_ms_per_step"] = ser_max

    # ---- the plain per-configuration FP64 kernel on the same configurations ----
    plain = None
    if not fp64 and not args.profile:
        plain = plain_fp64_run(P, wl, q_in, seg_args, n, d, dev, stream, flush, args, world)
        if plain is not None:
            # the projection alone on both sides (the separate-call timing when the step fuses the check)
            mp32 = sep_ms["project"] if sep_ms is not None else sum(t_proj) / len(t_proj)
            fp32_proj_value = conv / (mp32 * 1e-3)
            plain["fp32_projection"] = {"value": fp32_proj_value, "ms": mp32, "converged": conv}
            plain["ratio_projection"] = fp32_proj_value / plain["value"] if plain["value"] > 0 else None

    # ---- the oracle leg: CPU baseline, whole-batch parity, counted algorithmic flops ----
    cpu = parity = oflops = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.profile or sub):
        if seg_args is None:   # the oracle starts from the FP32 values the GPU projected
            q_or = np.asarray(cpu_q, dtype=np.float32).astype(np.float64)
        else:                  # the points formed in FP32 as the kernel forms them: start + t * delta
            q_or = segment_points_f32(seg_args)
        gpu_out = None
        if not fp64:
            gpu_out = (q_out.cpu().numpy(), flags.cpu().numpy(), iters.cpu().numpy(), hit.cpu().numpy())
        cpu, parity, oflops = oracle_leg(wl, q_or, gpu=gpu_out, whole_batch=not fp64 and not args.no_parity)

    # ---- roofline of the dominant kernel ----
    fm = FL.FlopModel(wl.robot, wl.constraints, cyclic=bool(wl.params.cyclic))
    if oflops is not None:
        fp32, fp64f = oflops["fp32"], oflops["fp64"]
        flop_src = oflops["source"]
    else:
        fp32, fp64f = fm.projection(it_np, sincos=False)
        flop_src = "kernel-structure model (flops.py) without sin/cos, the kernel's own step counts"
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    clk = sampler.summary()
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak32 = sms * 128 * 2 * sm_max * 1e6 / 1e12        # FP32 FMA lanes x 2 flops x max clock
    peaks = env.get("peaks") or {}
    peak64 = peaks.get("fp64_fma") or 1.25                # measured DFMA chains, else the nominal figure
    peak64_src = (peaks.get("source", "") + " (FP64)") if peaks.get("fp64_fma") else "nominal dense FP64"
    # one fused kernel: FP32 batch problems of the thread-per-configuration kernels
    one_kernel = fused and bool(tuning and tuning.get("fuse_check"))
    if fused and not one_kernel and sep_ms is not None:   # two launches: per-kernel times from the separate calls
        mp, mc = sep_ms["project"], sep_ms["check"]
    else:
        mp = sum(t_proj) / len(t_proj)
        mc = sum(t_check) / len(t_check)
    # collision: FK with translations + 8 flops (4 FMA) per overlap test performed (broad and
    # narrow phase); sphere transforms are not counted (conservative)
    check_flops = n * fm.fk_positions() + 8.0 * pairs_total
    check_roof = {"kernel": "k_check_f32", "pairs_per_config": pairs_total / n}
    peak_src = f"{sms} SMs x 128 FP32 lanes x 2 x max SM clock (measured FFMA chains: " \
               f"{peaks.get('fp32_fma', float('nan')):.1f} TFLOP/s)"
    common = {"peak_source": peak_src, "fp64_peak": peak64, "fp64_peak_source": peak64_src,
              "fp32_fma_measured": peaks.get("fp32_fma"), "flops_source": flop_src}
    if oflops is not None:
        common["flops_oracle"] = {k: oflops[k] for k in ("per_step", "per_eval", "oracle_mean_iters",
                                                           "special_per_step")}
    if one_kernel:
        t = mp * 1e-3
        ach32 = (fp32 + check_flops) / t / 1e12
        ach64 = fp64f / t / 1e12
        t_min = max((fp32 + check_flops) / (peak32 * 1e12), fp64f / (peak64 * 1e12))
        roof = {"bound": "alu", "achieved": ach32, "peak": peak32, "unit": "TFLOP/s", "frac": ach32 / peak32,
                "traffic": MEASURED_TRAFFIC.get((wname, "k_project_f32+check")),
                "kernel": "k_project_f32 with the check fused (persistent: FP32 steps, FP64 acceptance, "
                          "collision check)",
                "fp64_achieved": ach64, "fp64_frac": ach64 / peak64, "mixed_bound_frac": t_min / t,
                "flops_per_config": {"fp32_projection": fp32 / n, "fp32_check": check_flops / n, "fp64": fp64f / n},
                "check": check_roof, **common}
        kernel_ms = {"project_check": mp}
    else:
        check_roof["achieved"] = check_flops / (mc * 1e-3) / 1e12
        check_roof["frac"] = check_roof["achieved"] / peak32
        if fp64:
            flops_proj = fp32 + fp64f   # the plain kernel does all of it in FP64
            ach = flops_proj / (mp * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peak64, "unit": "TFLOP/s", "frac": ach / peak64,
                    "traffic": None, "kernel": "k_project_f64 (plain FP64)", **common}
        else:
            ach32 = fp32 / (mp * 1e-3) / 1e12
            ach64 = fp64f / (mp * 1e-3) / 1e12
            # both pipes: the time the FP32 and FP64 work need at their peaks bounds the kernel
            t_min = max(fp32 / (peak32 * 1e12), fp64f / (peak64 * 1e12))
            kshort = ("k_project_group" if name.startswith("humanoid") and not wl.params.cyclic else
                      "k_project_warp" if name.startswith("humanoid") else
                      "k_project_pair" if tuning and tuning.get("threads_per_config") == 2 else "k_project_f32")
            roof = {"bound": "alu", "achieved": ach32, "peak": peak32, "unit": "TFLOP/s", "frac": ach32 / peak32,
                    "traffic": MEASURED_TRAFFIC.get((wname, kshort)),
                    "kernel": kshort + {
                        "k_project_group": " (four lanes per configuration: FP32 steps, FP64 acceptance)",
                        "k_project_warp": " (warp per configuration, cyclic sweeps)",
                        "k_project_pair": " (persistent, one lane per arm: FP32 steps + FP64 acceptance)",
                        "k_project_f32": " (persistent, FP32 steps + FP64 acceptance)"}[kshort],
                    "fp64_achieved": ach64, "fp64_frac": ach64 / peak64,
                    "mixed_bound_frac": t_min / (mp * 1e-3),
                    "flops_per_config": {"fp32": fp32 / n, "fp64": fp64f / n}, **common}
        kernel_ms = {"project": mp, "check": mc}
        roof["check"] = check_roof
        if mc > mp and not fp64:   # the dominant kernel carries the headline roofline
            roof = {"bound": "alu", "achieved": check_roof["achieved"], "peak": peak32, "unit": "TFLOP/s",
                    "frac": check_roof["achieved"] / peak32, "traffic": None,
                    "kernel": "k_check_f32 (collision, 8 flops per overlap test, broad + narrow phase)",
                    "peak_source": peak_src, "projection": roof}
    if sep_ms is not None:
        kernel_ms["separate_calls"] = sep_ms
    if shard_info is not None:   # the host gather of every rank's outputs (after the timed region)
        t_g = time.perf_counter()
        full = SHD.gather_columns([q_out, flags, iters, resid, hit], shard_info["ranges"], shard_info["total"])
        shard_info.update(gathered_columns=int(full[0].shape[-1]), gather_s=round(time.perf_counter() - t_g, 3),
                          converged_gathered=int(((full[1] & mcproj.F_CONVERGED) != 0).sum()))
        del shard_info["ranges"]
    if cpu is not None and parity is not None:
        cpu["parity_vs_gpu"] = parity
    P.close()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "shard": shard_info,
            "vs_baseline": None, "vs_plain_fp64": plain, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": {"workload": wname, "batch": n, "dof": d, "k": wl.k, "tol": wl.params.tol,
                       "source": "segments (persistent launch, CUDA graph)" if seg_args is not None else "batch",
                       "cap": wl.params.max_iters, "lambda": wl.params.lam,
                       "form": "cyclic" if wl.params.cyclic else "stacked",
                       "precision": "fp64 plain" if fp64 else "fp32 + fp64 acceptance",
                       "obstacles": int(wl.obstacles.spheres.shape[0]), "robot_spheres": wl.robot.n_spheres,
                       "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"shard x{world}" if sharded else f"replicas x{world}",
                       "converged_per_step": conv,
                       "kernel_ms": kernel_ms, "mean_iters": float(it_np.mean()), "launch": tuning,
                       "flag_fractions": {k: float(((fl_np & b) != 0).mean()) for k, b in
                                          (("cap", mcproj.F_CAP), ("fp64_resolve", mcproj.F_FP64_RESOLVE),
                                           ("accept_fail", mcproj.F_ACCEPT_FAIL),
                                           ("nonfinite", mcproj.F_NONFINITE))}},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e if not sub else None, "gpu_launches": launches,
            "clocks": clk}


def segment_points_f32(seg_args):
    """The segment points as the kernel forms them, start + t * delta in FP32
    (one rounding), returned as FP64."""
    import torch
    starts, delta, length = (t.cpu() for t in seg_args)
    t = torch.cat([torch.arange(int(ln), dtype=torch.float32) for ln in length.tolist()])
    sid = torch.repeat_interleave(torch.arange(length.shape[0]), length.long())
    return torch.addcmul(starts.float()[:, sid], t[None, :], delta.float()[:, sid]).double().numpy()


def plain_fp64_run(P, wl, q_in, seg_args, n, d, dev, stream, flush, args, world, steps=3):
    """The plain per-configuration FP64 kernel (FP64 FK, Jacobian, Cholesky,
    CUDA's double-precision math; no FP32 step) projecting the same
    configurations: converged projections per second of the projection
    kernel alone, timed like the FP32 path (L2 flushed, CUDA events, warm-up
    first).  The configurations are the FP32 inputs, widened."""
    import copy
    import torch
    from paper_2604_13323_gb300 import mcproj
    from paper_2604_13323_gb300 import workloads as W
    p64 = copy.copy(wl.params)
    p64.precision = W.PREC_FP64
    out = torch.empty((d, n), dtype=torch.float64, device=dev)
    fl = torch.empty(n, dtype=torch.uint8, device=dev)
    it = torch.empty(n, dtype=torch.uint8, device=dev)
    rs = torch.empty(n, dtype=torch.float64, device=dev)
    if seg_args is not None:
        sa = (seg_args[0].double(), seg_args[1].double(), seg_args[2])

        def call():
            P.project_segments(*sa, p64, total=n, out=out, flags=fl, iters=it, resid=rs, stream=stream)
    else:
        q64 = q_in.double()

        def call():
            P.project(q64, p64, out=out, flags=fl, iters=it, resid=rs, stream=stream)
    try:
        call()
        torch.cuda.synchronize()
    except mcproj.MCPError as e:
        return {"unavailable": str(e)}
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = sum(ts) / len(ts)
    conv = int((((fl.cpu().numpy() & mcproj.F_CONVERGED) != 0) & (rs.cpu().numpy() <= wl.params.tol)).sum())
    ms_max, c_total = aggregate_replicas(ms, conv, world, dev)
    return {"value": c_total / (ms_max * 1e-3), "unit": UNIT, "ms": ms_max, "converged": conv, "steps": steps,
            "kernel": "k_project_f64 (plain FP64, one thread per configuration)"}


EXT_N = 16384   # extensions per step of the extend workload


def run_extend(args):
    """Batched ParallelConstrainedExtend (Alg. 2) on the dual arm: one step is
    one call extending EXT_N starts towards their targets; the metric counts
    the projected points that converged and passed validation (q_proj, the
    interpolated points and the bisection midpoints)."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_13323_gb300 import build as B
    B.build()
    from paper_2604_13323_gb300 import flops as FL
    from paper_2604_13323_gb300 import mcproj
    from paper_2604_13323_gb300 import workloads as W

    wl = W.extend_workload(n_ext=EXT_N, batch_seed=None if rank == 0 else 1010 + 1000 * rank)
    ex, p = wl.extra, wl.params
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles, device=local)
    stream = torch.cuda.current_stream(dev)
    # starts on the manifold (setup, untimed)
    q_s = P.project(torch.tensor(ex["raw_start"], dtype=torch.float32, device=dev), p)[0].contiguous()
    q_t = torch.tensor(ex["target"], dtype=torch.float32, device=dev)
    eps = torch.tensor(ex["eps"], dtype=torch.float32, device=dev)
    outs = (torch.empty_like(q_s), torch.empty(EXT_N, dtype=torch.uint8, device=dev),
            torch.empty(EXT_N, dtype=torch.int32, device=dev), torch.empty(EXT_N, dtype=torch.int32, device=dev))
    steps = torch.empty(EXT_N, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        P.extend(q_s, q_t, eps, p, ex["r"], ex["delta"], steps=steps, out=outs, stream=stream)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    with sampler:
        t0 = time.perf_counter()
        w = 0
        while w < args.warmup or (not args.profile and time.perf_counter() - t0 < 1.5):
            flush.zero_()
            step()
            w += 1
            if w % 16 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches0 = P.launches
        for s_ in range(args.steps):
            flush.zero_()
            evs[s_][0].record(stream)
            step()
            evs[s_][1].record(stream)
        torch.cuda.synchronize()
    launches = P.launches - launches0
    ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    st = outs[1].cpu().numpy()
    npts = outs[2].cpu().numpy()
    total_steps = float(steps.double().sum().item())
    pts = int(npts.sum())
    ms_max, c_total = aggregate_replicas(ms, pts, world, dev)
    value = c_total / (ms_max * 1e-3)
    # end to end: the step's inputs from pinned host memory, outputs back
    host_in = [t.cpu().pin_memory() for t in (q_s, q_t, eps)]
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    e2e_ms = []
    for s_ in range(0 if args.profile else args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for hi, di in zip(host_in, (q_s, q_t, eps)):
            di.copy_(hi, non_blocking=True)
        step()
        for ho, do in zip(host_out, outs):
            ho.copy_(do, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if s_ >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e = None
    if e2e_ms:
        e_ms, e_c = aggregate_replicas(sum(e2e_ms) / len(e2e_ms), int(host_out[2].numpy().sum()), world, dev)
        e2e = {"value": e_c / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in host_in),
               "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in host_out)}
    # roofline: Newton steps and evaluations of every projection the kernel ran
    fm = FL.FlopModel(wl.robot, wl.constraints)
    clk = sampler.summary()
    sm_max = clk.get("sm_max_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    peak32 = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    fp32 = total_steps * fm.iteration_alg
    ach = fp32 / (ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s", "frac": ach / peak32,
            "traffic": MEASURED_TRAFFIC.get((f"dual14_rel_extend_{EXT_N}", "k_extend")),
            "kernel": "k_extend (8 lanes per extension, four per warp: particles, interpolation, bisection)",
            "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock",
            "counted": "FP32 Newton steps of all projections x the step's flops (kernel-structure model without "
                       "sin/cos; evaluations, FP64 acceptance and collision checks not counted)",
            "newton_steps_per_step": total_steps}
    cpu = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.profile):
        from oracle import oracle as orc
        O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
        qs_np = q_s.double().cpu().numpy()
        t0 = time.perf_counter()
        done = pts_c = 0
        while time.perf_counter() - t0 < 10.0:
            sl = slice(done % EXT_N, done % EXT_N + 1024)
            res = O.extend(qs_np[:, sl], ex["target"][:, sl], ex["eps"][:, sl], p, ex["r"], ex["delta"])
            pts_c += int(res[2].sum())
            done += 1024
        dt = time.perf_counter() - t0
        cpu = {"value": pts_c / dt, "unit": UNIT, "cores": orc.default_threads(), "kind": "oracle",
               "sample": f"{done} extensions (chunks of 1024 of the bench batch), FP64, {dt:.1f} s wall"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"dual14_rel_extend_{EXT_N}", "extensions": EXT_N, "n": ex["n"],
                           "r": ex["r"], "delta": ex["delta"], "max_step": p.max_step, "tol": p.tol,
                           "cap": p.max_iters, "l2": "flushed between timed steps (512 MB write)",
                           "parallelism": f"replicas x{world}", "validated_points_per_step": pts,
                           "extensions_per_s": EXT_N * world / (ms_max * 1e-3),
                           "status_hist": np.bincount(st, minlength=9).tolist(),
                           "kernel_ms": {"extend": ms}},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        dist.destroy_process_group()


VJP_N = 65536          # projected dual-arm configurations per VJP step
PATHS, WAYPOINTS, SHORTEN_STEPS = 4096, 64, 100
SHORTEN_REF_PATHS = 64   # paths per step of the oracle's (reference arm) shortening


def run_adjoint(args, env=None, workload=None, sub=False):
    """The adjoint of the projection on the dual-arm closed chain: `vjp`
    times the VJP kernel v = g - J^T (J J^T)^{-1} J g on VJP_N projected
    configurations with g ~ N(0, 1) (one step = one call); `shorten` times
    gradient path shortening on the manifold (PATHS paths of WAYPOINTS
    waypoints, SHORTEN_STEPS steps of project -> length -> backward through
    the projection (VJP) -> clipped step; one bench step = one whole run) and
    reports the mean length reduction and the largest FP64 residual.  With
    `env` (a sub-record of the headline run) the process is set up already
    and the line is returned instead of printed; `sub` skips the e2e pass and
    the CPU baseline."""
    import torch
    import torch.distributed as dist

    standalone = env is None
    if standalone:
        world, rank, local, dev = init_dist()
        from paper_2604_13323_gb300 import build as B
        B.build()
    else:
        world, rank, local, dev = env["world"], env["rank"], env["local"], env["dev"]
    workload = workload or args.workload
    from paper_2604_13323_gb300 import flops as FL
    from paper_2604_13323_gb300 import mcproj
    from paper_2604_13323_gb300 import shorten as SH
    from paper_2604_13323_gb300 import workloads as W

    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    vjp_mode = workload == "vjp"
    extra = {}
    if vjp_mode:
        wl = W.dual_arm_workload(total=10, n_random=VJP_N, batch_seed=1011 + 1000 * rank)
        p = wl.params
        P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles, device=local)
        q_star = P.project(torch.tensor(wl.q, dtype=torch.float32, device=dev), p)[0].contiguous()  # setup
        g = torch.tensor(np.random.default_rng(1012 + 1000 * rank).standard_normal((14, VJP_N)),
                         dtype=torch.float32, device=dev)
        v = torch.empty_like(g)
        vf = torch.empty(VJP_N, dtype=torch.uint8, device=dev)

        def step():
            P.vjp(q_star, g, out=v, flags=vf, stream=stream)
        units_per_step = VJP_N
        unit, metric = "VJPs/s", "vector-Jacobian products/sec at q* (dual-arm closed chain, 1 GB300)"
        name = f"dual14_rel_vjp_{VJP_N}"
    else:
        pw = W.path_workload(n_paths=PATHS, n_way=WAYPOINTS)
        wl = pw["workload"]
        p = wl.params
        P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles, device=local)
        Q0 = SH.initial_paths(P, pw["qa"], pw["qb"], pw["noise"], p)   # setup
        # launch shape of the waypoints' projection: autotuned (setup, untimed)
        # on the waypoints one descent step moves off the manifold
        Q1 = P.project(Q0, p)[0]
        _, g1 = P.path_length_grad(Q1, PATHS, WAYPOINTS)
        P.path_step(Q1, P.vjp(Q1, g1)[0], PATHS, WAYPOINTS, 0.1, 0.05)
        shorten_tuning = dict(zip(("tpb", "blocks_per_sm", "chunk", "fuse_check", "threads_per_config"),
                                  P.autotune(Q1, p)))
        stats = {}

        def step():   # the graph-captured descent (the autograd one computes the same, more slowly)
            _, st = SH.shorten_paths_graph(P, Q0, PATHS, WAYPOINTS, p, SHORTEN_STEPS)
            stats.update(st)
        units_per_step = PATHS * WAYPOINTS * SHORTEN_STEPS
        unit, metric = "waypoint-steps/s", "path-shortening waypoint steps/sec on the manifold (dual arm, 1 GB300)"
        name = f"dual14_rel_shorten_{PATHS}x{WAYPOINTS}x{SHORTEN_STEPS}"
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    with sampler:
        t0 = time.perf_counter()
        w = 0
        while w < args.warmup or (not args.profile and time.perf_counter() - t0 < 1.5):
            flush.zero_()
            step()
            w += 1
            if w % 16 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches0 = P.launches
        for s_ in range(args.steps):
            flush.zero_()
            evs[s_][0].record(stream)
            step()
            evs[s_][1].record(stream)
        torch.cuda.synchronize()
    launches = P.launches - launches0
    ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    ms_max, u_total = aggregate_replicas(ms, units_per_step, world, dev)
    value = u_total / (ms_max * 1e-3)
    fm = FL.FlopModel(wl.robot, wl.constraints)
    clk = sampler.summary()
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak32 = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    if vjp_mode:
        # one VJP evaluates F and J at q*, builds and factors J J^T, solves
        # twice (with the refinement) and forms g - J^T y: counted as one LM step
        ach = VJP_N * fm.iteration_alg / (ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s", "frac": ach / peak32,
                "traffic": None, "kernel": "k_vjp (thread per configuration, FP32 + FP64 re-solve below the pivot)",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock",
                "counted": "one LM step's FP32 flops per VJP (FK, F, J, Gram, Cholesky, two solves, J^T y; "
                           "kernel-structure model without sin/cos)"}
        vfl = vf.cpu().numpy()
        extra = {"vjp_flags_nonzero": float((vfl != 0).mean())}
    else:
        # one shortening step, its calls timed one by one (after the timed runs)
        Qs = Q0.clone()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        Qv = Qs.detach().requires_grad_(True)
        ev[0].record(stream)
        out = P.project(Qv.detach(), p)[0]
        ev[1].record(stream)
        length, grad = P.path_length_grad(out, PATHS, WAYPOINTS)
        ev[2].record(stream)
        vv, _ = P.vjp(out, grad)
        ev[3].record(stream)
        P.path_step(out, vv, PATHS, WAYPOINTS, 0.1, 0.05)
        ev[4].record(stream)
        torch.cuda.synchronize()
        parts = {k: ev[i].elapsed_time(ev[i + 1]) for i, k in
                 enumerate(("project", "path_length_grad", "vjp", "path_step"))}
        extra = {k: stats[k] for k in ("mean_length_reduction", "min_length_reduction", "max_resid",
                                       "converged_fraction", "mean_length_before", "mean_length_after")}
        extra["kernel_ms_one_step"] = parts
        # the dominant call: the projection of the waypoints (FP32 steps of the
        # shortened points, a few per step, counted from the final projection)
        it = P.project(Qs, p)[2].cpu().numpy()
        fp32, fp64f = fm.projection(it, sincos=False)
        ach = fp32 / (parts["project"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s", "frac": ach / peak32,
                "traffic": None,
                "kernel": ("k_project_pair" if shorten_tuning["threads_per_config"] == 2 else "k_project_f32")
                + " (the waypoints' re-projection in one shortening step)", "launch": shorten_tuning,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock",
                "counted": "FP32 Newton-step and evaluation flops (kernel-structure model without sin/cos) of "
                           "the final waypoints' projection"}
    e2e = None
    if vjp_mode and not (args.profile or sub):   # q* and g from pinned host memory, v back, one step at a time
        hq, hg = q_star.cpu().pin_memory(), g.cpu().pin_memory()
        hv = torch.empty(v.shape, dtype=v.dtype).pin_memory()
        e_ms = []
        for s_ in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            q_star.copy_(hq, non_blocking=True)
            g.copy_(hg, non_blocking=True)
            step()
            hv.copy_(v, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            if s_ >= args.warmup:
                e_ms.append(e0.elapsed_time(e1))
        e_max, _ = aggregate_replicas(sum(e_ms) / len(e_ms), 0, world, dev)
        e2e = {"value": units_per_step * world / (e_max * 1e-3), "unit": unit,
               "h2d_bytes_per_step": 2 * hq.numel() * 4, "d2h_bytes_per_step": hv.numel() * 4}
    cpu = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.profile or sub) and vjp_mode:
        from oracle import oracle as orc
        O = orc.Oracle(wl.robot, wl.constraints)
        qn = q_star.double().cpu().numpy()
        gn = g.double().cpu().numpy()
        vg = v.double().cpu().numpy()
        t0 = time.perf_counter()
        done = 0
        rel = None
        while time.perf_counter() - t0 < 10.0:
            sl = slice(done % VJP_N, done % VJP_N + 4096)
            vo, fo = O.vjp(qn[:, sl], gn[:, sl])
            if rel is None:
                ok = fo == 0
                rel = float((np.abs(vg[:, sl][:, ok] - vo[:, ok]).max(axis=0) /
                             np.maximum(np.abs(vo[:, ok]).max(axis=0), 1e-12)).max())
            done += 4096
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt, "unit": unit, "cores": orc.default_threads(), "kind": "oracle",
               "sample": f"{done} VJPs (chunks of 4096 of the bench batch), FP64, {dt:.1f} s wall",
               "parity_vs_gpu": {"configs": 4096, "max_rel_err": rel}}
    if rank == 0:
        line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": name, "l2": "flushed between timed steps (512 MB write)",
                           "parallelism": f"replicas x{world}", **extra},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        if standalone:
            print(json.dumps(line), flush=True)
    else:
        line = None
    P.close()
    if standalone and world > 1:
        dist.destroy_process_group()
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "extend":
        run_extend(args)
    elif args.workload in ("vjp", "shorten"):
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
