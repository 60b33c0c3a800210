"""Parity helpers built on the FP64 oracle (test infrastructure only: used by
tests/ and by the package smoke check).

The Newton projection of an underdetermined system is chaotic from some
starts: near-singular J J^T + lambda I gives huge steps, and the FP64 oracle
itself lands elsewhere after a perturbation of the start of a few FP32 ulps.
Such configurations still converge to a valid point of the manifold, but
*which* point is not a well-defined function of the start, so point-wise
parity is only asserted on the configurations that are stable under such
perturbations; validity (FP64 residual below tol) is asserted everywhere.
"""
import numpy as np

from . import oracle as orc


def eligible_mask(o, q0, tol, max_iters, lam, max_step=0.0, rel=1e-6, thr=1e-5, reps=2, seed=0, cyclic=False,
                  stable_iters=False, stats=None, alpha=1.0, outer=False):
    """(mask, oracle result): mask[i] is True when `reps` random relative
    perturbations of size `rel` of start i move the oracle's result by <= thr
    and do not change its convergence flag (nor, with `stable_iters`, its
    number of iterations: active-set changes of bounded constraints and slow
    alternating projections can move the step at which ||F|| < tol is first
    met while the point barely moves).  `stats` (a dict), if given, receives
    how often the oracle disagrees with itself under those perturbations:
    the fraction of flipped convergence flags and of changed step counts,
    the scale of any other implementation's disagreement on the workload."""
    rng = np.random.default_rng(seed)
    kw = dict(max_step=max_step, cyclic=cyclic, alpha=alpha, outer=outer)
    base = o.project(q0, tol, max_iters, lam, **kw)
    dev_max = np.zeros(q0.shape[1])
    flips = np.zeros(q0.shape[1], bool)
    recount = np.zeros(q0.shape[1], bool)
    for _ in range(reps):
        q1 = q0 * (1.0 + rel * rng.choice([-1.0, 1.0], size=q0.shape))
        other = o.project(q1, tol, max_iters, lam, **kw)
        dev_max = np.maximum(dev_max, np.abs(base[0] - other[0]).max(axis=0))
        flips |= (base[1] & orc.CONVERGED) != (other[1] & orc.CONVERGED)
        recount |= base[2] != other[2]
    dev_max[flips] = np.inf
    if stable_iters:
        dev_max[recount] = np.inf
    if stats is not None:
        stats.update(self_flip_rate=float(flips.mean()), self_recount_rate=float(recount.mean()))
    return dev_max <= thr, base
