"""Parity helpers built on the FP64 oracle (test infrastructure only: used by
tests/ and by the package smoke check).

The Newton projection of an underdetermined system is chaotic from some
starts: near-singular J J^T + lambda I gives huge steps, and the FP64 oracle
itself lands elsewhere after a perturbation of the start of a few FP32 ulps.
Such configurations still converge to a valid point of the manifold, but
*which* point is not a well-defined function of the start, so point-wise
parity is only asserted on the configurations that are stable under such
perturbations; validity (FP64 residual below tol) is asserted everywhere.

The perturbation is the rounding scale of the precision the compared path
computes in, applied as 8 random sign patterns.  FP32 path: 8 unit roundoffs
(8 * 2^-24 ~ 5e-7).  One FP32 Newton step carries rounding of several unit
roundoffs (the Gram entries sum d products, the Cholesky K rows, each iterate
is rounded to FP32), so the compared path's iterates behave like starts
perturbed at that scale; a start whose FP64 result moves by more than the
point bar under such a perturbation has no answer that the path could
reproduce to within the bar.  Plain FP64 path: 1e-14 (~90 unit roundoffs of
FP64): it differs from the oracle not by the rounding of the same operations
but by other ones (CUDA's sin / cos against libm's, FMA contraction, another
order of products along the chain).  The threshold is the point bar itself
(1e-4 rad for the FP32 path, 1e-8 for the plain FP64 one).
"""
import numpy as np

from . import oracle as orc


REL_FP32, REL_FP64 = 5e-7, 1e-14   # 8 unit roundoffs of FP32; ~90 of FP64


def eligible_mask(o, q0, tol, max_iters, lam, max_step=0.0, rel=REL_FP32, thr=1e-4, reps=8, seed=0, cyclic=False,
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
