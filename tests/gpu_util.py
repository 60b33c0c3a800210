"""Helpers shared by the GPU parity tests (comparison of the CUDA path, called
through the C ABI, with the FP64 oracle on identical seeded inputs)."""
import numpy as np

from oracle import oracle as orc
from oracle import parity

# Acceptance bars (from the projection spec): converged configurations agree to
# 1e-4 rad in the infinity norm, the FP64 residual of every converged output is
# below tol, convergence flags agree on >= 99.9 % of configurations, collision
# verdicts agree exactly outside a 1e-5 m band around contact.
Q_TOL = 1e-4
FLAG_AGREE = 0.999
CONTACT_BAND = 1e-5
# the plain FP64 kernel against the FP64 oracle: both compute in FP64 but not
# the same operations -- CUDA's sin / cos against libm's (each within an ulp,
# not identical), FMA contraction, another order of the products along the
# chain -- so their difference behaves like a start perturbation of ~100 unit
# roundoffs (REL_FP64) rather than of a few; the point bar is 1e-8 rad
Q_TOL_FP64 = 1e-8


def f32_exact(q):
    """The FP32 start the GPU sees, as FP64, so both sides start identically."""
    return np.asarray(q, dtype=np.float32).astype(np.float64)


def eligible_mask(oracle, q0, params, rel=None, thr=None, reps=8, seed=0, stable_iters=False, stats=None):
    """Configurations whose projection is a well-defined function of the start
    at the compared path's precision (see oracle/parity.py): by default 8
    unit roundoffs of FP32 (FP64 for the plain FP64 path) against the point
    bar (Q_TOL, Q_TOL_FP64).  Returns (mask, oracle result)."""
    fp64 = getattr(params, "precision", 0) == 1
    if rel is None:
        rel = parity.REL_FP64 if fp64 else parity.REL_FP32
    if thr is None:
        thr = Q_TOL_FP64 if fp64 else Q_TOL
    return parity.eligible_mask(oracle, q0, params.tol, params.max_iters, params.lam, max_step=params.max_step,
                                rel=rel, thr=thr, reps=reps, seed=seed, cyclic=bool(getattr(params, "cyclic", False)),
                                stable_iters=stable_iters, stats=stats, alpha=getattr(params, "alpha", 1.0),
                                outer=bool(getattr(params, "outer", False)))


def compare_projection(gpu, ora, tol, q_tol=Q_TOL, flag_agree=FLAG_AGREE, oracle=None, sample_resid=256,
                       eligible=None, min_eligible=0.0, stable_only=False, overall_flag_agree=0.99,
                       max_recount=0.001, q_quantile=None):
    """gpu / ora: (q [d, n], flags, iters, resid) as numpy.  Flags are compared
    on every configuration, points on the eligible ones (all if None), and
    every converged GPU output must be a valid point of the manifold (FP64
    residual recomputed by the oracle below tol).  With `stable_only`, the
    flag bar and the iteration-count comparison apply to the eligible
    configurations (where the oracle's own flag and count survive a
    perturbation of the start), and all configurations must still agree on
    `overall_flag_agree` of the flags.  At most `max_recount` of the
    configurations may converge on both sides after step counts differing by
    more than one (their points are then only checked for validity).  With
    `q_quantile`, that quantile of the point errors (not the maximum) must be
    within q_tol.  Returns a stats dict."""
    qg, fg, ig, rg = gpu
    qo, fo, io, ro = ora
    cg = (fg & orc.CONVERGED) != 0
    co = (fo & orc.CONVERGED) != 0
    el = np.ones(cg.shape, bool) if eligible is None else eligible
    overall = float((cg == co).mean())
    agree = float((cg == co)[el].mean()) if stable_only and el.any() else overall
    if stable_only:
        assert overall >= overall_flag_agree, overall
    # Same number of steps: the same sequence of Newton iterates, compared at
    # q_tol.  Steps differing by one: the ||F|| < tol decision was taken on
    # either side of the boundary in different precisions; the points then
    # differ by one Newton step from a residual at the tolerance, at most
    # ||J(q*)^+|| tol = tol / sigma_min(J(q*)) (checked with the oracle's J).
    same_it = ig == io
    both = cg & co & el & same_it
    off_by_one = cg & co & el & (np.abs(ig.astype(np.int64) - io.astype(np.int64)) == 1)
    if oracle is not None:
        viol = []
        for i in np.flatnonzero(off_by_one):
            # rows of inactive bounded constraints are zero (and so is their
            # residual): the step lives in the span of the nonzero rows
            sv = np.linalg.svd(oracle.residual_jacobian(qo[:, i])[1], compute_uv=False)
            smin = sv[sv > 1e-12 * max(sv.max(), 1e-300)].min() if (sv > 0).any() else 1.0
            e = np.abs(qg[:, i] - qo[:, i]).max()
            if e > q_tol + 2.0 * tol / smin:
                viol.append((int(i), float(e), float(smin)))
        # a nonsmooth residual (bounded TSR, support hull) can switch its active
        # rows between the two iterates: there the bound holds at the quantile
        allowed = 0 if q_quantile is None else int((1.0 - q_quantile) * cg.size)
        assert len(viol) <= allowed, ("off-by-one points beyond the bound", viol[:5], len(viol), allowed)
    recount = int((cg & co & el & ~same_it & ~off_by_one).sum())
    assert recount <= max(1, int(max_recount * cg.size)), ("iteration counts differ", recount)
    err = np.abs(qg[:, both] - qo[:, both]).max(axis=0) if both.any() else np.zeros(0)
    stats = {"n": int(cg.size), "conv_gpu": float(cg.mean()), "conv_oracle": float(co.mean()), "flag_agree": agree,
             "q_err_max": float(err.max()) if err.size else 0.0,
             "q_err_p999": float(np.quantile(err, 0.999)) if err.size else 0.0,
             "resid_max": float(rg[cg].max()) if cg.any() else 0.0,
             "iters_equal": float(same_it[cg & co & (el if stable_only else True)].mean()) if (cg & co).any() else 1.0,
             "flag_agree_all": overall,
             "off_by_one": int(off_by_one.sum()),
             "eligible": float(el.mean())}
    assert stats["eligible"] >= min_eligible, stats
    assert agree >= flag_agree, stats
    if q_quantile is None:
        assert stats["q_err_max"] <= q_tol, stats
    else:
        assert (float(np.quantile(err, q_quantile)) if err.size else 0.0) <= q_tol, stats
    assert np.all(rg[cg] < tol), stats
    if oracle is not None and cg.any():
        # the reported FP64 residual is the residual of the returned configuration
        idx = np.flatnonzero(cg)[:: max(1, cg.sum() // sample_resid)]
        for i in idx:
            r = np.linalg.norm(oracle.residual(qg[:, i].astype(np.float64)))
            # both sides evaluate the same FP32 configuration in FP64: rounding only
            assert abs(r - rg[i]) <= 1e-12 * max(1.0, r), (i, r, rg[i])
            assert r < tol
    return stats


def compare_collision(hit_gpu, hit_oracle, margin_oracle, band=CONTACT_BAND):
    ok = margin_oracle >= band
    mism = (hit_gpu != hit_oracle) & ok
    assert not mism.any(), (np.flatnonzero(mism)[:10], int(mism.sum()))
    return {"n": int(hit_gpu.size), "excluded": int((~ok).sum()), "collide_frac": float(hit_oracle.mean())}
