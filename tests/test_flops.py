"""The algorithmic flop model behind the benchmark's roofline: the per-unit
counts the design notes state, and bounds that hold for any structure-aware
count (never more than the dense operation count, never less than the
multiply-adds every Newton step needs)."""
import numpy as np

from paper_2604_13323_gb300 import flops as F
from paper_2604_13323_gb300 import workloads as W


def models():
    return {"arm": F.FlopModel(W.arm_workload(n=4).robot, W.arm_workload(n=4).constraints),
            "dual": F.FlopModel(W.dual_arm_workload(total=10, n_random=4).robot,
                                W.dual_arm_workload(total=10, n_random=4).constraints),
            "humanoid": F.FlopModel(W.humanoid_workload(n=4).robot, W.humanoid_workload(n=4).constraints)}


def test_stated_counts():
    m = models()
    got = {k: (v.iteration, v.evaluation, v.acceptance, v.fk_positions()) for k, v in m.items()}
    assert got == {"arm": (447, 301, 280, 339), "dual": (2802, 823, 781, 678),
                   "humanoid": (13227, 3044, 2945, 1707)}


def test_counts_are_between_sparse_and_dense_bounds():
    for name, fm in models().items():
        d, k = fm.d, fm.k
        # dense: J J^T (k(k+1)/2 dot products of length d), Cholesky, solves, J^T y
        dense_linear = k * (k + 1) * d + k ** 3 + 4 * k * k + 2 * k * d
        # every step at least forms J^T y over one nonzero per row and solves a k x k system
        assert fm.iteration > fm.evaluation > 0, name
        assert fm.iteration - fm.evaluation < dense_linear + 60 * d * k, name
        assert fm.iteration - fm.evaluation > 2 * k + k * k, name
        assert 0 < fm.acceptance < fm.evaluation * 2, name


def test_projection_counts_scale_with_steps():
    fm = models()["dual"]
    it = np.array([0, 1, 5], dtype=np.uint8)
    fp32, fp64 = fm.projection(it)
    assert fp64 == 3 * fm.acceptance
    assert fp32 == 6 * fm.iteration + 3 * fm.evaluation
