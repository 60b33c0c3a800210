"""The synthetic workloads follow their stated recipe (shapes, sizes, value
ranges and structure of the paper's problems): these tests pin the recipe, so
a change to a generator that would silently change what the benchmark
measures fails here."""
import inspect

import numpy as np

from paper_2604_13323_gb300 import workloads as W


def test_sphere_recipe():
    wl = W.sphere_workload()
    pts = W.segment_points(wl.segments)
    assert wl.segments.length.shape[0] == 1024
    assert 27_000 < pts.shape[1] < 30_000          # inclusive 0.05 steps along the chords
    assert np.allclose(np.linalg.norm(wl.segments.start, axis=0), 1.0)
    o = wl.obstacles.spheres
    assert o.shape == (10, 4) and (np.abs(o[:, :3]) <= 1.5).all() and ((o[:, 3] > 0.05) & (o[:, 3] < 0.2)).all()
    assert wl.params.precision == W.PREC_FP64 and wl.params.tol == 1e-8 and wl.params.max_iters == 50
    assert wl.params.lam == 0.0


def test_arm_recipe():
    wl = W.arm_workload(n=4096)
    assert inspect.signature(W.arm_workload).parameters["n"].default == 65536
    q = wl.q
    assert q.shape == (7, 4096) and (np.abs(q) <= 2.8).all()
    rb = wl.robot
    assert np.allclose(rb.lower, -2.8) and np.allclose(rb.upper, 2.8)
    counts = np.bincount(np.asarray(rb.sphere_link), minlength=7)
    assert sorted(counts.tolist(), reverse=True) == [9, 9, 9, 9, 8, 8, 8]
    r = np.asarray(rb.sphere)[:, 3]
    assert ((r >= 0.03) & (r <= 0.08)).all()
    o = wl.obstacles.spheres
    assert o.shape == (64, 4)
    assert (o[:, 0] >= 0.2).all() and (o[:, 0] <= 1.7).all() and (np.abs(o[:, 1]) <= 0.75).all()
    assert (o[:, 2] >= 0.0).all() and (o[:, 2] <= 1.5).all() and ((o[:, 3] > 0.05) & (o[:, 3] < 0.2)).all()
    p = wl.params
    assert p.tol == 1e-5 and p.max_iters == 30 and p.lam == 1e-6


def test_dual_arm_recipe():
    wl = W.dual_arm_workload()
    ln = wl.extra["lengths"]
    assert ln.min() >= 2 and ln.max() <= 200
    assert ln.sum() >= 262_144 and ln[:-1].sum() < 262_144      # lengths drawn until the total is reached
    assert int(ln.sum()) == 262_240 and ln.shape[0] == 2644
    assert np.allclose(np.linalg.norm(wl.extra["raw_dir"], axis=0), 1.0)
    assert wl.extra["step"] == 0.05
    rb = wl.robot
    assert rb.parent.shape[0] == 14 and len(rb.sphere_link) == 120
    assert wl.obstacles.spheres.shape == (128, 4)
    p = wl.params
    assert p.tol == 1e-5 and p.max_iters == 30 and p.lam == 1e-6 and p.pivot_fp64 == 1e-7


def test_humanoid_recipe():
    wl = W.humanoid_workload(n=2048)
    assert inspect.signature(W.humanoid_workload).parameters["n"].default == 1_048_576
    rb = wl.robot
    assert rb.parent.shape[0] == 36 and len(rb.sphere_link) == 150
    assert (np.asarray(rb.type)[:3] == 1).all() and (np.asarray(rb.type)[3:] == 0).all()   # 3P + 33R
    assert sum(W.CONSTRAINT_DIM[c.kind] for c in wl.constraints) == 20
    assert wl.obstacles.spheres.shape == (200, 4) and wl.obstacles.aabbs.shape == (6, 6)
    p = wl.params
    assert p.tol == 1e-5 and p.max_iters == 40 and p.lam == 1e-6
    # starts: nominal stance + N(0, 0.3^2) on rotations, N(0, 0.05^2) m on the base translations
    dev = wl.q - wl.q.mean(axis=1, keepdims=True)
    assert np.allclose(dev[:3].std(axis=1), 0.05, rtol=0.1) and np.allclose(dev[3:].std(axis=1), 0.3, rtol=0.1)


def test_vjp_and_path_recipes():
    g = np.random.default_rng(1012).standard_normal((14, 65536))
    assert abs(g.std() - 1.0) < 0.01
    pw = W.path_workload(n_paths=16, n_way=64)
    assert pw["qa"].shape == (14, 16) and pw["qb"].shape == (14, 16)
