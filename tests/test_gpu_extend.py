"""Batched ParallelConstrainedExtend (Algorithm 2), CUDA path (C ABI) against
the FP64 oracle's statement of the algorithm."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc  # noqa: E402
from paper_2604_13323_gb300 import workloads as W  # noqa: E402
from tests.gpu_util import f32_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcproj():
    from paper_2604_13323_gb300 import build, mcproj as m
    build.build()
    m.load_library()
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _unit(v):
    return v / np.linalg.norm(v)


def test_extend_on_sphere_matches_oracle_and_geometry(mcproj):
    """On the unit sphere with lambda = 0 each projection is the radial one in
    a single step: q_proj is the normalised winning particle (index 0) and the
    outcome and point count follow from the arc geometry (the oracle pins);
    the GPU must agree with the oracle on all of it."""
    wl = W.sphere_workload(n_pairs=2)
    p = W.Params(tol=1e-6, max_iters=20, lam=0.0)
    rng = np.random.default_rng(61)
    m, n = 512, 8
    qs = f32_exact(np.stack([_unit(rng.standard_normal(3)) for _ in range(m)], 1))
    qt = f32_exact(np.stack([_unit(rng.standard_normal(3)) for _ in range(m)], 1) * 1.3)
    eps = f32_exact(0.03 * rng.standard_normal((n, m)))
    obs = W.Obstacles(spheres=np.array([[0.0, 0.0, 1.0, 0.3], [0.8, 0.6, 0.0, 0.2]]), aabbs=np.zeros((0, 6)))
    O = orc.Oracle(wl.robot, wl.constraints, obs)
    P = mcproj.Projector(wl.robot, wl.constraints, obs)
    qo, so, no, wo = O.extend(qs, qt, eps, p, 0.5, 0.03)
    qg, sg, ng, wg = (t.cpu().numpy() for t in P.extend(dev(qs), dev(qt), dev(eps), p, 0.5, 0.03))
    assert (sg == so).mean() > 0.99, np.bincount(so * 10 + sg)
    same = sg == so
    assert np.array_equal(wg[same], wo[same])
    ok = same & (so == orc.EXT_OK)
    assert ok.mean() > 0.3
    assert (ng[ok] == no[ok]).mean() > 0.99
    np.testing.assert_allclose(qg[:, wo >= 0], qo[:, wo >= 0], atol=2e-6)
    assert len(set(so.tolist())) >= 3   # several outcomes exercised


@pytest.mark.parametrize("n,n_ext", [(8, 2048), (3, 1023), (12, 1021)])
def test_extend_dual_arm_parity(mcproj, n, n_ext):
    """n = 8 and n = 3 run four extensions per warp (groups of 8 lanes, the
    latter with idle lanes in each group and a partial last claim); n = 12
    runs one extension per warp."""
    wl = W.extend_workload(n_ext=n_ext, n=n)
    ex = wl.extra
    p = wl.params
    O = orc.Oracle(wl.robot, wl.constraints, wl.obstacles)
    qs = O.project(ex["raw_start"], p.tol, p.max_iters, p.lam)[0]
    qs, qt, eps = f32_exact(qs), f32_exact(ex["target"]), f32_exact(ex["eps"])
    qo, so, no, wo = O.extend(qs, qt, eps, p, ex["r"], ex["delta"])
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    qg, sg, ng, wg = (t.cpu().numpy() for t in P.extend(dev(qs), dev(qt), dev(eps), p, ex["r"], ex["delta"]))
    agree = (sg == so).mean()
    assert agree > 0.98, (agree, np.bincount(so, minlength=9), np.bincount(sg, minlength=9))
    both_ok = (sg == orc.EXT_OK) & (so == orc.EXT_OK)
    assert both_ok.mean() > 0.3
    assert (wg[both_ok] == wo[both_ok]).mean() > 0.99
    same = both_ok & (wg == wo)
    err = np.abs(qg[:, same] - qo[:, same]).max(axis=0)
    assert np.quantile(err, 0.999) <= 1e-4, np.quantile(err, [0.5, 0.99, 1.0])
    assert (ng[same] == no[same]).mean() > 0.98
    # every returned q_proj of a successful extension is on the manifold (FP64)
    for i in np.flatnonzero(sg == orc.EXT_OK)[::37]:
        assert np.linalg.norm(O.residual(qg[:, i].astype(np.float64))) < p.tol


def test_extend_arguments(mcproj):
    wl = W.extend_workload(n_ext=4)
    P = mcproj.Projector(wl.robot, wl.constraints, wl.obstacles)
    q = dev(wl.extra["raw_start"])
    e = dev(wl.extra["eps"])
    for bad in ({"r": -1.0, "delta": 0.02}, {"r": 0.3, "delta": 0.0}):
        with pytest.raises(mcproj.MCPError):
            P.extend(q, q, e, wl.params, bad["r"], bad["delta"])
    with pytest.raises(mcproj.MCPError):
        P.extend(q, q, torch.zeros((33, 4), device="cuda"), wl.params, 0.3, 0.02)
    cyc = W.Params(tol=1e-5, max_iters=30, lam=1e-6, cyclic=True)
    with pytest.raises(mcproj.MCPError):
        P.extend(q, q, e, cyc, 0.3, 0.02)
    # q_t == q_s: degenerate, nothing projected
    qp, st, npts, win = P.extend(q, q, e, wl.params, 0.3, 0.02)
    assert (st.cpu().numpy() == mcproj.EXT_DEGENERATE).all() and (npts.cpu().numpy() == 0).all()
    hw = W.humanoid_workload(n=4)
    H = mcproj.Projector(hw.robot, hw.constraints, hw.obstacles)
    hq = dev(hw.q)
    with pytest.raises(mcproj.MCPError):
        H.extend(hq, hq, torch.zeros((4, 4), device="cuda"), hw.params, 0.3, 0.02)
