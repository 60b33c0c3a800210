"""Pins of the oracle's gradient path shortening on the manifold.

The oracle shortens waypoint paths by gradient descent on their total length
L = sum_w |q_{w+1} - q_w|: project every waypoint, take dL/dq at the
projected path, pull it back through the projection (the VJP
g - J^T (J J^T)^{-1} J g, the tangent component), step the interior
waypoints by -eta times it (the largest joint move clipped to max_step) and
project again.  These tests fix each part by something other than the oracle
itself: finite differences of the length, closed forms in free space
(a straight segment is the shortest path; descent reaches |b - a|) and on the
unit sphere (an evenly spaced great-circle polygon is stationary: its length
gradient is radial, so the tangent pull-back vanishes).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_13323_gb300 import workloads as W


def _sphere():
    wl = W.sphere_workload(n_pairs=2)
    return wl, orc.Oracle(wl.robot, wl.constraints)


def test_path_length_and_gradient_match_finite_differences():
    rng = np.random.default_rng(0)
    d, n_paths, n_way = 5, 3, 7
    Q = rng.standard_normal((d, n_paths * n_way))
    Q[:, 4] = Q[:, 3]                      # one zero-length edge: it adds nothing to L or to dL/dq
    L, G = orc.path_length_grad(Q, n_paths, n_way)
    E = Q.reshape(d, n_paths, n_way)
    np.testing.assert_allclose(L, np.linalg.norm(np.diff(E, axis=2), axis=0).sum(1), rtol=1e-14)
    h = 1e-6
    for col in range(Q.shape[1]):
        if col in (3, 4):                  # the length is not differentiable across the zero edge
            continue
        for j in range(d):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[j, col] += h
            Qm[j, col] -= h
            p = col // n_way
            fd = (orc.path_length_grad(Qp, n_paths, n_way)[0][p] - orc.path_length_grad(Qm, n_paths, n_way)[0][p]) / (2 * h)
            assert abs(fd - G[j, col]) < 1e-8, (col, j, fd, G[j, col])


def test_straight_path_is_stationary_in_free_space():
    """A straight segment with monotone waypoints: the interior gradient is
    zero, so shortening without constraints leaves the path where it is.
    (The straight path is a minimum whose curvature across the path is
    1/|e_w| + 1/|e_{w+1}|: descent is stable for eta below 2 over that, which
    the spacing here (>= 0.1 |b - a|) and eta = 0.01 respect; above it,
    rounding noise grows into a zig-zag that only the clip bounds.)"""
    rng = np.random.default_rng(1)
    wl, _ = _sphere()
    free = orc.Oracle(wl.robot, [])
    a, b = rng.standard_normal(3), rng.standard_normal(3)
    t = np.linspace(0.0, 1.0, 9)
    t[1:-1] += rng.uniform(-0.02, 0.02, 7)
    Q = a[:, None] + (b - a)[:, None] * t[None, :]
    _, G = orc.path_length_grad(Q, 1, t.size)
    assert np.abs(G[:, 1:-1]).max() < 1e-14
    Qf, fl, _, Ls = free.shorten(Q, 1, t.size, wl.params, steps=20, eta=0.01, max_step=0.05)
    np.testing.assert_allclose(Qf, Q, atol=1e-14)
    np.testing.assert_allclose(Ls[0], np.linalg.norm(b - a), rtol=1e-14)


def test_free_space_descent_reaches_the_straight_segment():
    """Without constraints the projection is the identity and the VJP is g:
    gradient descent on the length of a noisy path converges to |b - a|."""
    rng = np.random.default_rng(2)
    wl, _ = _sphere()
    free = orc.Oracle(wl.robot, [])
    n_paths, n_way = 4, 12
    A, B = rng.standard_normal((3, n_paths)), rng.standard_normal((3, n_paths))
    t = np.linspace(0, 1, n_way)
    Q = A[:, :, None] + (B - A)[:, :, None] * t
    Q[:, :, 1:-1] += 0.1 * rng.standard_normal((3, n_paths, n_way - 2))
    Qf, _, _, Ls = free.shorten(Q.reshape(3, -1), n_paths, n_way, wl.params, steps=2000, eta=0.01, max_step=0.0)
    np.testing.assert_allclose(Ls[:, 1], np.linalg.norm(Q[:, :, -1] - Q[:, :, 0], axis=0), rtol=1e-8)
    assert (Ls[:, 1] < Ls[:, 0]).all()
    # the endpoints never move
    Qf = Qf.reshape(3, n_paths, n_way)
    np.testing.assert_array_equal(Qf[:, :, 0], Q[:, :, 0])
    np.testing.assert_array_equal(Qf[:, :, -1], Q[:, :, -1])


def test_great_circle_polygon_is_stationary_on_the_sphere():
    """Evenly spaced points of a great-circle arc: dL/dq at an interior point
    is a multiple of the point itself (radial), the tangent pull-back
    g - (g . q) q vanishes, and shortening leaves the path in place."""
    wl, O = _sphere()
    rng = np.random.default_rng(3)
    n_way = 10
    a = rng.standard_normal(3)
    a /= np.linalg.norm(a)
    u = rng.standard_normal(3)
    u -= (u @ a) * a
    u /= np.linalg.norm(u)
    th = np.linspace(0.0, 1.7, n_way)
    Q = np.cos(th)[None, :] * a[:, None] + np.sin(th)[None, :] * u[:, None]
    _, G = orc.path_length_grad(Q, 1, n_way)
    v, fl = O.vjp(Q, G)
    assert (fl == 0).all()
    assert np.abs(v[:, 1:-1]).max() < 1e-14
    Qf, fl, r, Ls = O.shorten(Q, 1, n_way, wl.params, steps=10, eta=0.1, max_step=0.05)
    np.testing.assert_allclose(Qf, Q, atol=1e-14)
    np.testing.assert_allclose(Ls[0, 1], (n_way - 1) * 2 * np.sin(1.7 / (2 * (n_way - 1))), rtol=1e-14)


def test_one_step_is_the_clipped_tangent_step():
    """One descent step on the sphere from a path already on it: each
    interior waypoint moves by -eta (g - (g . q) q) (the projector's closed
    form on the sphere), its largest joint move clipped to max_step, and is
    then projected back (normalised)."""
    wl, O = _sphere()
    rng = np.random.default_rng(4)
    n_way = 9
    Q = rng.standard_normal((3, n_way))
    Q /= np.linalg.norm(Q, axis=0)
    for eta, max_step in ((0.01, 0.0), (0.5, 0.05)):
        _, G = orc.path_length_grad(Q, 1, n_way)
        V = G - (G * Q).sum(0) * Q
        m = np.abs(eta * V).max(axis=0)
        sc = np.where((max_step > 0) & (m > max_step), max_step / np.where(m > 0, m, 1.0), 1.0)
        Q1 = Q - sc * eta * V
        Q1[:, [0, -1]] = Q[:, [0, -1]]
        Q1 /= np.linalg.norm(Q1, axis=0)
        Qf, fl, _, _ = O.shorten(Q, 1, n_way, wl.params, steps=1, eta=eta, max_step=max_step)
        assert (fl & orc.CONVERGED).all()
        np.testing.assert_allclose(Qf, Q1, atol=1e-12)
        if max_step > 0:
            assert (sc[1:-1] < 1).any()     # the clip was exercised


@pytest.mark.parametrize("eta", [0.002, 0.01])
def test_small_steps_shorten_on_the_sphere(eta):
    """Descent with small steps lowers the length of every noisy path on the
    sphere and keeps every waypoint on it."""
    wl, O = _sphere()
    rng = np.random.default_rng(5)
    n_paths, n_way = 6, 16
    A = rng.standard_normal((3, n_paths))
    B = rng.standard_normal((3, n_paths))
    A /= np.linalg.norm(A, axis=0)
    B /= np.linalg.norm(B, axis=0)
    t = np.linspace(0, 1, n_way)
    Q = A[:, :, None] + (B - A)[:, :, None] * t
    Q[:, :, 1:-1] += 0.05 * rng.standard_normal((3, n_paths, n_way - 2))
    Q0 = O.project_params(Q.reshape(3, -1), wl.params)[0]
    prev = orc.path_length_grad(Q0, n_paths, n_way)[0]
    for steps in (5, 20):
        Qf, fl, r, Ls = O.shorten(Q0, n_paths, n_way, wl.params, steps=steps, eta=eta, max_step=0.0)
        assert (Ls[:, 1] < prev).all()
        prev = Ls[:, 1]
        assert (fl & orc.CONVERGED).all() and r.max() < wl.params.tol
