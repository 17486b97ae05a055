"""Pins for the oracle's gradient, divergence, TV and shrinkage."""
import numpy as np
import pytest

from oracle import tv


def test_div_is_negative_transpose_of_grad():
    rng = np.random.default_rng(20)
    u = rng.standard_normal((5, 7, 6))
    p = rng.standard_normal((3, 5, 7, 6))
    assert abs(np.vdot(tv.grad(u), p) + np.vdot(u, tv.div(p))) < 1e-12 * 100


def test_grad_of_ramps():
    x = np.arange(5.0)[:, None, None] * np.ones((5, 4, 3))
    g = tv.grad(2.0 * x)
    assert np.all(g[0, :4] == 2.0) and np.all(g[0, 4] == 0.0)   # Neumann end
    assert np.all(g[1] == 0.0) and np.all(g[2] == 0.0)
    z = np.arange(4.0)[None, :, None] * np.ones((5, 4, 3))
    g = tv.grad(z)
    assert np.all(g[1, :, :3] == 1.0) and np.all(g[1, :, 3] == 0.0)


def test_div_matches_explicit_matrix():
    # build grad as an explicit matrix from its definition and compare div
    shape = (3, 4, 2)
    N = int(np.prod(shape))
    D = np.zeros((3 * N, N))
    idx = np.arange(N).reshape(shape)
    for a in range(3):
        for i in np.ndindex(shape):
            if i[a] + 1 < shape[a]:
                j = list(i)
                j[a] += 1
                D[a * N + idx[i], idx[tuple(j)]] += 1.0
                D[a * N + idx[i], idx[i]] -= 1.0
    rng = np.random.default_rng(21)
    p = rng.standard_normal((3,) + shape)
    assert np.allclose(tv.div(p).ravel(), -(D.T @ p.ravel()), atol=1e-13)
    u = rng.standard_normal(shape)
    assert np.allclose(tv.grad(u).ravel(), D @ u.ravel(), atol=1e-13)


def test_tv_of_step_is_interface_area():
    u = np.zeros((6, 5, 4))
    u[:3] = 2.0                         # jump of 2 across one x-interface
    assert tv.tv(u) == pytest.approx(2.0 * 5 * 4)
    v = np.zeros((6, 5, 4))
    v[:, :2, :] = 1.0                   # jump of 1 across one z-interface
    assert tv.tv(v) == pytest.approx(6 * 4)


def test_tv_isotropic_diagonal_edge():
    u = np.zeros((2, 1, 2))
    u[0, 0, 0] = 1.0                    # grad at (0,0,0) = (-1, 0, -1)
    assert tv.tv(u) == pytest.approx(np.sqrt(2.0))


def test_shrink_closed_form():
    z = np.array([3.0, 4.0, 0.0]).reshape(3, 1, 1, 1)
    assert np.allclose(tv.shrink_iso(z, 1.0).ravel(), [2.4, 3.2, 0.0])
    assert np.all(tv.shrink_iso(z, 6.0) == 0.0)
    assert np.all(tv.shrink_iso(np.zeros((3, 1, 1, 1)), 1.0) == 0.0)


def test_shrink_is_the_proximal_map():
    # argmin_x k|x| + 1/2 |x - z|^2 by brute force over a fine grid around z
    z = np.array([0.7, -0.4, 0.2])
    k = 0.3
    best = tv.shrink_iso(z.reshape(3, 1, 1, 1), k).ravel()
    rng = np.random.default_rng(22)
    trial = best + rng.normal(scale=0.05, size=(20000, 3))
    f = lambda x: k * np.linalg.norm(x, axis=-1) + 0.5 * np.sum((x - z) ** 2, axis=-1)
    assert f(best[None])[0] <= f(trial).min() + 1e-12
