"""Pins of the oracle's periodic Voronoi weights: the cells tile the torus,
lattice cells are pitch x pitch, cell areas agree with brute-force nearest
generator counts on a raster, and the gradients with FP64 central
differences."""
import numpy as np
import pytest

pytest.importorskip("scipy.spatial")
from oracle import voronoi


def rand_xy(M, X, Y, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-X / 2, X / 2, M), rng.uniform(-Y / 2, Y / 2, M)], 1)


def test_cells_tile_the_torus_and_lattice_cells():
    X, Y = 1.3e-3, 0.9e-3
    xy = rand_xy(40, X, Y, 0)
    assert abs(voronoi.areas_2d(xy, X, Y).sum() - X * Y) <= 1e-12 * X * Y
    nx, ny = 6, 5
    g = np.array([((i + 0.3) * X / nx - X / 2, (j + 0.1) * Y / ny - Y / 2) for i in range(nx) for j in range(ny)])
    g += 1e-12 * np.random.default_rng(1).normal(size=g.shape)   # break the cocircular ties
    assert np.allclose(voronoi.areas_2d(g, X, Y), X * Y / (nx * ny), rtol=1e-6)
    x = np.random.default_rng(2).uniform(-X / 2, X / 2, 17)
    assert abs(voronoi.lengths_1d(x, X).sum() - X) <= 1e-15


def test_areas_match_raster_nearest_counts():
    X, Y = 1.0, 0.8
    xy = rand_xy(12, X, Y, 3)
    n = 800
    gx = (np.arange(n) + 0.5) / n * X - X / 2
    gy = (np.arange(n) + 0.5) / n * Y - Y / 2
    P = np.stack(np.meshgrid(gx, gy, indexing="ij"), -1).reshape(-1, 2)
    d = P[:, None, :] - xy[None, :, :]
    d[..., 0] -= X * np.round(d[..., 0] / X)
    d[..., 1] -= Y * np.round(d[..., 1] / Y)
    owner = np.argmin((d ** 2).sum(-1), axis=1)
    counts = np.bincount(owner, minlength=xy.shape[0]) * (X * Y / n ** 2)
    assert np.allclose(voronoi.areas_2d(xy, X, Y), counts, rtol=0.02)


def test_area_gradient_matches_finite_differences():
    X, Y = 1.0, 1.0
    xy = rand_xy(15, X, Y, 4)
    gh = np.random.default_rng(5).normal(size=15)
    got = voronoi.areas_2d_grad(xy, X, Y, gh)
    eps = 1e-7
    fd = np.zeros_like(xy)
    for m in range(15):
        for c in range(2):
            p, q = xy.copy(), xy.copy()
            p[m, c] += eps
            q[m, c] -= eps
            fd[m, c] = (gh @ voronoi.areas_2d(p, X, Y) - gh @ voronoi.areas_2d(q, X, Y)) / (2 * eps)
    assert np.linalg.norm(got - fd) <= 1e-6 * np.linalg.norm(fd)


def test_length_gradient_matches_finite_differences():
    X = 1.0
    x = np.random.default_rng(6).uniform(-X / 2, X / 2, 11)
    gh = np.random.default_rng(7).normal(size=11)
    got = voronoi.lengths_1d_grad(x, X, gh)
    eps = 1e-7
    fd = np.array([(gh @ voronoi.lengths_1d(x + eps * (np.arange(11) == m), X)
                    - gh @ voronoi.lengths_1d(x - eps * (np.arange(11) == m), X)) / (2 * eps) for m in range(11)])
    assert np.allclose(got, fd, atol=1e-7)
