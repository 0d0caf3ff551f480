"""Pins of the oracle's quality measures (appendix): the correlation
coefficient against numpy.corrcoef and its invariances, the Tenenbaum
function against scipy's 2-D convolution with the Sobel operator and against
closed forms (ramps, constants)."""
import numpy as np
import pytest

from oracle import metrics

SOBEL = np.array([[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]])


def test_correlation_matches_numpy_and_invariances():
    rng = np.random.default_rng(0)
    a = rng.normal(size=(9, 7, 5))
    b = 0.3 * a + rng.normal(size=a.shape)
    r = metrics.correlation(a, b)
    assert abs(r - np.corrcoef(a.ravel(), b.ravel())[0, 1]) <= 1e-13
    assert abs(metrics.correlation(a, 4.0 * b + 2.0) - r) <= 1e-13   # affine invariance
    assert abs(metrics.correlation(a, -b) + r) <= 1e-13
    assert abs(metrics.correlation(a, a) - 1.0) <= 1e-14


def test_tenenbaum_matches_scipy_convolution():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    u = rng.normal(size=(11, 8))
    gx = signal.convolve2d(u, SOBEL, mode="valid")
    gy = signal.convolve2d(u, SOBEL.T, mode="valid")
    ref = np.sum(gx ** 2 + gy ** 2) / u.size
    assert abs(metrics.tenenbaum(u) - ref) <= 1e-12 * ref


def test_tenenbaum_closed_forms():
    n0, n1 = 6, 9
    i, j = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    # U = a i + b j: every interior Sobel response is 8 b (second axis) and 8 a (first)
    a, b = 0.7, -1.3
    u = a * i + b * j
    ref = (n0 - 2) * (n1 - 2) * ((8 * b) ** 2 + (8 * a) ** 2) / u.size
    assert abs(metrics.tenenbaum(u) - ref) <= 1e-12 * ref
    assert metrics.tenenbaum(np.full((5, 5), 3.0)) == 0.0
    # a stack of slices sums the slices' responses over N of the whole stack
    v = np.stack([u, 2 * u, np.zeros_like(u)], axis=2)
    assert abs(metrics.tenenbaum(v) - (1 + 4) * ref / 3) <= 1e-12 * ref
