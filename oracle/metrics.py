"""Image quality measures of the paper's appendix, in FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

correlation   rho(U1, U2) = Cov(U1, U2) / sqrt(Var(U1) Var(U2))  (eq:corrcoeff),
              over all elements, population moments.
tenenbaum     F = sum_{x,y} (g * U)^2 + (g^T * U)^2 with g the 3x3 Sobel
              operator (rows (-1 0 1), (-2 0 2), (-1 0 1)), normalised by N,
              the number of elements of U.

Readings where the appendix is silent: the convolution takes the pixels
where the 3x3 stencil lies inside the image (no padding); a volume
U[n0][n1][n2] is a stack of n2 images over its first two axes (a 2-D image
is the stack n2 = 1), summed, and N = n0 n1 n2.
"""
from __future__ import annotations

import numpy as np


def correlation(u1, u2):
    a = np.asarray(u1, dtype=np.float64).ravel()
    b = np.asarray(u2, dtype=np.float64).ravel()
    da, db = a - a.mean(), b - b.mean()
    return float(np.sum(da * db) / np.sqrt(np.sum(da * da) * np.sum(db * db)))


def _as_stack(u):
    u = np.asarray(u, dtype=np.float64)
    return u[:, :, None] if u.ndim == 2 else u


def sobel_pair(u):
    """(g * U, g^T * U) on the interior pixels of each image of the stack:
    the sums over the 3x3 neighbourhood written out, index (i, j) = pixel
    (i + 1, j + 1).  Convolution flips g; the squares below do not see the
    sign."""
    u = _as_stack(u)
    n0, n1 = u.shape[0], u.shape[1]
    c = lambda di, dj: u[1 + di:n0 - 1 + di, 1 + dj:n1 - 1 + dj]
    # g: derivative along the second axis, smoothing (1 2 1) along the first
    gx = (c(-1, 1) - c(-1, -1)) + 2 * (c(0, 1) - c(0, -1)) + (c(1, 1) - c(1, -1))
    # g^T: derivative along the first axis, smoothing along the second
    gy = (c(1, -1) - c(-1, -1)) + 2 * (c(1, 0) - c(-1, 0)) + (c(1, 1) - c(-1, 1))
    return gx, gy


def tenenbaum(u):
    u = np.asarray(u, dtype=np.float64)
    gx, gy = sobel_pair(u)
    return float(np.sum(gx * gx + gy * gy) / u.size)
