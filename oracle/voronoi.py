"""Detector weights from the sensor positions as periodic Voronoi cells
(oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

eq:disc_rec weights sensor m by h_m, the detector area around x_m, with
sum h_m = X^(d-1) (Sec. 2).  The sums are X- (and Y-) periodic, so the
natural cells are the Voronoi cells of the periodic sensor set:
  areas_2d(xy, X, Y)   cell areas on the torus X x Y (scipy's Voronoi of the
                       3 x 3 tiling of the points, as the library step);
  lengths_1d(x, X)     cell lengths on the circle X (half the gaps to the
                       two neighbours).
Gradients of the cell sizes with respect to the positions, for the chain
rule dL/dx_m += sum_k dL/dh_k dh_k/dx_m:
  areas_2d_grad        edge (m, k) of length l at distance d with midpoint p:
                       dA_m/dx_k = (l/d)(x_k - p), dA_m/dx_m = sum_k (l/d)(p - x_m);
  lengths_1d_grad      h_m = (x_right - x_left)/2.
Reading where the paper is silent: the paper derives h_m for its masks from
a point density (r^3, r^2); for arbitrary positions the Voronoi cell is the
area "around x_m" that it describes, with the periodic extension the sums
already have.
"""
from __future__ import annotations

import numpy as np


def _tiled(xy, X, Y):
    shifts = [(sx * X, sy * Y) for sx in (-1, 0, 1) for sy in (-1, 0, 1)]
    pts = np.concatenate([xy + np.array(s) for s in shifts])
    return pts, shifts.index((0.0, 0.0)) * xy.shape[0]


def _cells(xy, X, Y):
    from scipy.spatial import Voronoi
    xy = np.asarray(xy, dtype=np.float64)
    M = xy.shape[0]
    pts, off = _tiled(xy, X, Y)
    vor = Voronoi(pts)
    return vor, off, M


def _polygon(vor, idx):
    reg = vor.regions[vor.point_region[idx]]
    v = vor.vertices[reg]
    c = vor.points[idx]
    ang = np.arctan2(v[:, 1] - c[1], v[:, 0] - c[0])
    return v[np.argsort(ang)]


def areas_2d(xy, X, Y):
    vor, off, M = _cells(xy, X, Y)
    out = np.empty(M)
    for m in range(M):
        v = _polygon(vor, off + m)
        x, y = v[:, 0], v[:, 1]
        out[m] = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    return out


def areas_2d_grad(xy, X, Y, grad_h):
    """sum_k grad_h[k] dA_k/dx_m, shape (M, 2)."""
    vor, off, M = _cells(xy, X, Y)
    out = np.zeros((M, 2))
    for (a, b), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if -1 in rv:
            continue
        ia, ib = a % M, b % M
        # ridges between two images of the same sensor move with it
        if ia == ib:
            continue
        pa_, pb = vor.points[a], vor.points[b]
        v0, v1 = vor.vertices[rv[0]], vor.vertices[rv[1]]
        l = np.linalg.norm(v1 - v0)
        d = np.linalg.norm(pb - pa_)
        p = 0.5 * (v0 + v1)
        # each ridge appears once per pair of images; count it for the
        # central copy of each endpoint
        if off <= a < off + M:
            out[ia] += (l / d) * (p - pa_) * grad_h[ia] + (l / d) * (pa_ - p) * grad_h[ib]
        if off <= b < off + M:
            out[ib] += (l / d) * (p - pb) * grad_h[ib] + (l / d) * (pb - p) * grad_h[ia]
    return out


def lengths_1d(x, X):
    x = np.asarray(x, dtype=np.float64)
    o = np.argsort(x, kind="stable")
    xs = x[o]
    nxt = np.roll(xs, -1)
    nxt[-1] += X
    prv = np.roll(xs, 1)
    prv[0] -= X
    out = np.empty_like(x)
    out[o] = 0.5 * (nxt - prv)
    return out


def lengths_1d_grad(x, X, grad_h):
    x = np.asarray(x, dtype=np.float64)
    o = np.argsort(x, kind="stable")
    g = np.asarray(grad_h, dtype=np.float64)[o]
    out = np.empty_like(x)
    # h_k = (x_{k+1} - x_{k-1}) / 2: dh_{m-1}/dx_m = 1/2, dh_{m+1}/dx_m = -1/2
    out[o] = 0.5 * (np.roll(g, 1) - np.roll(g, -1))
    return out
