"""Sensor masks that concentrate acquisition points around a centre of
interest (Sec. 4 of the paper and its appendix on the equi-steradian
arrangement), and their density weights h_m.

Host-side set-up only: the positions and weights feed an ordinary plan.

equisteradian_mask -- 3-D: points equally spaced in solid angle seen from a
    centre of interest at depth r0 below the middle of a square grid,
    projected onto the sensor plane and snapped to grid nodes; weights
    h_m ~ r^3 (r: distance to the centre of interest).
equiangular_mask -- 2-D: points on a line at equal angular steps seen from
    the centre of interest; weights h_m ~ r^2.

Readings where the paper's description is garbled or silent:
* the spherical cap is the one whose projection is the disc inscribed in the
  grid (polar angle up to atan(L/2 / r0), L the grid side);
* slice 1 is a single point on the axis; later slices hold j_k points, j_k a
  power of two that doubles when the chord between neighbours on the slice
  exceeds 1.8 times the angular step from the previous slice (both measured
  on the unit sphere at the slices' mean polar angles);
* the azimuth of point i of slice k is 2 pi i / j_k + pi / j_k + phi_r with
  phi_r the azimuth of the last point of slice k-1 plus (k-1) 2 pi / j_{k-1};
* the polar angle of slice k is the mean of its bounding angles; slices stop
  at the cap's edge, so the count is "rounded to the next convenient value";
* projected points snap to the nearest grid node (repeats are dropped), and
  the weights are normalised to sum to the plane's area (sum h_m = X Y), the
  convention of the plan's default weights.
"""
from __future__ import annotations

import math

import numpy as np


def _snap(x, pitch, n):
    """Nearest node of a lattice of n nodes at (i - floor(n/2)) * pitch."""
    i = np.clip(np.rint(x / pitch) + n // 2, 0, n - 1)
    return (i - n // 2) * pitch


def equisteradian_mask(n_points, grid_nodes, pitch, r0):
    """Sensor positions (M, 2) and weights (M,) of an equi-steradian mask.

    n_points    desired number of acquisition points (rounded).
    grid_nodes  nodes per side of the square sensor grid (x and y).
    pitch       grid spacing in metres.
    r0          depth of the centre of interest below the sensor plane (m)."""
    if n_points < 1 or grid_nodes < 1 or pitch <= 0 or r0 <= 0:
        raise ValueError("n_points, grid_nodes, pitch and r0 must be positive")
    half = 0.5 * grid_nodes * pitch
    theta_max = math.atan2(half, r0)
    cap = 2 * math.pi * (1 - math.cos(theta_max))
    omega = cap / n_points                       # unit solid angle
    # slice 1: one point on the axis; then rings of j (a power of two) points
    th1 = math.acos(max(-1.0, 1 - omega / (2 * math.pi)))
    slices = [(0.0, th1, 1, 0.0)]                # (theta_lo, theta_hi, j, mean polar angle)
    j = 2
    while True:
        th_lo, prev_mid = slices[-1][1], slices[-1][3]
        while True:
            th_hi = math.acos(max(-1.0, math.cos(th_lo) - omega * j / (2 * math.pi)))
            mid = 0.5 * (th_lo + th_hi)
            chord = 2 * math.sin(mid) * math.sin(math.pi / j)
            if chord > 1.8 * (mid - prev_mid):
                j *= 2
                continue
            break
        if mid > theta_max:
            break
        slices.append((th_lo, th_hi, j, mid))
    pts = []
    phi_last, j_prev = 0.0, 1
    for k, (_, _, jk, theta) in enumerate(slices, start=1):
        phi_r = phi_last + (k - 1) * 2 * math.pi / j_prev
        for i in range(jk):
            phi = 2 * math.pi * i / jk + math.pi / jk + phi_r
            rho = r0 * math.tan(theta)
            pts.append((rho * math.cos(phi), rho * math.sin(phi)))
        phi_last = 2 * math.pi * (jk - 1) / jk + math.pi / jk + phi_r
        j_prev = jk
    xy = np.array(pts, dtype=np.float64)
    xy[:, 0] = _snap(xy[:, 0], pitch, grid_nodes)
    xy[:, 1] = _snap(xy[:, 1], pitch, grid_nodes)
    xy = np.unique(xy, axis=0)
    r = np.sqrt(xy[:, 0] ** 2 + xy[:, 1] ** 2 + r0 ** 2)
    h = r ** 3
    area = (grid_nodes * pitch) ** 2
    return xy, h * (area / h.sum())


def equiangular_mask(n_points, grid_nodes, pitch, r0):
    """Positions (M,) on the sensor line and weights (M,) of an equiangular
    mask: equal angular steps seen from a centre of interest at depth r0
    below the middle of a line of grid_nodes nodes; weights h_m ~ r^2,
    normalised to sum to the line's length."""
    if n_points < 1 or grid_nodes < 1 or pitch <= 0 or r0 <= 0:
        raise ValueError("n_points, grid_nodes, pitch and r0 must be positive")
    half = 0.5 * grid_nodes * pitch
    theta_max = math.atan2(half, r0)
    step = 2 * theta_max / n_points
    theta = -theta_max + (np.arange(n_points) + 0.5) * step
    x = np.unique(_snap(r0 * np.tan(theta), pitch, grid_nodes))
    h = x ** 2 + r0 ** 2
    return x, h * (grid_nodes * pitch / h.sum())
