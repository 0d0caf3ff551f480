"""Equi-steradian and equiangular sensor masks (host set-up for a plan):
counts, grid nodes, equal solid angle per point, weights r^3 / r^2."""
import math

import numpy as np
import pytest

from paper_1501_02946_gb300 import masks


# The last flag: whether the grid is fine enough against r0 for the plane
# density to follow r0 / r^3 over thirds of the radius.  With a few hundred
# points the power-of-two ring counts step the density coarsely, and snapping
# to a 100 um pitch near a 2 mm focus moves the inner points by a ring width.
@pytest.mark.parametrize("n,nodes,pitch,r0,fine", [(1625, 226, 60e-6, 3.6e-3, True),
                                                   (400, 128, 1e-4, 2e-3, False),
                                                   (2000, 224, 60e-6, 5e-3, True)])
def test_equisteradian_mask(n, nodes, pitch, r0, fine):
    xy, h = masks.equisteradian_mask(n, nodes, pitch, r0)
    M = xy.shape[0]
    assert 0.85 * n <= M <= 1.15 * n                     # "rounded to a convenient value"
    # on grid nodes, inside the grid, no repeats
    idx = xy / pitch + nodes // 2
    assert np.allclose(idx, np.rint(idx), atol=1e-9)
    assert idx.min() >= 0 and idx.max() <= nodes - 1
    assert np.unique(xy, axis=0).shape[0] == M
    # centred and mirror-balanced
    assert np.abs(xy.mean(axis=0)).max() <= 2 * pitch
    # equal solid angle per point seen from the centre of interest: M points
    # over the solid angle the rings cover, about n over the whole cap
    r = np.sqrt((xy ** 2).sum(axis=1) + r0 ** 2)
    cap = 2 * math.pi * (1 - math.cos(math.atan2(0.5 * nodes * pitch, r0)))
    covered = 2 * math.pi * (1 - (r0 / r).min())
    assert abs((M / covered) / (n / cap) - 1) <= 0.15
    # so the density on the plane falls like r0 / r^3: inner disc against an
    # outer ring of the covered radius
    rho = np.hypot(xy[:, 0], xy[:, 1])
    R = rho.max()
    def expected(a, b):  # points per unit plane area ~ r0 / r^3, averaged over a <= rho < b
        t = np.linspace(a, b, 2001)
        f = r0 / (t ** 2 + r0 ** 2) ** 1.5 * t
        return f.sum() / t.sum()
    inner = (rho < R / 3).sum() / (math.pi * (R / 3) ** 2)
    outer = (rho >= 2 * R / 3).sum() / (math.pi * (R ** 2 - (2 * R / 3) ** 2))
    ratio = expected(0, R / 3) / expected(2 * R / 3, R)
    if fine:
        assert abs((inner / outer) / ratio - 1) <= 0.35
    # the slices cover the cap from the axis out: no quarter of the polar
    # range is empty
    th = np.arctan2(rho, r0)
    counts = np.histogram(th, bins=4, range=(0, th.max()))[0]
    assert counts.min() > 0
    # weights ~ r^3, summing to the plane's area
    assert np.allclose(h / h.sum(), r ** 3 / (r ** 3).sum())
    assert abs(h.sum() - (nodes * pitch) ** 2) <= 1e-12 * (nodes * pitch) ** 2


def test_equiangular_mask():
    n, nodes, pitch, r0 = 101, 226, 60e-6, 3.6e-3
    x, h = masks.equiangular_mask(n, nodes, pitch, r0)
    assert 0.9 * n <= x.size <= n
    th = np.arctan2(x, r0)
    steps = np.diff(th)
    # equal angular steps up to the snapping of each point to a node
    tol = pitch / r0
    assert np.abs(steps - np.median(steps)).max() <= 2 * tol
    assert np.allclose(h / h.sum(), (x ** 2 + r0 ** 2) / (x ** 2 + r0 ** 2).sum())
    assert abs(h.sum() - nodes * pitch) <= 1e-12


def test_masks_reject_bad_arguments():
    with pytest.raises(ValueError):
        masks.equisteradian_mask(0, 10, 1e-4, 1e-3)
    with pytest.raises(ValueError):
        masks.equiangular_mask(10, 10, 1e-4, -1.0)
