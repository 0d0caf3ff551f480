"""The seeded synthetic inputs follow their stated recipes: sensor layouts
(jitter bounds, the centre-dense density ratio, the dart-throwing minimum
spacing), phantom parameter ranges, the noise level, and the uneven batch's
size distribution."""
import numpy as np
import pytest

import synth


def _lattice_offsets(xy, nsx, nsy, px, py):
    """Offsets of the first nsx * nsy sensors from their lattice nodes, in
    pitches."""
    nodes = synth.lattice_positions(nsx, nsy, px, py)
    d = xy[: nsx * nsy] - nodes
    return d[:, 0] / px, d[:, 1] / py


def test_c1_recipe():
    P = synth.c1()
    assert P.xy.shape == (1024, 2) and P.g.shape == (1024, 128)
    assert P.grid.shape == (32, 32, 64) and P.grid.dx == P.grid.dz == 1e-4
    ox, oy = _lattice_offsets(P.xy, 32, 32, 1e-4, 1e-4)
    assert np.abs(ox).max() <= 0.4 and np.abs(oy).max() <= 0.4
    assert np.abs(ox).max() > 0.35  # jitter actually spans the range
    assert P.dt == 20e-9 and P.c == synth.C_WATER
    assert P.balls == [(0.0, 0.0, 1.5e-3, 0.4e-3, 1.0)]
    assert abs(P.h.sum() - (32e-4) ** 2) <= 1e-15


def test_c2_recipe():
    P = synth.c2()
    assert P.xy.shape == (16384, 2) and P.g.shape == (16384, 512)
    assert P.grid.shape == (128, 128, 256)
    # half on a jittered 128 x 64 lattice at 100 x 200 um
    ox, oy = _lattice_offsets(P.xy, 128, 64, 1e-4, 2e-4)
    assert np.abs(ox).max() <= 0.4 and np.abs(oy).max() <= 0.4
    # half drawn with twice the density inside r < 3.2 mm, within +-6.4 mm
    b = P.xy[8192:]
    assert np.abs(b).max() < 6.4e-3
    r = np.hypot(b[:, 0], b[:, 1])
    area_in = np.pi * 3.2e-3 ** 2
    area_out = (12.8e-3) ** 2 - area_in
    ratio = (np.sum(r < 3.2e-3) / area_in) / (np.sum(r >= 3.2e-3) / area_out)
    assert 1.85 <= ratio <= 2.15, ratio
    # 20 balls in the stated ranges
    assert len(P.balls) == 20
    for (x, y, z, R, p0) in P.balls:
        assert abs(x) <= 4.8e-3 and abs(y) <= 4.8e-3
        assert 1e-3 <= z <= 6e-3 and 1e-4 <= R <= 5e-4 and 0.5 <= p0 <= 1.0
    # noise: 1 % of the clean data's peak
    clean = synth.c2(noise=False).g
    noise = P.g - clean
    assert abs(noise.std() / (0.01 * np.abs(clean).max()) - 1.0) <= 0.01
    assert abs(noise.mean()) <= 1e-2 * noise.std()


def test_c3_positions_keep_the_minimum_spacing():
    spatial = pytest.importorskip("scipy.spatial")
    # the first draw of the 256 x 256 x 512 workload's generator
    xy = synth.dart_throwing(np.random.default_rng(1503), 65536, 12.8e-3, 4e-5)
    assert xy.shape == (65536, 2)
    assert np.abs(xy).max() <= 12.8e-3
    assert len(spatial.cKDTree(xy).query_pairs(4e-5 * (1 - 1e-12))) == 0
    # random-uniform: each quadrant holds a quarter, to sampling error
    q = np.bincount((xy[:, 0] > 0).astype(int) * 2 + (xy[:, 1] > 0).astype(int), minlength=4)
    assert np.all(np.abs(q / 65536 - 0.25) <= 0.01)


def test_batch_recipe():
    shapes = synth.batch_shapes()
    assert len(shapes) == 64
    sizes = synth.seven_smooth(64, 256)
    assert all(N in sizes for N, _ in shapes)
    assert {T for _, T in shapes} == {256, 512, 1024}
    sympy = pytest.importorskip("sympy")
    assert sizes == [n for n in range(64, 257) if set(sympy.factorint(n)) <= {2, 3, 5, 7}]
    P = synth.batch_instance(np.random.default_rng(0), 70, 256)
    assert P.xy.shape == (4900, 2) and P.grid.shape == (70, 70, 512)
