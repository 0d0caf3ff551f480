"""More planted mistakes (on the CPU, by monkeypatching), in the oracle's
d = 2 operator, weight gradient, Voronoi weights and image measures: at
least one pin catches each."""
import numpy as np
import pytest

from oracle import metrics, ndft, voronoi
import pinlib


def test_mutation_2d_row_spacing(monkeypatch):
    """The d = 2 grid's one y row taken with spacing dx instead of 1: the
    weights a_m = h_m/(dx dy) and nothing else change."""
    G0 = ndft.Grid2

    class Bad(G0):
        def __init__(self, nx, nz, dx, dz):
            super().__init__(nx, nz, dx, dz)
            self.dy = float(dx)
    monkeypatch.setattr(ndft, "Grid2", Bad)
    assert pinlib.pin_plane_wave_2d() > 1e-2
    assert pinlib.pin_2d_is_y_invariant_3d() > 1e-2


def test_mutation_2d_line_on_y(monkeypatch):
    """Sensors of the d = 2 operator placed along y instead of x."""
    monkeypatch.setattr(ndft, "_line", lambda x: np.stack([np.zeros_like(np.asarray(x, float).ravel()),
                                                          np.asarray(x, float).ravel()], axis=1))
    assert pinlib.pin_2d_is_y_invariant_3d() > 1e-2


def test_mutation_weight_grad_without_inverse_h(monkeypatch):
    from test_oracle_pins import test_weight_grad_is_the_per_sensor_image
    w0 = ndft.weight_grad
    monkeypatch.setattr(ndft, "weight_grad", lambda xy, h, *a: w0(xy, h, *a) * h)
    with pytest.raises(AssertionError):
        test_weight_grad_is_the_per_sensor_image()


def test_mutation_voronoi_wrong_period():
    pytest.importorskip("scipy.spatial")
    from test_voronoi_oracle import test_areas_match_raster_nearest_counts, test_cells_tile_the_torus_and_lattice_cells
    t0 = voronoi._tiled
    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(voronoi, "_tiled", lambda xy, X, Y: t0(xy, X, X))
        with pytest.raises(AssertionError):
            test_cells_tile_the_torus_and_lattice_cells()
        with pytest.raises(AssertionError):
            test_areas_match_raster_nearest_counts()


def test_mutation_voronoi_gradient_sign():
    pytest.importorskip("scipy.spatial")
    from test_voronoi_oracle import test_area_gradient_matches_finite_differences
    g0 = voronoi.areas_2d_grad
    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(voronoi, "areas_2d_grad", lambda xy, X, Y, gh: g0(xy, X, Y, gh) * np.array([1.0, -1.0]))
        with pytest.raises(AssertionError):
            test_area_gradient_matches_finite_differences()


def test_mutation_voronoi_one_sided_lengths():
    """Cell lengths on the circle taken as the gap to the right neighbour
    (they still sum to X)."""
    from test_voronoi_oracle import test_length_gradient_matches_finite_differences

    def right_gap(x, X):
        x = np.asarray(x, dtype=np.float64)
        o = np.argsort(x, kind="stable")
        xs = x[o]
        nxt = np.roll(xs, -1)
        nxt[-1] += X
        out = np.empty_like(x)
        out[o] = nxt - xs
        return out
    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(voronoi, "lengths_1d", right_gap)
        assert abs(voronoi.lengths_1d(np.array([-0.3, 0.1, 0.2]), 1.0).sum() - 1.0) <= 1e-15
        with pytest.raises(AssertionError):
            test_length_gradient_matches_finite_differences()


def test_mutation_tenenbaum_interior_normalisation():
    from test_metrics import test_tenenbaum_closed_forms, test_tenenbaum_matches_scipy_convolution

    def bad(u):
        gx, gy = metrics.sobel_pair(u)
        return float(np.sum(gx * gx + gy * gy) / gx.size)
    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(metrics, "tenenbaum", bad)
        with pytest.raises(AssertionError):
            test_tenenbaum_closed_forms()
        pytest.importorskip("scipy.signal")
        with pytest.raises(AssertionError):
            test_tenenbaum_matches_scipy_convolution()


def test_mutation_correlation_uncentred():
    from test_metrics import test_correlation_matches_numpy_and_invariances

    def bad(u1, u2):
        a = np.asarray(u1, dtype=np.float64).ravel()
        b = np.asarray(u2, dtype=np.float64).ravel()
        return float(np.sum(a * b) / np.sqrt(np.sum(a * a) * np.sum(b * b)))
    with pytest.MonkeyPatch.context() as mp:
        mp.setattr(metrics, "correlation", bad)
        with pytest.raises(AssertionError):
            test_correlation_matches_numpy_and_invariances()
