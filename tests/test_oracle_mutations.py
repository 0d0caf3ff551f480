"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching) and
check that at least one pin catches each.  This shows the pins are strong
enough that the oracle cannot be wrong in these ways and still pass."""
import numpy as np
import pytest

from oracle import ndft, nufft
import pinlib


def _orig(name):
    return getattr(ndft, name)


@pytest.fixture
def patch(monkeypatch):
    return monkeypatch


def test_mutation_omega_sign(patch):
    f0 = _orig("omega_and_weight")
    patch.setattr(ndft, "omega_and_weight", lambda grid, c: (-f0(grid, c)[0], f0(grid, c)[1]))
    assert pinlib.pin_plane_wave() > 1e-2
    assert pinlib.pin_integer_tau() > 1e-2


def test_mutation_weight_factor(patch):
    f0 = _orig("omega_and_weight")
    patch.setattr(ndft, "omega_and_weight", lambda grid, c: (f0(grid, c)[0], 0.5 * f0(grid, c)[1]))
    assert pinlib.pin_plane_wave() > 1e-2


def test_mutation_weight_at_l0(patch):
    f0 = _orig("omega_and_weight")

    def bad(grid, c):
        om, W = f0(grid, c)
        return om, np.where(W == 0, 2 * c, W)
    patch.setattr(ndft, "omega_and_weight", bad)
    assert pinlib.pin_depth_sum() > 1e-3


def test_mutation_spatial_sign(patch):
    f0 = _orig("spatial_factors")
    patch.setattr(ndft, "spatial_factors", lambda xy, grid, *a: tuple(E.conj() for E in f0(xy, grid, *a)))
    assert pinlib.pin_lattice_fft2() > 1e-2
    assert pinlib.pin_shift_roll() > 1e-2


def test_mutation_transposed_axes(patch):
    f0 = _orig("spatial_factors")

    def bad(xy, grid, *a):
        return f0(xy[:, ::-1].copy(), grid, *a)
    patch.setattr(ndft, "spatial_factors", bad)
    assert pinlib.pin_lattice_fft2() > 1e-2


def test_mutation_depth_origin(patch):
    f0 = _orig("image_factors")

    def bad(grid):
        Ax, Ay, Az = f0(grid)
        kz = 2 * np.pi * ndft.freqs(grid.nz) / (grid.nz * grid.dz)
        z = (np.arange(grid.nz) - grid.nz // 2) * grid.dz
        return Ax, Ay, np.exp(1j * np.outer(z, kz))
    patch.setattr(ndft, "image_factors", bad)
    assert pinlib.pin_plane_wave() > 1e-2


def test_mutation_time_origin(patch):
    f0 = _orig("time_transform")

    def bad(G1, omega, dt):
        shifted = np.zeros_like(G1)
        shifted[..., 1:] = G1[..., :-1]
        return f0(shifted, omega, dt)
    patch.setattr(ndft, "time_transform", bad)
    assert pinlib.pin_integer_tau() > 1e-2


def test_mutation_ner_centring_phase(patch):
    ner0 = nufft.ner

    def bad(G1, tau, sigma=2, width=16):
        nt = G1.shape[-1]
        return ner0(G1, tau, sigma, width) * np.exp(2j * np.pi * tau * (nt // 2) / nt)
    patch.setattr(nufft, "ner", bad)

    def via_ner(col, omega, dt):
        nt = col.shape[0]
        tau = np.array([[omega * nt * dt / (2 * np.pi)]])
        return nufft.ner(col[None, :], tau, 2, 16)[0, 0]
    assert pinlib.pin_integer_tau(via_ner) > 1e-2


def test_mutation_ned_deconvolution(patch):
    import oracle.nufft as nm
    phihat0 = nm.kb_phihat
    patch.setattr(nm, "kb_phihat", lambda xi, w, b: phihat0(0 * xi, w, b))
    assert pinlib.pin_lattice_fft2(lambda xy, h, g, grid: nufft.ned(xy, h, g, grid, 2, 16)) > 1e-3
