"""Pins of the CPU oracle to facts that do not come from the oracle itself."""
import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import ndft, nufft
from oracle.window import kb_beta, kb_phi, kb_phi_deriv, kb_phihat

import pinlib


@pytest.mark.parametrize("width,sigma", [(8, 2), (12, 2), (16, 2), (6, 2)])
def test_kb_transform_matches_quadrature(width, sigma):
    """The closed-form Kaiser-Bessel transform equals the integral of the
    window computed by adaptive quadrature (Sec. 3 asks for an analytically
    known transform), including the sin branch past pi w xi > beta."""
    beta = kb_beta(width, sigma)
    xis = np.array([0.0, 0.05, 0.1, 0.2, 0.25, 0.37, 0.5, 0.8, 1.3])
    ref = []
    for xi in xis:
        v, _ = integrate.quad(lambda x: kb_phi(x, width, beta) * np.cos(2 * np.pi * xi * x),
                              -width / 2, width / 2, limit=400, epsabs=0, epsrel=1e-13)
        ref.append(v)
    ref = np.array(ref)
    got = kb_phihat(xis, width, beta)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.abs(ref).max()


def test_kb_derivative_matches_fd():
    beta = kb_beta(8, 2)
    x = np.linspace(-3.9, 3.9, 41)
    e = 1e-6
    fd = (kb_phi(x + e, 8, beta) - kb_phi(x - e, 8, beta)) / (2 * e)
    assert np.max(np.abs(kb_phi_deriv(x, 8, beta) - fd)) <= 1e-6 * np.abs(fd).max()


def test_lattice_sensors_give_fft2_o1():
    assert pinlib.pin_lattice_fft2() <= 1e-12


def test_lattice_sensors_give_fft2_o2():
    assert pinlib.pin_lattice_fft2(lambda xy, h, g, grid: nufft.ned(xy, h, g, grid, 2, 16)) <= 1e-11


def test_integer_tau_is_fft_bin_o1():
    assert pinlib.pin_integer_tau() <= 1e-12


def test_integer_tau_is_fft_bin_o2():
    def via_ner(col, omega, dt):
        nt = col.shape[0]
        tau = np.array([[omega * nt * dt / (2 * np.pi)]])
        return nufft.ner(col[None, :], tau, 2, 16)[0, 0]
    assert pinlib.pin_integer_tau(via_ner) <= 1e-11


@pytest.mark.parametrize("halfstep", [False, True])
def test_plane_wave_profile_recovered_o1(halfstep):
    assert pinlib.pin_plane_wave(halfstep=halfstep) <= 1e-9


def test_plane_wave_profile_recovered_o2():
    rec = lambda xy, h, g, dt, c, grid: nufft.reconstruct(xy, h, g, dt, c, grid, 2, 16)
    assert pinlib.pin_plane_wave(rec) <= 1e-9


def test_depth_sum_constant():
    assert pinlib.pin_depth_sum() <= 1e-12


def test_shift_rolls_and_period_invariance():
    assert pinlib.pin_shift_roll() <= 1e-12


def test_linearity_in_data_and_weights():
    P = synth.tiny()
    rng = np.random.default_rng(1)
    g2 = rng.normal(size=P.g.shape)
    f_a = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    f_b = ndft.reconstruct(P.xy, P.h, g2, P.dt, P.c, P.grid)
    f_ab = ndft.reconstruct(P.xy, P.h, 2.0 * P.g - 3.0 * g2, P.dt, P.c, P.grid)
    assert pinlib.rel(f_ab, 2.0 * f_a - 3.0 * f_b) <= 1e-12
    f_h = ndft.reconstruct(P.xy, 2.5 * P.h, P.g, P.dt, P.c, P.grid)
    assert pinlib.rel(f_h, 2.5 * f_a) <= 1e-12


def test_adjoint_dot_o1():
    assert pinlib.pin_adjoint_dot(ndft.reconstruct, ndft.reconstruct_adjoint) <= 1e-12


def test_adjoint_dot_o2():
    rec = lambda *a: nufft.reconstruct(*a, sigma=2, width=8)
    adj = lambda *a: nufft.reconstruct_adjoint(*a, sigma=2, width=8)
    assert pinlib.pin_adjoint_dot(rec, adj) <= 1e-12


def test_position_grad_matches_finite_differences():
    assert pinlib.pin_position_grad_fd() <= 1e-6


@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_o2_matches_o1(name):
    """The NUFFT algorithm with a wide window reproduces the direct sum."""
    P = getattr(synth, name)()
    f1 = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    f16 = nufft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid, 2, 16)
    f8 = nufft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid, 2, 8)
    assert pinlib.rel(f16, f1) <= 1e-12
    assert pinlib.rel(f8, f1) <= 1e-6
    gb = np.random.default_rng(2).normal(size=P.grid.shape)
    a1 = ndft.reconstruct_adjoint(P.xy, P.h, gb, P.dt, P.c, P.grid, P.n_t)
    a16 = nufft.reconstruct_adjoint(P.xy, P.h, gb, P.dt, P.c, P.grid, P.n_t, 2, 16)
    assert pinlib.rel(a16, a1) <= 1e-12


def test_ball_closed_form_wide_aperture():
    """Uniform ball (closed-form N-shaped data) seen through a 9.6 mm
    aperture: the reconstruction correlates with the voxelised ball, peaks
    inside it and has no mirror image at Z - z.  Limited view leaves the
    absolute level only loosely determined, hence the wide amplitude band."""
    ns, nt, pitch = 96, 384, 1e-4
    xy = synth.lattice_positions(ns, ns, pitch, pitch)
    grid = synth.Grid(ns, ns, 64, pitch, pitch, pitch)
    balls = [(0.0, 0.0, 1.5e-3, 0.4e-3, 1.0)]
    g = synth.balls_data(xy, nt, 20e-9, balls, 1500.0)
    h = np.full(xy.shape[0], (ns * pitch) ** 2 / xy.shape[0])
    f = nufft.reconstruct(xy, h, g, 20e-9, 1500.0, grid, 2, 8)
    fv = synth.voxelise_balls(balls, grid)
    c = ns // 2
    box = (slice(c - 8, c + 8), slice(c - 8, c + 8), slice(7, 23))
    assert synth.correlation_coefficient(f[box], fv[box]) >= 0.85
    am = np.unravel_index(np.argmax(f), f.shape)
    assert fv[am] > 0
    assert 0.5 <= f[fv > 0].mean() <= 1.2
    assert np.abs(f[:, :, 32:]).max() < 0.1 * f.max()


def test_ball_c1_geometry():
    """configs' 32x32 sensor instance: peak inside the ball, no mirror."""
    P = synth.c1()
    f = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    fv = P.voxelised()
    am = np.unravel_index(np.argmax(f), f.shape)
    assert fv[am] > 0
    assert np.abs(f[:, :, 32:]).max() < 0.1 * f.max()
    assert f[fv > 0].mean() > 0.2


# --- single-column and single-voxel helpers (used for sampled checks at full size)
@pytest.mark.parametrize("shape", [(8, 8, 16), (7, 9, 11), (6, 5, 8)])
def test_column_depth_profile_matches_full_o1(shape):
    """Each column's depth profile equals the corresponding slice of the full
    O1 chain (Hermitian part of F, inverse DFT over depth), odd and even N."""
    nx, ny, nz = shape
    rng = np.random.default_rng(11)
    grid = synth.Grid(nx, ny, nz, 1e-4, 1.2e-4, 0.9e-4)
    X, Y = nx * grid.dx, ny * grid.dy
    xy = np.stack([rng.uniform(-X / 2, X / 2, 30), rng.uniform(-Y / 2, Y / 2, 30)], axis=1)
    h = np.full(30, X * Y / 30)
    g = rng.normal(size=(30, 24))
    dt, c = 40e-9, 1500.0
    _, aux = ndft.reconstruct(xy, h, g, dt, c, grid, full=True)
    F = aux["F"]
    hx, hy, hz = nx // 2, ny // 2, nz // 2
    ia = (2 * hx - np.arange(nx)) % nx
    ib = (2 * hy - np.arange(ny)) % ny
    ic = (2 * hz - np.arange(nz)) % nz
    Fsym = 0.5 * (F + np.conj(F[np.ix_(ia, ib, ic)]))
    E = np.exp(1j * np.outer(np.arange(nz) * grid.dz, 2 * np.pi * ndft.freqs(nz) / (nz * grid.dz)))
    full = np.einsum("zl,abl->abz", E, Fsym) / (nx * ny * nz)
    scale = np.abs(full).max()
    for jx in ndft.freqs(nx):
        for jy in ndft.freqs(ny):
            col = ndft.column_depth_profile(xy, h, g, dt, c, grid, int(jx), int(jy))
            assert np.abs(col - full[jx + hx, jy + hy]).max() <= 1e-12 * scale


@pytest.mark.parametrize("shape", [(8, 6, 5), (7, 9, 4)])
def test_half_spectrum_voxels_round_trip(shape):
    """A real image is rebuilt from its Hermitian half spectrum (taken with
    numpy.fft.fft2 over x and y), at every voxel, odd and even N."""
    nx, ny, nz = shape
    rng = np.random.default_rng(12)
    grid = synth.Grid(nx, ny, nz, 1e-4, 1e-4, 1e-4)
    f = rng.normal(size=shape)
    hx, hy = nx // 2, ny // 2
    # S(jx, jy, k) = 1/(nx ny) sum_{p,q} f exp(-i (kx x_p + ky y_q)), x_p = (p - hx) dx
    D = np.fft.fft2(f, axes=(0, 1)) / (nx * ny)
    jx, jy = ndft.freqs(nx), ndft.freqs(ny)
    ph = np.exp(2j * np.pi * (np.outer(jx, np.ones(ny)) * hx / nx + np.outer(np.ones(nx), jy) * hy / ny))
    S = D[np.ix_(jx % nx, jy % ny)] * ph[:, :, None]            # [jx + hx][jy + hy][k]
    half = S[:, hy:, :] if ny % 2 else np.concatenate([S[:, hy:, :], S[:, :1, :]], axis=1)
    pts = [(p, q, k) for p in range(nx) for q in range(ny) for k in range(nz)]
    got = ndft.half_spectrum_voxels(half, grid, pts)
    ref = np.array([f[p, q, k] for p, q, k in pts])
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape,nt", [((8, 8, 16), 32), ((7, 9, 11), 24)])
def test_spectrum_cotangent_and_sampled_sensor_helpers(shape, nt):
    """The helpers of the sampled full-size checks: the cotangent G1bar from
    the image adjoint, the weight and O2's NER adjoint (width 16, any number
    of jx rows at a time) equals O1's transposed chain; the O1 adjoint and
    the analytic gradient evaluated for a subset of the sensors equal the
    corresponding rows of the full evaluations; and the gradient of a subset
    matches FP64 central differences of the loss for that subset alone."""
    nx, ny, nz = shape
    rng = np.random.default_rng(13)
    grid = synth.Grid(nx, ny, nz, 1e-4, 1.1e-4, 0.9e-4)
    X, Y = nx * grid.dx, ny * grid.dy
    M = 40
    xy = np.stack([rng.uniform(-X / 2, X / 2, M), rng.uniform(-Y / 2, Y / 2, M)], axis=1)
    h = np.full(M, X * Y / M)
    g = rng.normal(size=(M, nt))
    fb = rng.normal(size=shape)
    dt, c = 40e-9, 1500.0
    gbar, aux = ndft.reconstruct_adjoint(xy, h, fb, dt, c, grid, nt, full=True)
    G1bar = aux["G1bar"]
    for rows in (None, 1, 3):
        got = nufft.spectrum_cotangent(fb, dt, c, grid, nt, rows=rows)
        assert np.abs(got - G1bar).max() <= 1e-11 * np.abs(G1bar).max()
    S = np.array([0, 3, 17, 39])
    sub = ndft.data_transform_adjoint(xy[S], h[S], G1bar, grid)
    assert np.abs(sub - gbar[S]).max() <= 1e-13 * np.abs(gbar).max()
    full = ndft.position_grad(xy, h, g, fb, dt, c, grid)
    gs = ndft.position_grad_from_cotangent(xy[S], h[S], g[S], G1bar, grid)
    assert np.abs(gs - full[S]).max() <= 1e-13 * np.abs(full).max()
    # dL/dx_m for sensor 3 by central differences of <fb, A(xy) g>
    eps = 1e-6 * grid.dx
    for axis in (0, 1):
        xp, xm = xy.copy(), xy.copy()
        xp[3, axis] += eps
        xm[3, axis] -= eps
        fd = (np.vdot(fb, ndft.reconstruct(xp, h, g, dt, c, grid)) -
              np.vdot(fb, ndft.reconstruct(xm, h, g, dt, c, grid))) / (2 * eps)
        assert abs(fd - gs[1, axis]) <= 1e-6 * np.abs(gs).max()


# ---------------------------------------------------------------- d = 2
def test_plane_wave_profile_recovered_2d():
    assert pinlib.pin_plane_wave_2d() <= 1e-9


def test_2d_matches_y_invariant_3d():
    assert pinlib.pin_2d_is_y_invariant_3d() <= 1e-12


def test_adjoint_dot_2d():
    assert pinlib.pin_adjoint_dot_2d() <= 1e-12


def test_position_grad_2d_matches_finite_differences():
    assert pinlib.pin_position_grad_2d() <= 1e-6


def test_weight_grad_is_the_per_sensor_image():
    """L is linear in h: dL/dh_m = <fbar, reconstruct(xy, e_m, g)> with e_m the
    m-th unit weight vector (one reconstruction per sensor)."""
    P = synth.tiny()
    rng = np.random.default_rng(31)
    fb = rng.normal(size=P.grid.shape)
    got = ndft.weight_grad(P.xy, P.h, P.g, fb, P.dt, P.c, P.grid)
    ref = np.empty(P.xy.shape[0])
    for m in range(P.xy.shape[0]):
        e = np.zeros(P.xy.shape[0])
        e[m] = 1.0
        ref[m] = np.vdot(fb, ndft.reconstruct(P.xy, e, P.g, P.dt, P.c, P.grid))
    assert pinlib.rel(got, ref) <= 1e-11
