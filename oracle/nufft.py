"""O2: the NEDNER-NUFFT algorithm in FP64 (oracle; test infrastructure).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows the three steps of Sec. 3 in the paper's order, each restated here:

1. NED-NUFFT (eq:NED_NUFFT): in each spatial coordinate the sensor positions
   become grid coordinates U = sigma N x / X on an oversampled grid of
   sigma*N cells (periodic, since the sum is X-periodic in x).  Every sample
   g[m, n], weighted by a_m = h_m/(dx dy), is spread with the tensor-product
   window phi(Ux - p) phi(Uy - q) onto the w x w nearest cells; the grid is
   Fourier transformed and each kept frequency j is divided by
   phihat(jx/(sigma nx)) phihat(jy/(sigma ny)).
2. NER-NUFFT (eq:NER_NUFFT): along time, with the samples re-indexed about
   the centre (n' = n - floor(nt/2), which is the paper's theta = 2 pi n/N - pi
   and gives the phase exp(-i pi (kappa - mu))), each sample is divided by
   phihat(n'/(sigma nt)), zero-padded to sigma*nt, Fourier transformed, and the
   value at the non-integer frequency tau = omega nt dt / (2 pi) is read off with
   the w nearest grid values weighted by phi(sigma tau - p), times
   exp(-2 pi i tau floor(nt/2) / nt).
3. Weight (dt/dz) W(j, l) and the uniform inverse 3D DFT, taken from O1.

The window is the Kaiser-Bessel pair of window.py.  The transpose of each step
is written out below for the dot-product checks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import ndft
from .window import kb_beta, kb_phi, kb_phihat


def grid_coords(pos, extent, M):
    """U = M * u where u = pos/extent reduced to [-1/2, 1/2) (exact: the sums
    are extent-periodic in pos)."""
    u = pos / extent
    u = u - np.floor(u + 0.5)
    return M * u


def footprint(U, width):
    """Taps p = floor(U) - width/2 + 1 + t (t = 0 .. width-1) and U - p."""
    base = np.floor(U).astype(np.int64)
    t = np.arange(width)
    p = base[..., None] - width // 2 + 1 + t
    return p, U[..., None] - p


def spread_matrix(xy, h, grid, sigma, width):
    """Sparse Phi with G0.ravel() = Phi @ g: rows (p mod Mx)*My + (q mod My)."""
    nx, ny, _, dx, dy, _ = grid.as_tuple()
    Mx, My = sigma * nx, sigma * ny
    beta = kb_beta(width, sigma)
    Ux = grid_coords(xy[:, 0], nx * dx, Mx)
    Uy = grid_coords(xy[:, 1], ny * dy, My)
    px, ddx = footprint(Ux, width)
    py, ddy = footprint(Uy, width)
    wx = kb_phi(ddx, width, beta)          # (M, w)
    wy = kb_phi(ddy, width, beta)
    a = h / (dx * dy)
    M = xy.shape[0]
    rows = (px[:, :, None] % Mx) * My + (py[:, None, :] % My)          # (M, w, w)
    vals = a[:, None, None] * wx[:, :, None] * wy[:, None, :]
    cols = np.broadcast_to(np.arange(M)[:, None, None], rows.shape)
    return sp.csr_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(Mx * My, M))


def ned(xy, h, g, grid, sigma=2, width=16):
    """Step 1: G1(jx, jy, n) on the full frequency grid, shape (nx, ny, nt)."""
    nx, ny = grid.nx, grid.ny
    Mx, My = sigma * nx, sigma * ny
    beta = kb_beta(width, sigma)
    Phi = spread_matrix(xy, h, grid, sigma, width)
    G0 = (Phi @ g).reshape(Mx, My, g.shape[1])
    G0hat = np.fft.fft2(G0, axes=(0, 1))
    jx, jy = ndft.freqs(nx), ndft.freqs(ny)
    G1 = G0hat[np.ix_(jx % Mx, jy % My)]
    deconv = 1.0 / (kb_phihat(jx / Mx, width, beta)[:, None] * kb_phihat(jy / My, width, beta)[None, :])
    return G1 * deconv[:, :, None]


def ned_adjoint(xy, h, G1bar, grid, sigma=2, width=16):
    """Transpose of ned (g real): g' = Phi^T Re(Mx My ifft2(zero-padded))."""
    nx, ny = grid.nx, grid.ny
    Mx, My = sigma * nx, sigma * ny
    nt = G1bar.shape[2]
    beta = kb_beta(width, sigma)
    jx, jy = ndft.freqs(nx), ndft.freqs(ny)
    deconv = 1.0 / (kb_phihat(jx / Mx, width, beta)[:, None] * kb_phihat(jy / My, width, beta)[None, :])
    H = np.zeros((Mx, My, nt), dtype=np.complex128)
    H[np.ix_(jx % Mx, jy % My)] = G1bar * deconv[:, :, None]
    G0bar = (np.fft.ifft2(H, axes=(0, 1)) * (Mx * My)).real
    Phi = spread_matrix(xy, h, grid, sigma, width)
    return Phi.T @ G0bar.reshape(Mx * My, nt)


def _ner_prepare(nt, sigma, width):
    Mt = sigma * nt
    nc = nt // 2
    nprime = np.arange(nt) - nc
    beta = kb_beta(width, sigma)
    return Mt, nc, nprime, beta


def ner(G1, tau, sigma=2, width=16):
    """Step 2: Ghat(..., l) = sum_n G1(..., n) exp(-2 pi i tau(..., l) n / nt)
    by the window method.  G1 has shape (..., nt), tau (..., nz)."""
    nt = G1.shape[-1]
    Mt, nc, nprime, beta = _ner_prepare(nt, sigma, width)
    v = G1 / kb_phihat(nprime / Mt, width, beta)
    H = np.zeros(G1.shape[:-1] + (Mt,), dtype=np.complex128)
    H[..., nprime % Mt] = v
    H = np.fft.fft(H, axis=-1)
    out = np.empty(tau.shape, dtype=np.complex128)
    for l in range(tau.shape[-1]):
        U = sigma * tau[..., l]
        p, d = footprint(U, width)
        vals = np.take_along_axis(H, p % Mt, axis=-1)
        out[..., l] = np.sum(kb_phi(d, width, beta) * vals, axis=-1)
    return out * np.exp(-2j * np.pi * tau * nc / nt)


def ner_adjoint(Ghatbar, tau, nt, sigma=2, width=16):
    """Transpose of ner (complex-linear, so the conjugate transpose)."""
    Mt, nc, nprime, beta = _ner_prepare(nt, sigma, width)
    vals = Ghatbar * np.exp(2j * np.pi * tau * nc / nt)
    lead = Ghatbar.shape[:-1]
    ncol = int(np.prod(lead))
    Hbar = np.zeros((ncol, Mt), dtype=np.complex128)
    col = np.arange(ncol)
    for l in range(tau.shape[-1]):
        U = (sigma * tau[..., l]).reshape(ncol)
        p, d = footprint(U, width)
        w = kb_phi(d, width, beta) * vals[..., l].reshape(ncol)[:, None]
        np.add.at(Hbar, (np.repeat(col, width), (p % Mt).ravel()), w.ravel())
    vbar = np.fft.ifft(Hbar, axis=-1) * Mt
    G1bar = vbar[:, nprime % Mt] / kb_phihat(nprime / Mt, width, beta)
    return G1bar.reshape(lead + (nt,))


def tau_of(grid, c, dt, nt):
    omega, W = ndft.omega_and_weight(grid, c)
    return omega * nt * dt / (2 * np.pi), W


def spectrum_cotangent(fbar, dt, c, grid, nt, sigma=2, width=16, rows=None):
    """G1bar(j, n): the cotangent of the spatial spectrum G1 in the transposed
    chain of reconstruct -- the image adjoint, the weight (dt/dz) W and the NER
    adjoint, i.e. reconstruct_adjoint without its last (NED) step -- on the
    full index sets, shape (nx, ny, nt).  With `rows`, the NER adjoint takes
    that many jx rows at a time (each column is independent, so the values
    are the same; only the memory held at once is smaller)."""
    tau, W = tau_of(grid, c, dt, nt)
    Fbar = ndft.image_transform_adjoint(fbar, grid)
    Ghatbar = (dt / grid.dz) * W * Fbar
    del Fbar
    if rows is None:
        return ner_adjoint(Ghatbar, tau, nt, sigma, width)
    out = np.empty(Ghatbar.shape[:2] + (nt,), dtype=np.complex128)
    for a in range(0, Ghatbar.shape[0], rows):
        out[a:a + rows] = ner_adjoint(Ghatbar[a:a + rows], tau[a:a + rows], nt, sigma, width)
    return out


def reconstruct(xy, h, g, dt, c, grid, sigma=2, width=16, full=False):
    nt = g.shape[1]
    G1 = ned(xy, h, g, grid, sigma, width)
    tau, W = tau_of(grid, c, dt, nt)
    Ghat = ner(G1, tau, sigma, width)
    F = (dt / grid.dz) * W * Ghat
    Y = ndft.image_transform(F, grid)
    if full:
        return Y.real, dict(G1=G1, Ghat=Ghat, F=F, Y=Y)
    return Y.real


def reconstruct_adjoint(xy, h, fbar, dt, c, grid, nt, sigma=2, width=16):
    tau, W = tau_of(grid, c, dt, nt)
    Fbar = ndft.image_transform_adjoint(fbar, grid)
    Ghatbar = (dt / grid.dz) * W * Fbar
    G1bar = ner_adjoint(Ghatbar, tau, nt, sigma, width)
    return ned_adjoint(xy, h, G1bar, grid, sigma, width)
