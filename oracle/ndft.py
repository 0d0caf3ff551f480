"""O1: direct FP64 evaluation of the discrete reconstruction (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is computed (Sec. 2: the inversion formula eq:exact discretised as the
Riemann sum eq:disc_rec; restated in physical units, sound speed c):

    a_m       = h_m / (dx dy)                               (detector area weight)
    G1(j, n)  = sum_m a_m g[m, n] exp(-i (kx x_m + ky y_m))  (eq:NUDFT2 per sample)
    omega(j,l)= c * s(l) * sqrt(kx^2 + ky^2 + kz^2),  s(l) = +1 (l >= 0), -1 (l < 0)
    Ghat(j,l) = sum_n G1(j, n) exp(-i omega(j, l) n dt)        (eq:NUDFT1)
    W(j, l)   = 2 c |kz| / |K|,  W(0, 0) = 2 c                   (factor 2 K_y / kappa)
    F(j, l)   = (dt / dz) W(j, l) Ghat(j, l)
    f[p,q,k]  = Re( 1/(nx ny nz) sum_{j,l} F(j,l) exp(i (kx x_p + ky y_q + kz z_k)) )

with k = 2 pi j / X on the index sets {-floor(N/2) .. ceil(N/2) - 1} of Sec. 2,
x_p = (p - floor(nx/2)) dx, y_q likewise and z_k = k dz.  Readings taken where
the paper is silent or garbled: same-sign exponents in x and t with omega
taking the sign of kz; sign(0) = +1 and W(j != 0, 0) = 0; one-sided data from
t_0 = 0 with plain Riemann weight dt; the output is the real part.

Everything here is dense (an explicit sum per frequency), so it is O(M N^2)
and meant for small problems (8x8x16 up to 32x32x64).
"""
from __future__ import annotations

import numpy as np


def freqs(N):
    """Frequency index set {-floor(N/2), .., ceil(N/2) - 1} (Sec. 2, G_x)."""
    return np.arange(-(N // 2), N - N // 2)


def wavenumbers(grid):
    nx, ny, nz, dx, dy, dz = grid.as_tuple()
    kx = 2 * np.pi * freqs(nx) / (nx * dx)
    ky = 2 * np.pi * freqs(ny) / (ny * dy)
    kz = 2 * np.pi * freqs(nz) / (nz * dz)
    return kx, ky, kz


def wrap_index(j, N):
    """Integer frequency j moved into the index set freqs(N) (period N)."""
    lo = -(N // 2)
    return (np.asarray(j) - lo) % N + lo


def omega_weight_at(kx, ky, kz, c):
    """omega = c s(kz) |K| and W = 2 c |kz| / |K| (W = 2c at K = 0), elementwise."""
    K = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    s = np.where(kz >= 0, 1.0, -1.0)
    omega = c * s * K
    W = np.where(K > 0, 2.0 * c * np.abs(kz) / np.where(K > 0, K, 1.0), 2.0 * c)
    return omega, W


def omega_and_weight(grid, c):
    """omega(j, l) and W(j, l) on the full (jx, jy, l) grid, shape (nx, ny, nz)."""
    kx, ky, kz = wavenumbers(grid)
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    return omega_weight_at(KX, KY, KZ, c)


def spatial_factors(xy, grid, jx=None, jy=None):
    """Ex[jx, m] = exp(-i kx x_m), Ey[jy, m] = exp(-i ky y_m), by default on
    the index sets of Sec. 2; jx, jy select other integer frequencies."""
    if jx is None:
        kx, ky, _ = wavenumbers(grid)
    else:
        kx = 2 * np.pi * np.asarray(jx) / (grid.nx * grid.dx)
        ky = 2 * np.pi * np.asarray(jy) / (grid.ny * grid.dy)
    Ex = np.exp(-1j * np.outer(kx, xy[:, 0]))
    Ey = np.exp(-1j * np.outer(ky, xy[:, 1]))
    return Ex, Ey


def data_transform(xy, h, g, grid, jx=None, jy=None):
    """G1(jx, jy, n) = sum_m (h_m/(dx dy)) g[m, n] exp(-i(kx x_m + ky y_m)),
    on the index sets of Sec. 2 or on the integer frequencies jx, jy given."""
    a = h / (grid.dx * grid.dy)
    ga = (a[:, None] * g).astype(np.complex128)
    Ex, Ey = spatial_factors(xy, grid, jx, jy)
    G1 = np.empty((Ex.shape[0], Ey.shape[0], g.shape[1]), dtype=np.complex128)
    for ix in range(Ex.shape[0]):
        G1[ix] = (Ey * Ex[ix][None, :]) @ ga
    return G1


def data_transform_adjoint(xy, h, G1bar, grid):
    """Transpose of data_transform for real g: Re sum_j a_m conj(E(j, m)) G1bar."""
    a = h / (grid.dx * grid.dy)
    Ex, Ey = spatial_factors(xy, grid)
    out = np.zeros((xy.shape[0], G1bar.shape[2]))
    for ix in range(grid.nx):
        E = Ey * Ex[ix][None, :]                       # (ny, M)
        out += (E.conj().T @ G1bar[ix]).real
    return a[:, None] * out


def time_transform(G1, omega, dt):
    """Ghat(j, l) = sum_n G1(j, n) exp(-i omega(j, l) n dt)."""
    nt = G1.shape[2]
    t = np.arange(nt) * dt
    out = np.empty(omega.shape, dtype=np.complex128)
    for ix in range(G1.shape[0]):
        E = np.exp(-1j * omega[ix][:, :, None] * t[None, None, :])   # (ny, nz, nt)
        out[ix] = np.einsum("yln,yn->yl", E, G1[ix])
    return out


def time_transform_adjoint(Ghatbar, omega, dt, nt):
    """Conjugate transpose of time_transform: sum_l Ghatbar exp(+i omega n dt)."""
    t = np.arange(nt) * dt
    out = np.empty(omega.shape[:2] + (nt,), dtype=np.complex128)
    for ix in range(omega.shape[0]):
        E = np.exp(1j * omega[ix][:, :, None] * t[None, None, :])
        out[ix] = np.einsum("yln,yl->yn", E, Ghatbar[ix])
    return out


def image_factors(grid):
    """Ax[p, jx] = exp(i kx x_p), Ay[q, jy], Az[k, l] = exp(i kz z_k)."""
    nx, ny, nz, dx, dy, dz = grid.as_tuple()
    kx, ky, kz = wavenumbers(grid)
    x = (np.arange(nx) - nx // 2) * dx
    y = (np.arange(ny) - ny // 2) * dy
    z = np.arange(nz) * dz
    return np.exp(1j * np.outer(x, kx)), np.exp(1j * np.outer(y, ky)), np.exp(1j * np.outer(z, kz))


def image_transform(F, grid):
    """Complex image 1/(nx ny nz) sum_{j,l} F exp(i(kx x_p + ky y_q + kz z_k))."""
    Ax, Ay, Az = image_factors(grid)
    Y = np.tensordot(Ax, F, axes=([1], [0]))            # (p, jy, l)
    Y = np.tensordot(Ay, Y, axes=([1], [1]))            # (q, p, l)
    Y = np.tensordot(Az, Y, axes=([1], [2]))            # (k, q, p)
    return Y.transpose(2, 1, 0) / (grid.nx * grid.ny * grid.nz)


def image_transform_adjoint(fbar, grid):
    """Transpose of f = Re(image_transform(F)) for real fbar."""
    Ax, Ay, Az = image_factors(grid)
    Y = np.tensordot(Ax.conj(), fbar, axes=([0], [0]))  # (jx, q, k)
    Y = np.tensordot(Ay.conj(), Y, axes=([0], [1]))     # (jy, jx, k)
    Y = np.tensordot(Az.conj(), Y, axes=([0], [2]))     # (l, jy, jx)
    return Y.transpose(2, 1, 0) / (grid.nx * grid.ny * grid.nz)


def reconstruct(xy, h, g, dt, c, grid, full=False):
    """f = Re(image_transform((dt/dz) W Ghat)); with full=True also returns the
    intermediates (G1, Ghat, F, complex image)."""
    G1 = data_transform(xy, h, g, grid)
    omega, W = omega_and_weight(grid, c)
    Ghat = time_transform(G1, omega, dt)
    F = (dt / grid.dz) * W * Ghat
    Y = image_transform(F, grid)
    if full:
        return Y.real, dict(G1=G1, Ghat=Ghat, F=F, Y=Y, omega=omega, W=W)
    return Y.real


def reconstruct_adjoint(xy, h, fbar, dt, c, grid, nt, full=False):
    """Exact transpose of reconstruct (as a real-linear map g -> f)."""
    omega, W = omega_and_weight(grid, c)
    Fbar = image_transform_adjoint(fbar, grid)
    Ghatbar = (dt / grid.dz) * W * Fbar
    G1bar = time_transform_adjoint(Ghatbar, omega, dt, nt)
    gbar = data_transform_adjoint(xy, h, G1bar, grid)
    if full:
        return gbar, dict(G1bar=G1bar)
    return gbar


def position_grad(xy, h, g, fbar, dt, c, grid):
    """Gradient of L = <fbar, reconstruct(xy, h, g)> with respect to the sensor
    positions (M, 2), holding h fixed.

    Only G1 depends on x_m: dG1(j, n)/dx_m = -i kx a_m g[m, n] E(j, m), so
    dL/dx_m = Re sum_{j,n} conj(G1bar(j, n)) (-i kx) a_m g[m, n] E(j, m), with
    G1bar the cotangent of G1 from the transposed chain."""
    nt = g.shape[1]
    _, aux = reconstruct_adjoint(xy, h, fbar, dt, c, grid, nt, full=True)
    return position_grad_from_cotangent(xy, h, g, aux["G1bar"], grid)


def position_grad_from_cotangent(xy, h, g, G1bar, grid):
    """The last step of position_grad: dL/dx_m and dL/dy_m from the cotangent
    G1bar(j, n) of the spatial spectrum (on the index sets of Sec. 2), for the
    sensors xy given (any subset: each row depends on its own sensor only)."""
    nt = g.shape[1]
    a = h / (grid.dx * grid.dy)
    kx, ky, _ = wavenumbers(grid)
    Ex, Ey = spatial_factors(xy, grid)
    Dx = np.zeros((xy.shape[0], nt), dtype=np.complex128)
    Dy = np.zeros((xy.shape[0], nt), dtype=np.complex128)
    for ix in range(grid.nx):
        E = Ey * Ex[ix][None, :]                        # (ny, M)
        C = G1bar[ix].conj()                             # (ny, nt)
        Dx += (-1j * kx[ix]) * (E.T @ C)
        Dy += (E * (-1j * ky)[:, None]).T @ C
    gx = a * np.sum(g * Dx.real, axis=1)
    gy = a * np.sum(g * Dy.real, axis=1)
    return np.stack([gx, gy], axis=1)


# ---------------------------------------------------------------------------
# Single columns and single voxels, for checks at sizes where the full dense
# sums are out of reach.

def column_spectrum(xy, h, g, dt, c, grid, jx, jy):
    """F(j, l) = (dt/dz) W(j, l) sum_n G1(j, n) exp(-i omega(j, l) n dt) for one
    column of integer frequencies j = (jx, jy) and every l in freqs(nz)."""
    nt = g.shape[1]
    a = h / (grid.dx * grid.dy)
    Ex, Ey = spatial_factors(xy, grid, [jx], [jy])
    E = Ex[0] * Ey[0]                                             # (M,)
    ag = a[:, None] * g                                           # real (M, nt)
    G = E.real @ ag + 1j * (E.imag @ ag)                          # G1(j, n)
    l = freqs(grid.nz)
    kx = 2 * np.pi * jx / (grid.nx * grid.dx)
    ky = 2 * np.pi * jy / (grid.ny * grid.dy)
    kz = 2 * np.pi * l / (grid.nz * grid.dz)
    omega, W = omega_weight_at(kx, ky, kz, c)
    t = np.arange(nt) * dt
    Ghat = np.exp(-1j * np.outer(omega, t)) @ G
    return (dt / grid.dz) * W * Ghat


def column_depth_profile(xy, h, g, dt, c, grid, jx, jy):
    """(1/(nx ny nz)) sum_l Fsym(j, l) exp(i kz z_k), k = 0..nz-1, for one column
    j of the index sets, where Fsym(k) = (F(k) + conj F(-k mod N)) / 2 is the
    Hermitian part of F (its inverse DFT is the real part of F's)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    F = column_spectrum(xy, h, g, dt, c, grid, jx, jy)
    Fm = column_spectrum(xy, h, g, dt, c, grid, int(wrap_index(-jx, nx)), int(wrap_index(-jy, ny)))
    l = freqs(nz)
    Fsym = 0.5 * (F + np.conj(Fm[wrap_index(-l, nz) - l[0]]))
    z = np.arange(nz) * grid.dz
    kz = 2 * np.pi * l / (nz * grid.dz)
    return (np.exp(1j * np.outer(z, kz)) @ Fsym) / (nx * ny * nz)


def half_spectrum_voxels(half, grid, pts):
    """f[p, q, k] at the voxels pts (P x 3 integers) from a Hermitian half
    spectrum half[ix][iy][k] over jx = ix - floor(nx/2) (all nx) and jy = iy
    (iy = 0..floor(ny/2); for even ny the last entry is the unpaired
    jy = -ny/2): f = sum over the whole (jx, jy) plane of S(j, k)
    exp(i (kx x_p + ky y_q)), with S(jx, -jy) = conj S(-jx, jy) off the stored
    half."""
    nx, ny = grid.nx, grid.ny
    hx, hy = nx // 2, ny // 2
    jxs, jys = freqs(nx), freqs(ny)
    S = np.empty((nx, ny, half.shape[2]), dtype=np.complex128)
    for a, jx in enumerate(jxs):
        for b, jy in enumerate(jys):
            if jy >= 0:
                S[a, b] = half[jx + hx, jy]
            elif ny % 2 == 0 and jy == -hy:
                S[a, b] = half[jx + hx, hy]
            else:
                S[a, b] = np.conj(half[int(wrap_index(-jx, nx)) + hx, -jy])
    kx = 2 * np.pi * jxs / (nx * grid.dx)
    ky = 2 * np.pi * jys / (ny * grid.dy)
    out = np.empty(len(pts))
    for i, (p, q, k) in enumerate(pts):
        x = (p - hx) * grid.dx
        y = (q - hy) * grid.dy
        E = np.exp(1j * np.add.outer(kx * x, ky * y))
        out[i] = np.sum(E * S[:, :, k]).real
    return out


# ---------------------------------------------------------------------------
# The d = 2 operator (Sec. 2 with d - 1 = 1: sensors on the line z = 0 at
# x_m, images f[p, k]).  eq:disc_rec for d = 2 is the general formula with a
# one-dimensional x: a_m = h_m / dx, G1(jx, n) = sum_m a_m g[m, n]
# exp(-i kx x_m), omega and W as above with ky = 0, and
# f[p, k] = Re 1/(nx nz) sum_{jx,l} F(jx, l) exp(i (kx x_p + kz z_k)).  The
# functions below evaluate exactly that through the general sums on a grid
# with one y row of unit spacing (ny = 1, dy = 1: the y index set is {0}, so
# ky = 0, a_m = h_m/(dx * 1) and 1/(nx * 1 * nz)).

class Grid2:
    """(nx, nz, dx, dz) of the d = 2 operator, seen as the general grid with
    one y row of unit spacing."""

    def __init__(self, nx, nz, dx, dz):
        self.nx, self.ny, self.nz = int(nx), 1, int(nz)
        self.dx, self.dy, self.dz = float(dx), 1.0, float(dz)

    @property
    def shape(self):
        return (self.nx, self.nz)

    def as_tuple(self):
        return (self.nx, self.ny, self.nz, self.dx, self.dy, self.dz)


def _line(x):
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    return np.stack([x, np.zeros_like(x)], axis=1)


def reconstruct_2d(x, h, g, dt, c, grid2):
    """f[p, k] of the d = 2 operator; x: (M,) positions, h: (M,) lengths."""
    return reconstruct(_line(x), h, g, dt, c, grid2)[:, 0, :]


def reconstruct_adjoint_2d(x, h, fbar, dt, c, grid2, nt):
    """Exact transpose of reconstruct_2d."""
    return reconstruct_adjoint(_line(x), h, np.asarray(fbar)[:, None, :], dt, c, grid2, nt)


def position_grad_2d(x, h, g, fbar, dt, c, grid2):
    """d/dx_m of <fbar, reconstruct_2d(x, h, g)>, shape (M,)."""
    return position_grad(_line(x), h, g, np.asarray(fbar)[:, None, :], dt, c, grid2)[:, 0]


def weight_grad(xy, h, g, fbar, dt, c, grid):
    """Gradient of L = <fbar, reconstruct(xy, h, g)> with respect to the
    weights h (M,): reconstruct is linear in h, so dL/dh_m = (1/h_m)
    sum_n g[m, n] (reconstruct_adjoint(fbar))[m, n]."""
    gb = reconstruct_adjoint(xy, h, fbar, dt, c, grid, g.shape[1])
    return np.sum(g * gb, axis=1) / h
