"""Checks that pin the oracle to facts outside itself.

Each function returns an error measure (0 means agreement) so that the pin
tests can assert on it and the mutation tests can show that a planted mistake
in the oracle makes it large.  None of these retypes the oracle's formula:
they compare it with numpy's FFT on special cases that reduce to one, with
closed forms of the wave equation, with exact invariants of the discrete sum,
or with finite differences.
"""
from __future__ import annotations

import numpy as np

import synth
from oracle import ndft, nufft


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def lattice_problem(nx=12, ny=10, nt=6, seed=3, dx=1e-4, dy=1.3e-4):
    """Sensors exactly on the output lattice, h = dx dy, random data."""
    rng = np.random.default_rng(seed)
    xy = synth.lattice_positions(nx, ny, dx, dy)
    g = rng.normal(size=(nx * ny, nt))
    h = np.full(nx * ny, dx * dy)
    grid = synth.Grid(nx, ny, 8, dx, dy, 1e-4)
    return xy, h, g, grid


def pin_lattice_fft2(data_transform=None):
    """Sensors on the lattice (eq:equiv_rec from eq:disc_rec, Sec. 2): the
    spatial transform is a plain 2D DFT of the data rolled so that the sensor
    at x = 0 sits at index 0.  Compared with numpy.fft.fft2."""
    xy, h, g, grid = lattice_problem()
    nx, ny, nt = grid.nx, grid.ny, g.shape[1]
    if data_transform is None:
        G1 = ndft.data_transform(xy, h, g, grid)
    else:
        G1 = data_transform(xy, h, g, grid)
    d = g.reshape(nx, ny, nt)
    d = np.roll(d, (-(nx // 2), -(ny // 2)), axis=(0, 1))
    D = np.fft.fft2(d, axes=(0, 1))
    jx, jy = ndft.freqs(nx), ndft.freqs(ny)
    ref = D[np.ix_(jx % nx, jy % ny)]
    return rel(G1, ref)


def integer_tau_setup(nt=16):
    """Grid with X = Y = Z = c nt dt, so tau(j, l) = sign(l) |(jx, jy, l)|."""
    c = 1500.0
    dt = 20e-9
    L = c * nt * dt
    n = 16
    grid = synth.Grid(n, n, n, L / n, L / n, L / n)
    return c, dt, grid


# (jx, jy, l) with integer Euclidean norm: tau is an integer and the
# non-uniform time transform must equal an FFT bin.
INTEGER_TRIPLES = [(0, 0, 3), (0, 0, -5), (3, 4, 0), (0, 3, 4), (4, 0, -3), (2, 3, 6),
                   (-2, 3, -6), (1, 2, 2), (-1, -2, -2), (2, -1, 2), (0, 0, 0), (-6, 3, 2)]


def pin_integer_tau(time_transform_at=None):
    """At integer tau the time transform is a DFT bin of the column; the sign
    of tau follows l (Sec. 2: kappa = sign(K_y) |K|)."""
    nt = 16
    c, dt, grid = integer_tau_setup(nt)
    rng = np.random.default_rng(11)
    omega, _ = ndft.omega_and_weight(grid, c)
    errs = []
    for (jx, jy, l) in INTEGER_TRIPLES:
        col = rng.normal(size=nt) + 1j * rng.normal(size=nt)
        ix, iy, il = jx + grid.nx // 2, jy + grid.ny // 2, l + grid.nz // 2
        tau_int = int(np.sign(l) if l != 0 else 1) * int(round(np.sqrt(jx * jx + jy * jy + l * l)))
        ref = np.fft.fft(col)[tau_int % nt]
        if time_transform_at is None:
            G1 = np.zeros((grid.nx, grid.ny, nt), dtype=complex)
            G1[ix, iy] = col
            val = ndft.time_transform(G1, omega, dt)[ix, iy, il]
        else:
            val = time_transform_at(col, omega[ix, iy, il], dt)
        errs.append(abs(val - ref) / abs(ref))
    return max(errs)


def pin_plane_wave(reconstruct=None, halfstep=False):
    """Laterally uniform source F(z) (Gaussian) seen by a full lattice of
    sensors: every sensor records F(c t)/2 (1D d'Alembert).  The
    reconstruction must return F(z_k) at every (x, y): this fixes the weight
    2c at K = (0, 0, kz), the factor dt/dz, the 1/N of the inverse DFT and the
    sign pairing of omega with kz (a wrong sign mirrors F)."""
    nx, ny, nz = 6, 4, 48
    dz = 1e-4
    c = 1500.0
    if halfstep:
        dt, nt = dz / (2 * c), 2 * nz
    else:
        dt, nt = dz / c, nz
    grid = synth.Grid(nx, ny, nz, 1e-4, 1.2e-4, dz)
    xy = synth.lattice_positions(nx, ny, grid.dx, grid.dy)
    M = xy.shape[0]
    h = np.full(M, nx * grid.dx * ny * grid.dy / M)
    F = synth.gaussian_profile(1.6e-3, 2.2e-4, 1.0)
    g = synth.plane_profile_data(M, nt, dt, c, F)
    if reconstruct is None:
        f = ndft.reconstruct(xy, h, g, dt, c, grid)
    else:
        f = reconstruct(xy, h, g, dt, c, grid)
    ref = np.broadcast_to(F(np.arange(nz) * dz)[None, None, :], f.shape)
    return rel(f, ref)


def pin_depth_sum(reconstruct=None):
    """sum_k f[p, q, k] does not depend on (p, q): only l = 0 survives the sum
    over z and W(j != 0, 0) = 0 there.  Returns the spread of the sums
    relative to the image norm."""
    P = synth.tiny()
    rng = np.random.default_rng(5)
    g = rng.normal(size=P.g.shape)
    rec = reconstruct or ndft.reconstruct
    f = rec(P.xy, P.h, g, P.dt, P.c, P.grid)
    s = f.sum(axis=2)
    return float(np.abs(s - s.mean()).max() / np.linalg.norm(f))


def pin_shift_roll(reconstruct=None):
    """Moving every sensor by +dx rolls the image by one voxel along x, moving
    by X leaves it unchanged (the discrete sum is X-periodic)."""
    P = synth.tiny()
    rec = reconstruct or ndft.reconstruct
    f0 = rec(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    xy1 = P.xy + np.array([P.grid.dx, 0.0])
    f1 = rec(xy1, P.h, P.g, P.dt, P.c, P.grid)
    xy2 = P.xy + np.array([0.0, P.grid.ny * P.grid.dy])
    f2 = rec(xy2, P.h, P.g, P.dt, P.c, P.grid)
    return max(rel(f1, np.roll(f0, 1, axis=0)), rel(f2, f0))


def pin_adjoint_dot(reconstruct, reconstruct_adjoint, problem=None, seed=7):
    """|<A g, f> - <g, A^T f>| / (|A g| |f|)."""
    P = problem or synth.tiny()
    rng = np.random.default_rng(seed)
    g = rng.normal(size=P.g.shape)
    fb = rng.normal(size=P.grid.shape)
    Ag = reconstruct(P.xy, P.h, g, P.dt, P.c, P.grid)
    Atf = reconstruct_adjoint(P.xy, P.h, fb, P.dt, P.c, P.grid, P.g.shape[1])
    return abs(float(np.sum(Ag * fb)) - float(np.sum(g * Atf))) / (np.linalg.norm(Ag) * np.linalg.norm(fb))


def pin_position_grad_fd(position_grad=None, n_coords=12, seed=9):
    """Analytic position gradient vs FP64 central differences of
    L(x) = <fbar, reconstruct(x)>."""
    P = synth.tiny()
    rng = np.random.default_rng(seed)
    fb = rng.normal(size=P.grid.shape)
    pg = position_grad or ndft.position_grad
    G = pg(P.xy, P.h, P.g, fb, P.dt, P.c, P.grid)

    def L(xy):
        return float(np.sum(fb * ndft.reconstruct(xy, P.h, P.g, P.dt, P.c, P.grid)))

    eps = 1e-6 * P.grid.dx
    errs = []
    idx = rng.choice(P.xy.shape[0], size=n_coords, replace=False)
    scale = np.abs(G).max()
    for m in idx:
        for a in (0, 1):
            xp = P.xy.copy()
            xm = P.xy.copy()
            xp[m, a] += eps
            xm[m, a] -= eps
            fd = (L(xp) - L(xm)) / (2 * eps)
            errs.append(abs(fd - G[m, a]) / scale)
    # random direction
    d = rng.normal(size=P.xy.shape)
    fd = (L(P.xy + eps * d) - L(P.xy - eps * d)) / (2 * eps)
    errs.append(abs(fd - np.sum(G * d)) / (scale * np.linalg.norm(d)))
    return max(errs)


# --------------------------------------------------------------- d = 2 pins
def pin_plane_wave_2d():
    """d = 2: a laterally uniform source F(z) seen by sensors on every x node
    records F(c t)/2 (1-D d'Alembert, the same in any dimension); the 2-D
    reconstruction returns F(z_k) at every x."""
    nx, nz, dz, c = 6, 48, 1e-4, 1500.0
    dt, nt = dz / c, nz
    grid = ndft.Grid2(nx, nz, 1e-4, dz)
    x = (np.arange(nx) - nx // 2) * grid.dx
    h = np.full(nx, grid.dx)
    F = synth.gaussian_profile(1.6e-3, 2.2e-4, 1.0)
    g = synth.plane_profile_data(nx, nt, dt, c, F)
    f = ndft.reconstruct_2d(x, h, g, dt, c, grid)
    ref = np.broadcast_to(F(np.arange(nz) * dz)[None, :], f.shape)
    return rel(f, ref)


def pin_2d_is_y_invariant_3d():
    """Data that do not depend on y, recorded by every y node of a full y
    lattice, reconstruct in 3-D to the same image at every y; with ky = 0
    alone surviving, that image is the d = 2 reconstruction of the data along
    one row (weights h_m dy per 3-D sensor)."""
    rng = np.random.default_rng(21)
    nx, ny, nz, nt = 7, 5, 12, 20
    dx, dy, dz, c, dt = 1e-4, 1.3e-4, 1e-4, 1500.0, 3e-8
    x = (np.arange(nx) - nx // 2) * dx + rng.uniform(-0.4, 0.4, nx) * dx
    hx = rng.uniform(0.5, 1.5, nx) * dx
    g = rng.normal(size=(nx, nt))
    y = (np.arange(ny) - ny // 2) * dy
    xy = np.array([(xm, yq) for xm in x for yq in y])
    h3 = np.array([hm * dy for hm in hx for _ in y])
    g3 = np.repeat(g, ny, axis=0)
    f3 = ndft.reconstruct(xy, h3, g3, dt, c, synth.Grid(nx, ny, nz, dx, dy, dz))
    f2 = ndft.reconstruct_2d(x, hx, g, dt, c, ndft.Grid2(nx, nz, dx, dz))
    return max(rel(f3[:, q, :], f2) for q in range(ny))


def pin_adjoint_dot_2d():
    rng = np.random.default_rng(22)
    nx, nz, nt = 9, 14, 24
    grid = ndft.Grid2(nx, nz, 1e-4, 1e-4)
    x = (np.arange(nx) - nx // 2) * grid.dx + rng.uniform(-0.4, 0.4, nx) * grid.dx
    h = rng.uniform(0.5, 1.5, nx) * grid.dx
    g = rng.normal(size=(nx, nt))
    fb = rng.normal(size=(nx, nz))
    dt, c = 2e-8, 1500.0
    lhs = np.vdot(ndft.reconstruct_2d(x, h, g, dt, c, grid), fb)
    rhs = np.vdot(g, ndft.reconstruct_adjoint_2d(x, h, fb, dt, c, grid, nt))
    return abs(lhs - rhs) / max(abs(lhs), abs(rhs))


def pin_position_grad_2d():
    """FP64 central differences of <fbar, f(x)> against position_grad_2d."""
    rng = np.random.default_rng(23)
    nx, nz, nt = 8, 10, 16
    grid = ndft.Grid2(nx, nz, 1e-4, 1e-4)
    x = (np.arange(nx) - nx // 2) * grid.dx + rng.uniform(-0.4, 0.4, nx) * grid.dx
    h = np.full(nx, grid.dx)
    g = rng.normal(size=(nx, nt))
    fb = rng.normal(size=(nx, nz))
    dt, c = 2e-8, 1500.0
    grad = ndft.position_grad_2d(x, h, g, fb, dt, c, grid)
    eps = 1e-9
    fd = np.empty(nx)
    for m in range(nx):
        xp, xm = x.copy(), x.copy()
        xp[m] += eps
        xm[m] -= eps
        fd[m] = (np.vdot(fb, ndft.reconstruct_2d(xp, h, g, dt, c, grid)) -
                 np.vdot(fb, ndft.reconstruct_2d(xm, h, g, dt, c, grid))) / (2 * eps)
    return rel(grad, fd)
