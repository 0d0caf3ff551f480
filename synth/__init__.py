"""Seeded synthetic inputs for planar-sensor photoacoustic reconstruction.

This module generates sensor layouts, phantoms and the pressure data those
phantoms produce on the plane z = 0.  It holds none of the reconstruction
method's arithmetic: it is the *forward physics* (closed-form solutions of the
wave equation of Sec. 2) plus random layouts.  Both the CPU oracle and the GPU
path consume what it returns, so neither side generates its own inputs.

Conventions (Sec. 2, grids G_x and G_y):
  * sensors lie on z = 0 at positions (x_m, y_m) in metres, centred on (0, 0);
  * data g[m, n] = p(x_m, y_m, 0, t_n) with t_n = n * dt, n = 0 .. n_t - 1;
  * the output grid has voxel centres x_p = (p - floor(nx/2)) * dx,
    y_q = (q - floor(ny/2)) * dy and z_k = k * dz.

Physics used for the data (Sec. 2, the initial value problem with
p(., 0) = f and d/dt p(., 0) = 0, sound speed c):
  * a uniform ball of radius R and amplitude p0 seen at distance r gives the
    N-shaped signal p(r, t) = p0 * (r - c t) / (2 r) for |r - c t| < R, else 0
    (d'Alembert's solution for r*p with the radial profile extended evenly);
  * a laterally uniform source f(x, y, z) = F(z) (z > 0) gives
    p(x, y, 0, t) = F(c t) / 2 at every sensor.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

C_WATER = 1500.0  # m/s


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)

    def as_tuple(self):
        return (self.nx, self.ny, self.nz, self.dx, self.dy, self.dz)


@dataclass
class Problem:
    """One reconstruction problem: sensors, data and output grid."""
    name: str
    xy: np.ndarray          # (M, 2) float64, metres
    h: np.ndarray           # (M,) float64, detector areas in m^2 (sum = X*Y)
    g: np.ndarray           # (M, n_t) float64 pressure samples
    dt: float
    c: float
    grid: Grid
    sigma: int = 2
    width: int = 8
    balls: list = field(default_factory=list)   # (x, y, z, R, p0) tuples

    @property
    def n_sensors(self):
        return self.xy.shape[0]

    @property
    def n_t(self):
        return self.g.shape[1]

    def voxelised(self):
        """The phantom sampled at voxel centres (sum of the balls)."""
        return voxelise_balls(self.balls, self.grid)


# --------------------------------------------------------------------------
# sensor layouts
# --------------------------------------------------------------------------

def lattice_positions(nsx, nsy, pitch_x, pitch_y):
    """Regular lattice x = (i - floor(nsx/2)) * pitch_x, same for y."""
    ix = np.arange(nsx) - nsx // 2
    iy = np.arange(nsy) - nsy // 2
    X, Y = np.meshgrid(ix * pitch_x, iy * pitch_y, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)


def jittered_lattice(rng, nsx, nsy, pitch_x, pitch_y, jitter=0.4):
    """Lattice with each coordinate jittered uniformly by +-jitter*pitch."""
    xy = lattice_positions(nsx, nsy, pitch_x, pitch_y)
    xy[:, 0] += rng.uniform(-jitter, jitter, xy.shape[0]) * pitch_x
    xy[:, 1] += rng.uniform(-jitter, jitter, xy.shape[0]) * pitch_y
    return xy


def centre_dense_positions(rng, n, half_width, r_dense, ratio=2.0):
    """n points in the square [-hw, hw)^2 by rejection sampling from a density
    that is `ratio` times higher inside r < r_dense than outside."""
    out = np.empty((0, 2))
    while out.shape[0] < n:
        cand = rng.uniform(-half_width, half_width, size=(2 * n, 2))
        r = np.hypot(cand[:, 0], cand[:, 1])
        accept_p = np.where(r < r_dense, 1.0, 1.0 / ratio)
        keep = rng.uniform(size=cand.shape[0]) < accept_p
        out = np.concatenate([out, cand[keep]], axis=0)
    return out[:n].copy()


def dart_throwing(rng, n, half_width, r_min):
    """n uniform random points in [-hw, hw)^2 with pairwise distance >= r_min
    (dart throwing with a background grid of cell size r_min/sqrt(2), so each
    cell holds at most one point)."""
    cell = r_min / math.sqrt(2.0)
    ncell = int(math.ceil(2 * half_width / cell))
    occ = -np.ones((ncell, ncell), dtype=np.int64)
    pts = np.empty((n, 2))
    count = 0
    r2 = r_min * r_min
    while count < n:
        cand = rng.uniform(-half_width, half_width, size=(4096, 2))
        for x, y in cand:
            ci = min(int((x + half_width) / cell), ncell - 1)
            cj = min(int((y + half_width) / cell), ncell - 1)
            if occ[ci, cj] >= 0:
                continue
            ok = True
            for a in range(max(ci - 2, 0), min(ci + 3, ncell)):
                row = occ[a]
                for b in range(max(cj - 2, 0), min(cj + 3, ncell)):
                    k = row[b]
                    if k >= 0:
                        dx = pts[k, 0] - x
                        dy = pts[k, 1] - y
                        if dx * dx + dy * dy < r2:
                            ok = False
                            break
                if not ok:
                    break
            if ok:
                occ[ci, cj] = count
                pts[count] = (x, y)
                count += 1
                if count == n:
                    break
    return pts


# --------------------------------------------------------------------------
# phantoms and their data
# --------------------------------------------------------------------------

def ball_signal(xy, t, ball, c):
    """Closed-form pressure of one uniform ball at sensors xy, times t.

    p(r, t) = p0 (r - c t) / (2 r) when |r - c t| < R, else 0 (sensor outside
    the ball).  Returns an (M, len(t)) array.
    """
    bx, by, bz, R, p0 = ball
    r = np.sqrt((xy[:, 0] - bx) ** 2 + (xy[:, 1] - by) ** 2 + bz ** 2)[:, None]
    s = r - c * np.asarray(t)[None, :]
    return np.where(np.abs(s) < R, p0 * s / (2.0 * r), 0.0)


def balls_data(xy, n_t, dt, balls, c, chunk=1024):
    """Sum of closed-form ball signals (linear superposition), float64.

    Only the samples with |r - c t_n| < R are touched: per ball, each sensor's
    K candidate samples n_lo .. n_lo + K - 1 (n_lo = ceil((r - R) / (c dt)))
    are evaluated at once as an array, for blocks of `chunk` sensors whose
    rows of g stay in cache while every ball is added (in ball order).
    """
    M = xy.shape[0]
    g = np.zeros((M, n_t))
    for a in range(0, M, chunk):
        b = min(M, a + chunk)
        gc = g[a:b]
        xs, ys = xy[a:b, 0], xy[a:b, 1]
        for (bx, by, bz, R, p0) in balls:
            r = np.sqrt((xs - bx) ** 2 + (ys - by) ** 2 + bz ** 2)
            n_lo = np.ceil((r - R) / (c * dt)).astype(np.int64)
            K = int(math.ceil(2 * R / (c * dt))) + 2
            live = np.nonzero((n_lo < n_t) & (n_lo + K > 0))[0]
            if live.size == 0:
                continue
            rl = r[live][:, None]
            n = n_lo[live][:, None] + np.arange(K)[None, :]
            s = rl - c * (n * dt)
            ok = (np.abs(s) < R) & (n >= 0) & (n < n_t)
            m = np.broadcast_to(live[:, None], n.shape)[ok]
            gc[m, n[ok]] += p0 * s[ok] / (2.0 * np.broadcast_to(rl, n.shape)[ok])
    return g


def voxelise_balls(balls, grid: Grid):
    """Phantom sampled at voxel centres: sum of p0 * [inside ball]."""
    x = (np.arange(grid.nx) - grid.nx // 2) * grid.dx
    y = (np.arange(grid.ny) - grid.ny // 2) * grid.dy
    z = np.arange(grid.nz) * grid.dz
    f = np.zeros(grid.shape)
    for (bx, by, bz, R, p0) in balls:
        ix = np.nonzero(np.abs(x - bx) <= R)[0]
        iy = np.nonzero(np.abs(y - by) <= R)[0]
        iz = np.nonzero(np.abs(z - bz) <= R)[0]
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        X, Y, Z = np.meshgrid(x[ix], y[iy], z[iz], indexing="ij")
        inside = (X - bx) ** 2 + (Y - by) ** 2 + (Z - bz) ** 2 <= R * R
        f[np.ix_(ix, iy, iz)] += p0 * inside
    return f


def plane_profile_data(M, n_t, dt, c, profile):
    """Laterally uniform source f = F(z): every sensor sees F(c t_n) / 2."""
    t = np.arange(n_t) * dt
    g1 = 0.5 * profile(c * t)
    return np.repeat(g1[None, :], M, axis=0)


def random_balls(rng, n, xy_half, z_range, r_range, p_range):
    balls = []
    for _ in range(n):
        balls.append((rng.uniform(-xy_half, xy_half), rng.uniform(-xy_half, xy_half),
                      rng.uniform(*z_range), rng.uniform(*r_range), rng.uniform(*p_range)))
    return balls


def vessel_balls(rng, n_vessels, xy_half, z_range, rad_range, len_range, p0=1.0):
    """Cylinders as chains of balls spaced at half the radius (no closed form
    exists for a finite cylinder, so the chain's superposition stands in)."""
    balls = []
    for _ in range(n_vessels):
        rad = rng.uniform(*rad_range)
        length = rng.uniform(*len_range)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        c0 = np.array([rng.uniform(-xy_half, xy_half), rng.uniform(-xy_half, xy_half),
                       rng.uniform(*z_range)])
        nb = max(int(length / (0.5 * rad)), 1)
        for i in range(nb):
            p = c0 + (i - nb / 2) * 0.5 * rad * d
            if p[2] <= rad * 1.5:
                continue
            balls.append((float(p[0]), float(p[1]), float(p[2]), rad, p0 * 0.25))
    return balls


def _uniform_weights(M, X, Y):
    return np.full(M, X * Y / M)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def tiny(seed=1500, n_t=32):
    """8x8 jittered sensors, n_t=32 samples, 8x8x16 output at 100 um; one
    ball.  Small enough for the brute-force non-uniform DFT."""
    rng = np.random.default_rng(seed)
    pitch = 1e-4
    xy = jittered_lattice(rng, 8, 8, pitch, pitch)
    grid = Grid(8, 8, 16, pitch, pitch, pitch)
    c, dt = C_WATER, 40e-9
    balls = [(0.0, 0.0, 0.6e-3, 0.25e-3, 1.0)]
    g = balls_data(xy, n_t, dt, balls, c)
    return Problem("tiny_8x8x16", xy, _uniform_weights(64, 8 * pitch, 8 * pitch), g, dt, c,
                   grid, balls=balls)


def c1(seed=1501):
    """32x32 sensors at 100 um pitch, +-0.4 pitch jitter; 128 samples at
    dt = 20 ns; one ball R = 0.4 mm, p0 = 1 at (0, 0, 1.5 mm); output
    32x32x64 at 100 um; sigma = 2, width 8."""
    rng = np.random.default_rng(seed)
    pitch = 1e-4
    xy = jittered_lattice(rng, 32, 32, pitch, pitch)
    grid = Grid(32, 32, 64, pitch, pitch, pitch)
    c, dt = C_WATER, 20e-9
    balls = [(0.0, 0.0, 1.5e-3, 0.4e-3, 1.0)]
    g = balls_data(xy, 128, dt, balls, c)
    X = grid.nx * grid.dx
    return Problem("c1_32x32x64", xy, _uniform_weights(xy.shape[0], X, X), g, dt, c, grid,
                   balls=balls)


def c2(seed=1502, noise=True):
    """16384 sensors over 12.8 mm: 8192 on a jittered 128x64 lattice (pitch
    100 x 200 um) plus 8192 drawn with twice the density inside r < 3.2 mm;
    512 samples at dt = 20 ns; 20 random balls (R 0.1-0.5 mm, p0 in
    U[0.5, 1], x, y in +-4.8 mm, z in 1-6 mm) plus Gaussian noise of 1 % of
    the peak; output 128x128x256 at 100 um."""
    rng = np.random.default_rng(seed)
    half = 6.4e-3
    a = jittered_lattice(rng, 128, 64, 1e-4, 2e-4)
    b = centre_dense_positions(rng, 8192, half, 3.2e-3, 2.0)
    xy = np.concatenate([a, b], axis=0)
    grid = Grid(128, 128, 256, 1e-4, 1e-4, 1e-4)
    c, dt = C_WATER, 20e-9
    balls = random_balls(rng, 20, 4.8e-3, (1e-3, 6e-3), (1e-4, 5e-4), (0.5, 1.0))
    g = balls_data(xy, 512, dt, balls, c)
    if noise:
        g += rng.normal(0.0, 0.01 * np.abs(g).max(), size=g.shape)
    X = grid.nx * grid.dx
    return Problem("c2_128x128x256", xy, _uniform_weights(xy.shape[0], X, X), g, dt, c, grid,
                   balls=balls)


def c3(seed=1503, n_vessels=6):
    """65536 random-uniform sensors over 25.6 mm with minimum spacing 40 um;
    1024 samples at dt = 10 ns; balls plus vessels; output 256x256x512 at
    100 um."""
    rng = np.random.default_rng(seed)
    half = 12.8e-3
    xy = dart_throwing(rng, 65536, half, 4e-5)
    grid = Grid(256, 256, 512, 1e-4, 1e-4, 1e-4)
    c, dt = C_WATER, 10e-9
    balls = random_balls(rng, 20, 9.6e-3, (1e-3, 8e-3), (1e-4, 5e-4), (0.5, 1.0))
    balls += vessel_balls(rng, n_vessels, 8e-3, (2e-3, 8e-3), (5e-5, 1.5e-4), (2e-3, 8e-3))
    g = balls_data(xy, 1024, dt, balls, c)
    X = grid.nx * grid.dx
    return Problem("c3_256x256x512", xy, _uniform_weights(xy.shape[0], X, X), g, dt, c, grid,
                   balls=balls)


def seven_smooth(lo, hi):
    out = []
    for n in range(lo, hi + 1):
        m = n
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


def batch_instance(rng, n_side, n_t, name="batch", n_balls=5, dt=20e-9):
    """One instance of the uneven batch: n_side^2 jittered sensors at 100 um,
    n_t samples at dt = 20 ns, output n_side x n_side x 2 n_t at 100 um."""
    pitch = 1e-4
    xy = jittered_lattice(rng, n_side, n_side, pitch, pitch)
    grid = Grid(n_side, n_side, 2 * n_t, pitch, pitch, pitch)
    half = 0.35 * n_side * pitch
    zmax = min(0.6 * C_WATER * n_t * dt, 6e-3)
    balls = random_balls(rng, n_balls, half, (0.5e-3, zmax), (1e-4, 5e-4), (0.5, 1.0))
    g = balls_data(xy, n_t, dt, balls, C_WATER)
    X = n_side * pitch
    return Problem(f"{name}_{n_side}x{n_side}x{2 * n_t}", xy,
                   _uniform_weights(xy.shape[0], X, X), g, dt, C_WATER, grid, balls=balls)


def batch_shapes(seed=1505, n=64, lo=64, hi=256, t_choices=(256, 512, 1024)):
    """Sizes of the uneven batch: N uniform over the 7-smooth integers in
    [lo, hi], T uniform over t_choices."""
    rng = np.random.default_rng(seed)
    sizes = seven_smooth(lo, hi)
    return [(int(rng.choice(sizes)), int(rng.choice(t_choices))) for _ in range(n)]


def batch(seed=1505, n=64, lo=64, hi=256, t_choices=(256, 512, 1024), n_balls=5):
    rng = np.random.default_rng(seed + 1000)
    return [batch_instance(rng, N, T, n_balls=n_balls)
            for (N, T) in batch_shapes(seed, n, lo, hi, t_choices)]


def gaussian_profile(z0, s, p0=1.0):
    return lambda z: p0 * np.exp(-0.5 * ((z - z0) / s) ** 2)


def correlation_coefficient(u1, u2):
    """Correlation coefficient Cov(U1, U2) / sqrt(Var U1 Var U2) (App. B)."""
    a = np.asarray(u1, dtype=np.float64).ravel()
    b = np.asarray(u2, dtype=np.float64).ravel()
    a = a - a.mean()
    b = b - b.mean()
    return float((a @ b) / math.sqrt((a @ a) * (b @ b)))
