"""Device Voronoi weights (pa_voronoi_weights / pa_voronoi_grad) against the
oracle's periodic Voronoi cells, and the gradient through position-dependent
weights end to end: d/dx of <fbar, A(x, h(x)) g> with h the Voronoi areas,
from pa_position_grad + pa_weight_grad + pa_voronoi_grad, against FP64
central differences of the direct sums."""
import numpy as np
import pytest
import torch

import synth
from oracle import ndft, voronoi

from test_gpu_parity import TOL, dev, host, pa, rel

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy.spatial")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def reduce(xy, X, Y):
    out = xy.copy()
    out[:, 0] -= X * np.floor(out[:, 0] / X + 0.5)
    out[:, 1] -= Y * np.floor(out[:, 1] / Y + 0.5)
    return out


@pytest.mark.parametrize("layout", ["c1", "c2", "random", "clustered"])
def test_voronoi_areas_match_oracle(layout):
    rng = np.random.default_rng(5)
    if layout in ("c1", "c2"):
        P = getattr(synth, layout)()
        xy, grid, nt, dt, c = P.xy, P.grid, P.n_t, P.dt, P.c
    else:
        grid = synth.Grid(32, 24, 16, 1e-4, 1e-4, 1e-4)
        X, Y = grid.nx * grid.dx, grid.ny * grid.dy
        if layout == "random":
            xy = np.stack([rng.uniform(-X, X, 300), rng.uniform(-Y, Y, 300)], 1)
        else:
            xy = np.concatenate([rng.normal(0, 3e-4, (150, 2)), np.stack([rng.uniform(-X / 2, X / 2, 50),
                                                                             rng.uniform(-Y / 2, Y / 2, 50)], 1)])
        nt, dt, c = 32, 20e-9, 1500.0
    X, Y = grid.nx * grid.dx, grid.ny * grid.dy
    plan = pa().Plan(xy, nt, dt, c, grid.as_tuple())
    h = host(plan.voronoi_weights())
    ref = voronoi.areas_2d(reduce(xy, X, Y), X, Y)
    err = rel(h, ref)
    print(f"{layout}: Voronoi areas rel L2 = {err:.3e}, sum/XY = {h.sum() / (X * Y):.7f}")
    assert err <= 1e-5
    assert plan.status() == 0
    gh = rng.normal(size=xy.shape[0])
    gxy = torch.zeros((xy.shape[0], 2), dtype=torch.float32, device="cuda")
    plan.voronoi_grad(dev(gh), gxy)
    refg = voronoi.areas_2d_grad(reduce(xy, X, Y), X, Y, gh)
    errg = rel(host(gxy), refg)
    print(f"{layout}: Voronoi gradient rel L2 = {errg:.3e}")
    assert errg <= 1e-4


def test_voronoi_lengths_2d_plan():
    rng = np.random.default_rng(8)
    nx, nz = 40, 32
    X = nx * 1e-4
    x = rng.uniform(-X, X, 37)
    plan = pa().Plan2D(x, 32, 20e-9, 1500.0, (nx, nz, 1e-4, 1e-4))
    xr = x - X * np.floor(x / X + 0.5)
    assert rel(host(plan.voronoi_weights()), voronoi.lengths_1d(xr, X)) <= 1e-6
    gh = rng.normal(size=37)
    gxy = torch.zeros((37, 2), dtype=torch.float32, device="cuda")
    plan.voronoi_grad(dev(gh), gxy)
    got = host(gxy)
    assert rel(got[:, 0], voronoi.lengths_1d_grad(xr, X, gh)) <= 1e-6
    assert np.all(got[:, 1] == 0.0)


def test_gradient_through_voronoi_weights_end_to_end():
    """L(x) = <fbar, A(x, h(x)) g> with h(x) the Voronoi areas: the device
    chain (explicit position gradient + weight gradient through the Voronoi
    derivative) against FP64 central differences of the direct sums."""
    rng = np.random.default_rng(9)
    grid = synth.Grid(12, 10, 16, 1e-4, 1e-4, 1e-4)
    X, Y = grid.nx * grid.dx, grid.ny * grid.dy
    xy = synth.jittered_lattice(rng, 12, 10, grid.dx, grid.dy, 0.3)
    nt, dt, c = 32, 20e-9, 1500.0
    g = rng.normal(size=(xy.shape[0], nt))
    fb = rng.normal(size=grid.shape)
    h = voronoi.areas_2d(reduce(xy, X, Y), X, Y)
    plan = pa().Plan(xy, nt, dt, c, grid.as_tuple(), weights=h)
    gd, fd = dev(g), dev(fb)
    _, gxy = plan.position_grad(gd, fd)
    plan.voronoi_grad(plan.weight_grad(gd, fd), gxy)
    got = host(gxy)

    def L(p):
        return float(np.vdot(fb, ndft.reconstruct(p, voronoi.areas_2d(reduce(p, X, Y), X, Y), g, dt, c, grid)))

    eps = 1e-9
    idx = rng.choice(xy.shape[0], size=12, replace=False)
    ref = np.zeros((12, 2))
    for r, m in enumerate(idx):
        for k in range(2):
            a, b = xy.copy(), xy.copy()
            a[m, k] += eps
            b[m, k] -= eps
            ref[r, k] = (L(a) - L(b)) / (2 * eps)
    err = rel(got[idx], ref)
    print(f"gradient through Voronoi weights: rel L2 vs FD = {err:.3e}")
    assert err <= 1e-3


def test_set_weights_matches_a_fresh_plan():
    rng = np.random.default_rng(10)
    P = synth.c1()
    plan = pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    h = plan.voronoi_weights()
    plan.set_weights(h)
    fresh = pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=host(h))
    gd = dev(P.g)
    assert rel(host(plan.reconstruct(gd)), host(fresh.reconstruct(gd))) <= 1e-6
    fb = dev(rng.normal(size=P.grid.shape))
    assert rel(host(plan.adjoint(fb)), host(fresh.adjoint(fb))) <= 1e-6
    # on the lattice path too (lattice amplitudes rescaled)
    xy = synth.lattice_positions(P.grid.nx, P.grid.ny, P.grid.dx, P.grid.dy)
    pl = pa().Plan(xy, P.n_t, P.dt, P.c, P.grid.as_tuple())
    assert pl.is_lattice
    hw = rng.uniform(0.5, 1.5, xy.shape[0]) * P.grid.dx * P.grid.dy
    pl.set_weights(dev(hw))
    fr = pa().Plan(xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=hw)
    g = dev(rng.normal(size=(xy.shape[0], P.n_t)))
    assert rel(host(pl.reconstruct(g)), host(fr.reconstruct(g))) <= 1e-6


def test_autograd_with_voronoi_weights():
    """reconstruct(..., voronoi=True): the loss gradient to the positions
    includes the weights' dependence on them (FP64 central differences of the
    direct sums with Voronoi weights)."""
    rng = np.random.default_rng(11)
    grid = synth.Grid(10, 12, 16, 1e-4, 1e-4, 1e-4)
    X, Y = grid.nx * grid.dx, grid.ny * grid.dy
    xy0 = synth.jittered_lattice(rng, 10, 12, grid.dx, grid.dy, 0.3)
    nt, dt, c = 32, 20e-9, 1500.0
    g = rng.normal(size=(xy0.shape[0], nt))
    fb = rng.normal(size=grid.shape)
    plan = pa().Plan(xy0, nt, dt, c, grid.as_tuple())
    xy = torch.tensor(xy0, dtype=torch.float64, requires_grad=True)
    f = pa().reconstruct(dev(g), xy, plan, voronoi=True)
    (f * dev(fb)).sum().backward()
    got = xy.grad.numpy()

    def L(p):
        return float(np.vdot(fb, ndft.reconstruct(p, voronoi.areas_2d(reduce(p, X, Y), X, Y), g, dt, c, grid)))

    eps = 1e-9
    idx = rng.choice(xy0.shape[0], size=10, replace=False)
    ref = np.zeros((10, 2))
    for r, m in enumerate(idx):
        for k in range(2):
            a, b = xy0.copy(), xy0.copy()
            a[m, k] += eps
            b[m, k] -= eps
            ref[r, k] = (L(a) - L(b)) / (2 * eps)
    err = rel(got[idx], ref)
    print(f"autograd with Voronoi weights: rel L2 vs FD = {err:.3e}")
    assert err <= 1e-3
