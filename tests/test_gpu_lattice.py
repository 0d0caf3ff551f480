"""The lattice spatial step (sensors exactly on the output lattice): a plain
DFT over the lattice instead of window spreading, against the direct FP64
sums and against the general path on the same sensors."""
import numpy as np
import pytest
import torch

import synth
from oracle import ndft

from test_gpu_parity import TOL, close, dev, host, pa, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def lattice_case(nx, ny, nz, nt, seed=0, shuffle=True):
    rng = np.random.default_rng(seed)
    grid = synth.Grid(nx, ny, nz, 1e-4, 1.1e-4, 0.9e-4)
    xy = synth.lattice_positions(nx, ny, grid.dx, grid.dy)
    if shuffle:  # any sensor order; some positions shifted by whole periods
        xy = xy[rng.permutation(xy.shape[0])]
        xy[::7, 0] += 2 * nx * grid.dx
    h = np.full(xy.shape[0], grid.dx * grid.dy)
    g = rng.normal(size=(xy.shape[0], nt))
    return xy, h, g, grid


def make(xy, h, nt, grid, lattice=True):
    return pa().Plan(xy, nt, 20e-9, 1500.0, grid.as_tuple(), weights=h, lattice=lattice)


SIZES = [(8, 8, 16, 32), (9, 10, 12, 30), (32, 32, 64, 64), (12, 10, 16, 24), (16, 12, 20, 36)]


def test_lattice_detected():
    xy, h, g, grid = lattice_case(8, 8, 16, 32)
    assert make(xy, h, 32, grid).is_lattice
    assert not make(xy, h, 32, grid, lattice=False).is_lattice
    xy2 = xy.copy()
    xy2[3, 0] += 1e-7
    assert not make(xy2, h, 32, grid).is_lattice


@pytest.mark.parametrize("nx,ny,nz,nt", SIZES)
def test_lattice_forward_and_adjoint_match_direct_sums(nx, ny, nz, nt):
    xy, h, g, grid = lattice_case(nx, ny, nz, nt, seed=nx + ny)
    plan = make(xy, h, nt, grid)
    assert plan.is_lattice
    dt, c = 20e-9, 1500.0
    f = host(plan.reconstruct(dev(g)))
    ref = ndft.reconstruct(xy, h, g, dt, c, grid)
    close(f, ref, f"lattice {nx}x{ny}x{nz} nt={nt} forward")
    fb = np.random.default_rng(5).normal(size=grid.shape)
    gb = host(plan.adjoint(dev(fb)))
    refb = ndft.reconstruct_adjoint(xy, h, fb, dt, c, grid, nt)
    close(gb, refb, f"lattice {nx}x{ny}x{nz} nt={nt} adjoint")
    # the two are transposes of each other in FP32
    lhs = float(np.vdot(f, fb))
    rhs = float(np.vdot(g.astype(np.float32).astype(np.float64), gb))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("nx,ny,nz,nt", SIZES[:3])
def test_lattice_path_agrees_with_general_path(nx, ny, nz, nt):
    xy, h, g, grid = lattice_case(nx, ny, nz, nt, seed=1)
    a = make(xy, h, nt, grid)
    b = make(xy, h, nt, grid, lattice=False)
    gd = dev(g)
    assert rel(host(a.reconstruct(gd)), host(b.reconstruct(gd))) <= 1e-5
    fb = dev(np.random.default_rng(6).normal(size=grid.shape))
    assert rel(host(a.adjoint(fb)), host(b.adjoint(fb))) <= 1e-5
    # the position gradient keeps the windowed path on both (equal to the
    # rounding of the adjoint's shared-memory accumulation)
    assert rel(host(a.position_grad(gd, fb)[1]), host(b.position_grad(gd, fb)[1])) <= 1e-6


def test_device_position_update_leaves_the_lattice_path():
    xy, h, g, grid = lattice_case(8, 8, 16, 32)
    plan = make(xy, h, 32, grid)
    assert plan.is_lattice
    plan.update_positions(torch.tensor(xy.astype(np.float32), device="cuda"))
    assert not plan.is_lattice
    plan.update_positions(xy)
    assert plan.is_lattice
