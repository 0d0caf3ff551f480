"""The warp-per-column NER kernels (sigma 2, width 8, n_t and nz powers of
two in [256, 1024]) against the direct FP64 sums, and against the block NER
kernels on the same plan: forward, adjoint, the dot-product test and the
position gradient.  Sizes cover even and odd nx, ny (the two-source Nyquist
columns) and every pair of transform lengths the warp kernels are built for
that the direct sums finish in seconds."""
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


def case(nx, ny, nz, nt, seed):
    rng = np.random.default_rng(seed)
    grid = synth.Grid(nx, ny, nz, 1e-4, 1.1e-4, 0.9e-4)
    xy = synth.jittered_lattice(rng, nx, ny, grid.dx, grid.dy)
    h = np.full(xy.shape[0], nx * ny * grid.dx * grid.dy / xy.shape[0])
    g = rng.normal(size=(xy.shape[0], nt))
    return xy, h, g, grid


def make(xy, h, nt, grid, warp=True):
    return pa().Plan(xy, nt, 20e-9, 1500.0, grid.as_tuple(), weights=h, warp_ner=warp)


SIZES = [(8, 10, 256, 256), (9, 9, 512, 256), (8, 9, 256, 512), (9, 8, 1024, 256), (10, 8, 256, 1024),
         (8, 8, 512, 1024), (8, 9, 1024, 1024), (16, 12, 512, 512)]


@pytest.mark.parametrize("nx,ny,nz,nt", SIZES)
def test_warp_ner_matches_direct_sums(nx, ny, nz, nt):
    xy, h, g, grid = case(nx, ny, nz, nt, seed=nx * 31 + ny + nz + nt)
    plan = make(xy, h, nt, grid)
    assert plan.warp_ner
    dt, c = 20e-9, 1500.0
    f = host(plan.reconstruct(dev(g)))
    close(f, ndft.reconstruct(xy, h, g, dt, c, grid), f"warp NER {nx}x{ny}x{nz} nt={nt} forward")
    fb = np.random.default_rng(7).normal(size=grid.shape)
    gb = host(plan.adjoint(dev(fb)))
    ref_b, aux = ndft.reconstruct_adjoint(xy, h, fb, dt, c, grid, nt, full=True)
    close(gb, ref_b, f"warp NER {nx}x{ny}x{nz} nt={nt} adjoint")
    # the position gradient through the warp NER adjoint, against the
    # analytic O1 gradient from the same transposed chain
    gg, gxy = plan.position_grad(dev(g), dev(fb))
    close(host(gxy), ndft.position_grad_from_cotangent(xy, h, g, aux["G1bar"], grid),
          f"warp NER {nx}x{ny}x{nz} nt={nt} position gradient")
    close(host(gg), ref_b, f"warp NER {nx}x{ny}x{nz} nt={nt} data gradient")
    lhs = float(np.vdot(f, fb))
    rhs = float(np.vdot(g.astype(np.float32).astype(np.float64), gb))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    assert plan.status() == 0


@pytest.mark.parametrize("nx,ny,nz,nt", SIZES[:4])
def test_warp_and_block_ner_agree(nx, ny, nz, nt):
    xy, h, g, grid = case(nx, ny, nz, nt, seed=3)
    a, b = make(xy, h, nt, grid), make(xy, h, nt, grid, warp=False)
    assert a.warp_ner and not b.warp_ner
    gd = dev(g)
    assert rel(host(a.reconstruct(gd)), host(b.reconstruct(gd))) <= 1e-5
    fb = dev(np.random.default_rng(1).normal(size=grid.shape))
    assert rel(host(a.adjoint(fb)), host(b.adjoint(fb))) <= 1e-5
    _, ga = a.position_grad(gd, fb)
    _, gb = b.position_grad(gd, fb)
    assert rel(host(ga), host(gb)) <= 1e-4


def test_warp_ner_at_the_128x128x256_workload():
    P = synth.c2(noise=False)
    a, b = (pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h, warp_ner=w) for w in (True, False))
    assert a.warp_ner and not b.warp_ner
    gd = dev(P.g)
    err = rel(host(a.reconstruct(gd)), host(b.reconstruct(gd)))
    print(f"128x128x256: warp vs block NER forward rel L2 = {err:.3e}")
    assert err <= 1e-5
    fb = dev(np.random.default_rng(2).normal(size=P.grid.shape))
    errb = rel(host(a.adjoint(fb)), host(b.adjoint(fb)))
    print(f"128x128x256: warp vs block NER adjoint rel L2 = {errb:.3e}")
    assert errb <= 1e-5
    assert a.status() == 0


def test_block_ner_flag_for_ineligible_sizes():
    xy, h, g, grid = case(8, 8, 64, 128, seed=0)   # lengths below the warp kernels' range
    assert not make(xy, h, 128, grid).warp_ner
