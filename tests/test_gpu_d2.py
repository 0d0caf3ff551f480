"""The d = 2 operator (pa_plan_create_2d): forward, adjoint and position
gradient against the direct FP64 sums (oracle reconstruct_2d and its
transpose), dot-product tests, even and odd nx, the warp and the block NER
kernels, and the arguments the 2-D plans refuse."""
import numpy as np
import pytest
import torch

from oracle import ndft

from test_gpu_parity import TOL, close, dev, host, pa, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def line_case(nx, nz, nt, ns, seed, dx=1e-4, dz=1e-4):
    rng = np.random.default_rng(seed)
    X = nx * dx
    # ns sensors, jittered around an equispaced line over the aperture
    x = (np.arange(ns) + 0.5) * (X / ns) - X / 2 + rng.uniform(-0.4, 0.4, ns) * (X / ns)
    h = rng.uniform(0.6, 1.4, ns) * (X / ns)
    g = rng.normal(size=(ns, nt))
    return x, h, g, ndft.Grid2(nx, nz, dx, dz)


CASES = [(16, 32, 64, 16), (15, 24, 50, 21), (32, 256, 256, 40), (24, 36, 40, 17), (64, 512, 256, 50),
         (300, 64, 128, 90)]


@pytest.mark.parametrize("nx,nz,nt,ns", CASES)
def test_2d_forward_adjoint_match_direct_sums(nx, nz, nt, ns):
    x, h, g, grid = line_case(nx, nz, nt, ns, seed=nx + nz)
    dt, c = 20e-9, 1500.0
    plan = pa().Plan2D(x, nt, dt, c, (nx, nz, grid.dx, grid.dz), weights=h)
    f = host(plan.reconstruct(dev(g)))
    assert f.shape == (nx, nz)
    close(f, ndft.reconstruct_2d(x, h, g, dt, c, grid), f"2-D {nx}x{nz} nt={nt} M={ns} warp={plan.warp_ner} forward")
    fb = np.random.default_rng(3).normal(size=(nx, nz))
    gb = host(plan.adjoint(dev(fb)))
    close(gb, ndft.reconstruct_adjoint_2d(x, h, fb, dt, c, grid, nt), f"2-D {nx}x{nz} nt={nt} adjoint")
    lhs = float(np.vdot(f, fb))
    rhs = float(np.vdot(g.astype(np.float32).astype(np.float64), gb))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    assert plan.status() == 0


@pytest.mark.parametrize("nx,nz,nt,ns", CASES[:3])
def test_2d_position_grad_matches_oracle(nx, nz, nt, ns):
    x, h, g, grid = line_case(nx, nz, nt, ns, seed=7)
    dt, c = 20e-9, 1500.0
    plan = pa().Plan2D(x, nt, dt, c, (nx, nz, grid.dx, grid.dz), weights=h)
    fb = np.random.default_rng(4).normal(size=(nx, nz))
    gg, gxy = plan.position_grad(dev(g), dev(fb))
    gxy = host(gxy)
    ref = ndft.position_grad_2d(x, h, g, fb, dt, c, grid)
    close(gxy[:, 0], ref, f"2-D {nx}x{nz} position gradient")
    assert np.all(gxy[:, 1] == 0.0)
    close(host(gg), ndft.reconstruct_adjoint_2d(x, h, fb, dt, c, grid, nt), f"2-D {nx}x{nz} data gradient")


def test_2d_warp_and_block_ner_agree():
    x, h, g, grid = line_case(32, 256, 256, 40, seed=9)
    a = pa().Plan2D(x, 256, 20e-9, 1500.0, (32, 256, grid.dx, grid.dz), weights=h)
    b = pa().Plan2D(x, 256, 20e-9, 1500.0, (32, 256, grid.dx, grid.dz), weights=h, warp_ner=False)
    assert a.warp_ner and not b.warp_ner
    gd = dev(g)
    assert rel(host(a.reconstruct(gd)), host(b.reconstruct(gd))) <= 1e-5


def test_2d_default_weights_are_x_over_m():
    x, h, g, grid = line_case(16, 32, 64, 12, seed=11)
    dt, c = 20e-9, 1500.0
    plan = pa().Plan2D(x, 64, dt, c, (16, 32, grid.dx, grid.dz))
    hdef = np.full(12, 16 * grid.dx / 12)
    close(host(plan.reconstruct(dev(g))), ndft.reconstruct_2d(x, hdef, g, dt, c, grid), "2-D default weights forward")


def test_2d_plans_refuse_unsupported_calls():
    x, h, g, grid = line_case(16, 32, 64, 12, seed=12)
    plan = pa().Plan2D(x, 64, 20e-9, 1500.0, (16, 32, grid.dx, grid.dz), weights=h)
    with pytest.raises(pa().PaError):
        plan.autotune()
    with pytest.raises(pa().PaError):
        plan.update_positions(np.zeros((12, 2)))


def test_2d_bench_size_dot_and_columns():
    """The 512 x 512, 1024-sample, 256-sensor workload of the bench: dot test
    of forward and adjoint, and three image columns against the direct sums
    (oracle column_depth_profile on the one-row grid)."""
    rng = np.random.default_rng(1507)
    nx, nz, nt, M = 512, 512, 1024, 256
    X = nx * 1e-4
    x = np.sort(np.concatenate([rng.uniform(-X / 2, X / 2, M // 2),
                                rng.normal(0.0, X / 8, M // 2).clip(-X / 2, X / 2 - 1e-7)]))
    dt, c = 20e-9, 1500.0
    plan = pa().Plan2D(x, nt, dt, c, (nx, nz, 1e-4, 1e-4))
    g = rng.normal(size=(M, nt))
    gd = dev(g)
    f = host(plan.reconstruct(gd))
    spec = plan.buffer(1).cpu().numpy()  # before the adjoint reuses the buffer
    fb = rng.normal(size=(nx, nz))
    gb = host(plan.adjoint(dev(fb)))
    lhs = float(np.vdot(f, fb))
    rhs = float(np.vdot(g.astype(np.float32).astype(np.float64), gb))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    # spectrum columns jx of the image spectrum after NER (buffer 1) against O1
    grid = ndft.Grid2(nx, nz, 1e-4, 1e-4)
    h = np.full(M, X / M)
    for jx in (0, 37, -101):
        ref = ndft.column_depth_profile(np.stack([x, np.zeros_like(x)], 1), h, g, dt, c, grid, jx, 0)
        got = spec[jx + nx // 2, 0, :]
        close(got, ref, f"2-D bench size column jx={jx}")
