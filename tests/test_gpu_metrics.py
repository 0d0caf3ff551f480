"""Device quality measures (pa_correlation, pa_tenenbaum) against the FP64
oracle: reconstructions, stacks, 2-D images and edge sizes."""
import numpy as np
import pytest
import torch

from oracle import metrics

from test_gpu_parity import dev, pa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("shape", [(128, 128, 256), (33, 17, 5), (2, 3), (1000001,)])
def test_correlation_matches_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.normal(size=shape).astype(np.float32)
    b = (0.6 * a + rng.normal(size=shape) + 5.0).astype(np.float32)
    got = pa().correlation(dev(a), dev(b))
    ref = metrics.correlation(a, b)
    assert abs(got - ref) <= 1e-12 + 1e-10 * abs(ref)


@pytest.mark.parametrize("shape", [(128, 128, 256), (3, 3), (37, 19), (9, 11, 1), (64, 31, 7)])
def test_tenenbaum_matches_oracle(shape):
    rng = np.random.default_rng(len(shape) + shape[0])
    u = rng.normal(size=shape).astype(np.float32)
    got = pa().tenenbaum(dev(u))
    ref = metrics.tenenbaum(u)
    assert abs(got - ref) <= 1e-10 * ref


def test_metrics_of_a_reconstruction():
    import synth
    P = synth.tiny()
    plan = pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    f = plan.reconstruct(dev(P.g))
    ref = P.voxelised()
    fh = f.cpu().numpy().astype(np.float64)
    assert abs(pa().correlation(f, dev(ref)) - metrics.correlation(fh, ref)) <= 1e-6
    assert abs(pa().tenenbaum(f) - metrics.tenenbaum(fh)) <= 1e-6 * metrics.tenenbaum(fh)


def test_metrics_reject_bad_arguments():
    with pytest.raises(pa().PaError):
        pa().tenenbaum(dev(np.zeros((2, 5))))


@pytest.mark.parametrize("d", [3, 2])
def test_weight_grad_matches_oracle(d):
    from oracle import ndft
    import synth
    rng = np.random.default_rng(40 + d)
    if d == 3:
        P = synth.tiny()
        plan = pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
        fb = rng.normal(size=P.grid.shape)
        ref = ndft.weight_grad(P.xy, P.h, P.g, fb, P.dt, P.c, P.grid)
        g = P.g
    else:
        nx, nz, nt, M = 24, 40, 64, 19
        grid = ndft.Grid2(nx, nz, 1e-4, 1e-4)
        x = rng.uniform(-nx * 5e-5, nx * 5e-5, M)
        h = rng.uniform(0.5, 1.5, M) * (nx * 1e-4 / M)
        g = rng.normal(size=(M, nt))
        plan = pa().Plan2D(x, nt, 20e-9, 1500.0, (nx, nz, 1e-4, 1e-4), weights=h)
        fb = rng.normal(size=(nx, nz))
        xy = np.stack([x, np.zeros_like(x)], 1)
        ref = ndft.weight_grad(xy, h, g, fb[:, None, :], 20e-9, 1500.0, grid)
    got = plan.weight_grad(dev(g), dev(fb)).cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"d={d}: weight gradient rel L2 = {err:.3e}")
    assert err <= 1e-4
