"""The variational workload on the oracle: L(g, xy) = ||A(xy) g - target||^2
+ lam TV_eps(A(xy) g) on the 32x32x64 instance (one jittered 32x32 lattice,
one ball), FP64 throughout.

The chain rule that the library's autograd function applies -- the data
gradient A^T dL/df and the position gradient of <dL/df, A(xy) g> through the
window derivative -- is checked here against central finite differences of
the loss itself, in FP64 on the CPU."""
import numpy as np
import pytest

import synth
from oracle import ndft

import varloss


def test_tv_loss_gradient_matches_fd():
    rng = np.random.default_rng(31)
    f = rng.normal(size=(5, 4, 6))
    f[2] = f[1]  # flat regions: the eps keeps the square root smooth there
    t = rng.normal(size=f.shape)
    G = varloss.grad_f_np(f, t, lam=0.3, eps=1e-4)
    d = rng.normal(size=f.shape)
    h = 1e-6
    fd = (varloss.loss_np(f + h * d, t, 0.3, 1e-4) - varloss.loss_np(f - h * d, t, 0.3, 1e-4)) / (2 * h)
    assert abs(fd - np.sum(G * d)) <= 1e-7 * abs(fd)
    # data term alone: 2 (f - t)
    assert np.allclose(varloss.grad_f_np(f, t, lam=0.0), 2 * (f - t), rtol=0, atol=1e-14)


@pytest.fixture(scope="module")
def c1():
    P = synth.c1()
    target = P.voxelised()
    return P, target


def _loss(P, target, g, xy):
    return varloss.loss_np(ndft.reconstruct(xy, P.h, g, P.dt, P.c, P.grid), target)


def test_variational_gradients_match_fd(c1):
    P, target = c1
    f = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    dLdf = varloss.grad_f_np(f, target)
    grad_g = ndft.reconstruct_adjoint(P.xy, P.h, dLdf, P.dt, P.c, P.grid, P.n_t)
    grad_xy = ndft.position_grad(P.xy, P.h, P.g, dLdf, P.dt, P.c, P.grid)
    rng = np.random.default_rng(32)
    # data direction
    dg = rng.normal(size=P.g.shape)
    e = 1e-5 * np.linalg.norm(P.g) / np.linalg.norm(dg)
    fd = (_loss(P, target, P.g + e * dg, P.xy) - _loss(P, target, P.g - e * dg, P.xy)) / (2 * e)
    an = float(np.sum(grad_g * dg))
    print(f"data direction: FD {fd:.9e} analytic {an:.9e}")
    assert abs(fd - an) <= 1e-6 * abs(an)
    # position direction (metres)
    dxy = rng.normal(size=P.xy.shape)
    e = 1e-7 * P.grid.dx
    fd = (_loss(P, target, P.g, P.xy + e * dxy) - _loss(P, target, P.g, P.xy - e * dxy)) / (2 * e)
    an = float(np.sum(grad_xy * dxy))
    print(f"position direction: FD {fd:.9e} analytic {an:.9e}")
    assert abs(fd - an) <= 1e-5 * abs(an)


def test_variational_gradient_descends(c1):
    """A small step against the gradient lowers the loss by its first-order
    prediction (data and positions separately)."""
    P, target = c1
    L0 = _loss(P, target, P.g, P.xy)
    f = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    dLdf = varloss.grad_f_np(f, target)
    grad_g = ndft.reconstruct_adjoint(P.xy, P.h, dLdf, P.dt, P.c, P.grid, P.n_t)
    grad_xy = ndft.position_grad(P.xy, P.h, P.g, dLdf, P.dt, P.c, P.grid)
    for which, grad in (("g", grad_g), ("xy", grad_xy)):
        eta = 1e-3 * L0 / np.sum(grad * grad)
        if which == "g":
            L1 = _loss(P, target, P.g - eta * grad, P.xy)
        else:
            assert eta * np.abs(grad).max() < 0.05 * P.grid.dx
            L1 = _loss(P, target, P.g, P.xy - eta * grad)
        ratio = (L0 - L1) / (eta * np.sum(grad * grad))
        print(f"{which}: L0 {L0:.6e} L1 {L1:.6e} decrease / prediction {ratio:.4f}")
        assert 0.9 <= ratio <= 1.1
