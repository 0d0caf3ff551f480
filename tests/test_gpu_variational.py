"""The variational workload on the device: L = ||A(xy) g - target||^2 +
lam TV_eps(A(xy) g), backpropagated through the library's autograd function
to the data g and the sensor positions xy.

32x32x64 instance: the gradients against the FP64 oracle's chain (A^T dL/df
and the window-derivative position gradient), with dL/df taken from the
device image in FP64 so that only the library's steps are compared.
128x128x256 (the non-equispaced 16384-sensor workload): the gradients
against the library's own adjoint and position-gradient calls, and a step
against each gradient lowering the loss by its first-order prediction."""
import numpy as np
import pytest
import torch

import synth
from oracle import ndft

import varloss
from test_gpu_parity import TOL, close, dev, host, pa, plan_of, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _forward_backward(P, plan, target_d, xy0=None):
    g = dev(P.g).requires_grad_(True)
    xy = torch.tensor(P.xy if xy0 is None else xy0, dtype=torch.float64, requires_grad=True)
    f = pa().reconstruct(g, xy, plan)
    L = varloss.loss(f, target_d)
    L.backward()
    return f, float(L), g.grad, xy.grad


def test_variational_gradients_match_oracle_c1():
    P = synth.c1()
    target = P.voxelised()
    plan = plan_of(P)
    f, L, gg, gxy = _forward_backward(P, plan, dev(target))
    f_ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    close(host(f), f_ref, "c1 variational forward")
    dLdf = varloss.grad_f_np(host(f), target)
    ref_g = ndft.reconstruct_adjoint(P.xy, P.h, dLdf, P.dt, P.c, P.grid, P.n_t)
    ref_xy = ndft.position_grad(P.xy, P.h, P.g, dLdf, P.dt, P.c, P.grid)
    print(f"c1 variational: loss {L:.6e}")
    close(host(gg), ref_g, "c1 variational grad g")
    close(gxy.numpy(), ref_xy, "c1 variational grad xy")
    assert abs(L - varloss.loss_np(f_ref, target)) <= 1e-4 * L


@pytest.fixture(scope="module")
def c2():
    P = synth.c2()
    return P, P.voxelised()


def test_variational_c2_gradients_and_descent(c2):
    P, target = c2
    plan = plan_of(P)
    target_d = dev(target)
    f, L0, gg, gxy = _forward_backward(P, plan, target_d)
    assert torch.isfinite(gg).all() and torch.isfinite(gxy).all()
    # the same gradients from the library's calls, with dL/df formed on the device
    ft = f.detach().clone().requires_grad_(True)
    varloss.loss(ft, target_d).backward()
    dLdf = ft.grad.contiguous()
    g_cal, xy_cal = plan.position_grad(dev(P.g), dLdf)
    assert rel(host(gg), host(g_cal)) <= 1e-6
    assert rel(gxy.numpy(), host(xy_cal)) <= 1e-6
    assert rel(host(gg), host(plan.adjoint(dLdf))) <= 1e-5
    # descent along -grad g (positions fixed) and along -grad xy (data fixed)
    G = host(gg).astype(np.float64)
    eta = 1e-3 * L0 / np.sum(G * G)
    with torch.no_grad():
        L1 = float(varloss.loss(plan.reconstruct(dev(P.g - eta * G)), target_d))
    r_g = (L0 - L1) / (eta * np.sum(G * G))
    X = gxy.numpy()
    eta = 1e-3 * L0 / np.sum(X * X)
    step = eta * X
    assert np.abs(step).max() < 0.05 * P.grid.dx
    plan.update_positions(P.xy - step)
    with torch.no_grad():
        L2 = float(varloss.loss(plan.reconstruct(dev(P.g)), target_d))
    r_xy = (L0 - L2) / (eta * np.sum(X * X))
    print(f"c2 variational: L0 {L0:.6e}; decrease / first-order prediction: data {r_g:.4f}, positions {r_xy:.4f}")
    assert 0.8 <= r_g <= 1.2
    assert 0.8 <= r_xy <= 1.2


def test_autograd_positions_on_the_device():
    """Positions given as a CUDA tensor are re-binned on the device (no copy
    to the host): the gradients equal those of the same positions given on
    the host to float rounding (the device path takes float32 positions), a
    second call with the same tensor keeps the binning, and an in-place step
    of the tensor is seen (its version counter)."""
    P = synth.c1()
    target_d = dev(P.voxelised())
    xy32 = P.xy.astype(np.float32).astype(np.float64)
    plan_h, plan_d = plan_of(P), plan_of(P)
    _, L_h, gg_h, gxy_h = _forward_backward(P, plan_h, target_d, xy0=xy32)
    xy_d = torch.tensor(xy32, dtype=torch.float32, device="cuda", requires_grad=True)
    for call in range(2):
        g = dev(P.g).requires_grad_(True)
        L = varloss.loss(pa().reconstruct(g, xy_d, plan_d), target_d)
        xy_d.grad = None
        L.backward()
        assert abs(float(L) - L_h) <= 1e-6 * abs(L_h)
        assert rel(host(g.grad), host(gg_h)) <= 1e-5
        assert rel(host(xy_d.grad), gxy_h.numpy()) <= 1e-4
        assert plan_d._xy is None            # no host copy of the positions was made
    with torch.no_grad():
        xy_d -= 3e-6 * xy_d.grad.sign()
    f2 = pa().reconstruct(dev(P.g), xy_d, plan_d)
    ref = plan_of(P)
    ref.update_positions(xy_d.detach().double().cpu().numpy())
    assert rel(host(f2), host(ref.reconstruct(dev(P.g)))) <= 1e-5
