"""The loss of the variational workload: data misfit plus total variation,
L(f) = ||f - target||^2 + lam * TV_eps(f), with the isotropic total variation
TV_eps(f) = sum_voxels sqrt(|D f|^2 + eps) of the forward differences D f
along the three image axes (zero across the last face of each axis).

This is the user's side of the workload (plain torch on whatever device f
lives on); the library supplies f = A(xy) g and its gradients."""
from __future__ import annotations

import numpy as np
import torch

LAM = 1e-3
EPS = 1e-8


def tv_eps(f, eps=EPS):
    d0 = torch.diff(f, dim=0, append=f[-1:])
    d1 = torch.diff(f, dim=1, append=f[:, -1:])
    d2 = torch.diff(f, dim=2, append=f[:, :, -1:])
    return torch.sqrt(d0 * d0 + d1 * d1 + d2 * d2 + eps).sum()


def loss(f, target, lam=LAM, eps=EPS):
    """FP64 accumulation whatever the dtype of f."""
    f = f.to(torch.float64)
    r = f - target.to(torch.float64)
    return (r * r).sum() + lam * tv_eps(f, eps)


def loss_np(f, target, lam=LAM, eps=EPS):
    return float(loss(torch.from_numpy(np.asarray(f, dtype=np.float64)), torch.from_numpy(target), lam, eps))


def grad_f_np(f, target, lam=LAM, eps=EPS):
    """dL/df in FP64 on the CPU."""
    ft = torch.tensor(np.asarray(f, dtype=np.float64), requires_grad=True)
    loss(ft, torch.from_numpy(np.asarray(target, dtype=np.float64)), lam, eps).backward()
    return ft.grad.numpy()
