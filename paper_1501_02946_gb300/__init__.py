"""GB300 (sm_103a) NEDNER-NUFFT for planar-sensor photoacoustic reconstruction.

Thin Python binding of the C ABI declared in include/pa_nufft.h: every step of
the reconstruction runs in the CUDA kernels of libpa_nufft.so; this module only
marshals arguments (torch tensors -> device pointers, the current torch
stream).  PyTorch provides device memory and streams.

    plan = Plan(xy, n_t=512, dt=20e-9, c=1500.0, grid=(128, 128, 256, 1e-4, 1e-4, 1e-4))
    f = plan.reconstruct(g)            # g: cuda float32 [M, n_t] -> f: [nx, ny, nz]
    g2 = plan.adjoint(f)               # exact transpose
    f = reconstruct(g, xy_param, plan) # autograd: gradients to g and positions
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_int, c_int64, c_void_p

import numpy as np

from . import _lib
from ._lib import PaError, PaGrid, PaGrid2, check

__all__ = ["Plan", "Plan2D", "Batch", "reconstruct", "ReconstructFunction", "PaError", "library_path",
           "correlation", "tenenbaum"]

library_path = _lib.LIB_PATH


def _torch():
    import torch
    return torch


def _stream_ptr(device=None):
    torch = _torch()
    return c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_tensor(t, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """A reconstruction plan (pa_plan_create).

    xy: (M, 2) sensor positions in metres; weights: (M,) detector areas in m^2
    or None (X*Y/M each); grid: (nx, ny, nz, dx, dy, dz)."""

    def __init__(self, xy, n_t, dt, c, grid, weights=None, sigma=2, width=8, device=None, lattice=True,
                 warp_ner=True):
        torch = _torch()
        lib = _lib.load()
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
        self.M = xy.shape[0]
        self.n_t = int(n_t)
        self.dt = float(dt)
        self.c = float(c)
        nx, ny, nz, dx, dy, dz = grid
        self.grid = (int(nx), int(ny), int(nz), float(dx), float(dy), float(dz))
        self.sigma = int(sigma)
        self.width = int(width)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        w = None
        if weights is not None:
            w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
            if w.shape[0] != self.M:
                raise ValueError("weights must have one entry per sensor")
        g = PaGrid(*self.grid)
        ptr = c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.pa_plan_create(byref(ptr), self.M, xy.ctypes.data_as(c_void_p),
                                    None if w is None else w.ctypes.data_as(c_void_p),
                                    self.n_t, self.dt, self.c, byref(g), self.sigma, self.width,
                                    (0 if lattice else 1)  # PA_FLAG_NO_LATTICE
                                    | (0 if warp_ner else 2),  # PA_FLAG_BLOCK_NER
                                    _stream_ptr(self.device))
        check(rc)
        self._ptr = ptr
        self._xy, self._xy_dev, self._dev_key = xy.copy(), None, None

    # -- properties
    @property
    def image_shape(self):
        return self.grid[:3]

    @property
    def data_shape(self):
        return (self.M, self.n_t)

    @property
    def handle(self):
        if self._ptr is None or not self._ptr.value:
            raise RuntimeError("plan was destroyed")
        return self._ptr

    @property
    def is_lattice(self):
        """True when the sensors sit on the output lattice and the plan takes
        the lattice spatial step (pa_plan_is_lattice)."""
        v = c_int()
        check(_lib.load().pa_plan_is_lattice(self.handle, byref(v)))
        return bool(v.value)

    @property
    def warp_ner(self):
        """True when the NER stage runs the warp-per-column kernels
        (pa_plan_uses_warp_ner)."""
        v = c_int()
        check(_lib.load().pa_plan_uses_warp_ner(self.handle, byref(v)))
        return bool(v.value)

    def info(self):
        M, nt, ws = c_int64(), c_int64(), c_int64()
        check(_lib.load().pa_plan_info(self.handle, byref(M), byref(nt), byref(ws)))
        return {"n_sensors": M.value, "n_t": nt.value, "workspace_bytes": ws.value}

    # -- operators
    def reconstruct(self, g, out=None):
        torch = _torch()
        _check_tensor(g, self.data_shape, "g")
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.float32, device=g.device)
        _check_tensor(out, self.image_shape, "out")
        check(_lib.load().pa_reconstruct(self.handle, c_void_p(g.data_ptr()), c_void_p(out.data_ptr()),
                                         _stream_ptr(g.device)))
        return out

    def reconstruct_cubic(self, g, out=None):
        torch = _torch()
        _check_tensor(g, self.data_shape, "g")
        if out is None:
            out = torch.empty(self.image_shape, dtype=torch.float32, device=g.device)
        _check_tensor(out, self.image_shape, "out")
        check(_lib.load().pa_reconstruct_cubic(self.handle, c_void_p(g.data_ptr()), c_void_p(out.data_ptr()),
                                               _stream_ptr(g.device)))
        return out

    def adjoint(self, f, out=None):
        torch = _torch()
        _check_tensor(f, self.image_shape, "f")
        if out is None:
            out = torch.empty(self.data_shape, dtype=torch.float32, device=f.device)
        _check_tensor(out, self.data_shape, "out")
        check(_lib.load().pa_reconstruct_adjoint(self.handle, c_void_p(f.data_ptr()), c_void_p(out.data_ptr()),
                                                 _stream_ptr(f.device)))
        return out

    def position_grad(self, g, grad_f, want_grad_g=True):
        """(A^T grad_f or None, dL/dxy [M, 2]) for L = <grad_f, A(xy) g>."""
        torch = _torch()
        _check_tensor(g, self.data_shape, "g")
        _check_tensor(grad_f, self.image_shape, "grad_f")
        grad_xy = torch.empty((self.M, 2), dtype=torch.float32, device=g.device)
        grad_g = torch.empty(self.data_shape, dtype=torch.float32, device=g.device) if want_grad_g else None
        check(_lib.load().pa_position_grad(self.handle, c_void_p(g.data_ptr()), c_void_p(grad_f.data_ptr()),
                                           c_void_p(grad_g.data_ptr()) if grad_g is not None else None,
                                           c_void_p(grad_xy.data_ptr()), _stream_ptr(g.device)))
        return grad_g, grad_xy

    def weight_grad(self, g, grad_f):
        """dL/dh [M] for L = <grad_f, A(h) g> (pa_weight_grad)."""
        torch = _torch()
        _check_tensor(g, self.data_shape, "g")
        _check_tensor(grad_f, self.image_shape, "grad_f")
        out = torch.empty(self.M, dtype=torch.float32, device=g.device)
        check(_lib.load().pa_weight_grad(self.handle, c_void_p(g.data_ptr()), c_void_p(grad_f.data_ptr()),
                                         c_void_p(out.data_ptr()), _stream_ptr(g.device)))
        return out

    def voronoi_weights(self):
        """Voronoi cell sizes [M] of the plan's sensors in the periodic domain
        (pa_voronoi_weights)."""
        torch = _torch()
        out = torch.empty(self.M, dtype=torch.float32, device=self.device)
        check(_lib.load().pa_voronoi_weights(self.handle, c_void_p(out.data_ptr()), _stream_ptr(self.device)))
        return out

    def set_weights(self, h):
        """New detector weights [M] (CUDA tensor or host array) for this plan
        (pa_plan_set_weights_device)."""
        torch = _torch()
        t = torch.as_tensor(h, dtype=torch.float32, device=self.device).contiguous().reshape(-1)
        if t.numel() != self.M:
            raise ValueError("set_weights needs one weight per sensor")
        check(_lib.load().pa_plan_set_weights_device(self.handle, c_void_p(t.data_ptr()), _stream_ptr(self.device)))

    def voronoi_grad(self, grad_h, grad_xy):
        """grad_xy [M, 2] += sum_k grad_h[k] dh_k/dx (pa_voronoi_grad); returns grad_xy."""
        _check_tensor(grad_xy, (self.M, 2), "grad_xy")
        gh = grad_h.contiguous()
        check(_lib.load().pa_voronoi_grad(self.handle, c_void_p(gh.data_ptr()), c_void_p(grad_xy.data_ptr()),
                                          _stream_ptr(self.device)))
        return grad_xy

    def position_grad_noalloc(self, g, grad_f, want_grad_g=True):
        """position_grad whose scratch is the library's static device array
        (no device allocation in the call; see include/pa_nufft.h)."""
        torch = _torch()
        _check_tensor(g, self.data_shape, "g")
        _check_tensor(grad_f, self.image_shape, "grad_f")
        grad_xy = torch.empty((self.M, 2), dtype=torch.float32, device=g.device)
        grad_g = torch.empty(self.data_shape, dtype=torch.float32, device=g.device) if want_grad_g else None
        check(_lib.load().pa_position_grad_noalloc(
            self.handle, c_void_p(g.data_ptr()), c_void_p(grad_f.data_ptr()),
            c_void_p(grad_g.data_ptr()) if grad_g is not None else None, c_void_p(grad_xy.data_ptr()),
            _stream_ptr(g.device)))
        return grad_g, grad_xy

    def update_positions(self, xy):
        """New sensor positions (M, 2) in metres: a host array (re-binned on
        the host in FP64) or a CUDA tensor (float32, re-binned on the device)."""
        torch = _torch()
        if isinstance(xy, torch.Tensor) and xy.is_cuda:
            t = xy.detach().to(torch.float32).reshape(-1, 2).clone()
            if t.shape[0] != self.M:
                raise ValueError("update_positions needs one position per sensor")
            check(_lib.load().pa_plan_update_positions_device(self.handle, c_void_p(t.data_ptr()),
                                                              _stream_ptr(self.device)))
            # the host copy is made only if `positions` is asked for
            self._xy, self._xy_dev = None, t
            self._dev_key = None
            return
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
        if xy.shape[0] != self.M:
            raise ValueError("update_positions needs one position per sensor")
        check(_lib.load().pa_plan_update_positions(self.handle, xy.ctypes.data_as(c_void_p),
                                                   _stream_ptr(self.device)))
        self._xy, self._xy_dev = xy.copy(), None
        self._dev_key = None

    @property
    def positions(self):
        """The plan's current sensor positions (M, 2) as a host float64 array."""
        if self._xy is None:
            self._xy = self._xy_dev.cpu().numpy().astype(np.float64)
        return self._xy.copy()

    def buffer(self, which):
        """Copy of an intermediate buffer (0: G1 spatial spectrum, 1: image
        spectrum after NER) as a complex64 torch tensor."""
        torch = _torch()
        lib = _lib.load()
        nbytes = c_int64()
        check(lib.pa_plan_buffer(self.handle, which, None, 0, byref(nbytes), _stream_ptr(self.device)))
        nx, ny, nz = self.image_shape
        if which == 0:
            shape = (2 * (nx // 2) + 1, ny // 2 + 1, self.n_t)
        else:
            shape = (nx, ny // 2 + 1, nz)
        out = torch.empty(shape, dtype=torch.complex64, device=self.device)
        check(lib.pa_plan_buffer(self.handle, which, c_void_p(out.data_ptr()), out.numel() * 8, byref(nbytes),
                                 _stream_ptr(self.device)))
        return out

    def profile(self, enable=True, stages=None):
        """Record CUDA events around every kernel launch of this plan, or
        (stages: names from profile_read) around those stages' launches only."""
        if stages is None:
            check(_lib.load().pa_profile_enable(self.handle, 1 if enable else 0))
            return
        lib = _lib.load()
        names, n = {}, 0
        while lib.pa_profile_stage_name(n):
            names[lib.pa_profile_stage_name(n).decode()] = n
            n += 1
        mask = 0
        for st in stages:
            if st not in names:
                raise ValueError(f"unknown stage {st!r}")
            mask |= 1 << names[st]
        check(lib.pa_profile_select(self.handle, mask if enable else 0))

    def profile_read(self):
        """{stage name: (total ms, launches)} since the last read (waits for
        the recorded events)."""
        lib = _lib.load()
        n = 0
        while lib.pa_profile_stage_name(n):  # names run out after the last stage
            n += 1
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        check(lib.pa_profile_read(self.handle, ms, cnt))
        return {lib.pa_profile_stage_name(k).decode(): (ms[k], cnt[k]) for k in range(n) if cnt[k]}

    def autotune(self):
        """Time the alternative launch shapes of the spread, NER and
        interpolation kernels and keep the fastest (pa_plan_autotune)."""
        arr = (c_int * 4)()
        check(_lib.load().pa_plan_autotune(self.handle, _stream_ptr(self.device), arr))
        return {"spread_samples_per_lane": arr[0], "ner_columns_per_block": arr[1],
                "ner_threads": arr[2], "interp_tile_columns": arr[3]}

    def status(self):
        v = c_int()
        rc = _lib.load().pa_status(self.handle, byref(v), _stream_ptr(self.device))
        if rc not in (0, 6):
            check(rc)
        return v.value

    def close(self):
        if getattr(self, "_ptr", None) is not None and self._ptr.value:
            _lib.load().pa_plan_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan2D(Plan):
    """A plan of the d = 2 operator (pa_plan_create_2d): sensors on the line
    z = 0, images f[nx][nz].

    x: (M,) sensor positions in metres; weights: (M,) detector lengths in m
    or None (X/M each); grid: (nx, nz, dx, dz).  reconstruct, adjoint,
    reconstruct_cubic and position_grad (d/dx_m in column 0, zeros in
    column 1) work as for Plan."""

    def __init__(self, x, n_t, dt, c, grid, weights=None, sigma=2, width=8, device=None, warp_ner=True):
        torch = _torch()
        lib = _lib.load()
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
        self.M = x.shape[0]
        self.n_t = int(n_t)
        self.dt = float(dt)
        self.c = float(c)
        nx, nz, dx, dz = grid
        self.grid = (int(nx), int(nz), float(dx), float(dz))
        self.sigma = int(sigma)
        self.width = int(width)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        w = None
        if weights is not None:
            w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
            if w.shape[0] != self.M:
                raise ValueError("weights must have one entry per sensor")
        g = PaGrid2(*self.grid)
        ptr = c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.pa_plan_create_2d(byref(ptr), self.M, x.ctypes.data_as(c_void_p),
                                       None if w is None else w.ctypes.data_as(c_void_p),
                                       self.n_t, self.dt, self.c, byref(g), self.sigma, self.width,
                                       0 if warp_ner else 2,  # PA_FLAG_BLOCK_NER
                                       _stream_ptr(self.device))
        check(rc)
        self._ptr = ptr
        self._xy = np.stack([x, np.zeros_like(x)], axis=1)
        self._xy_dev, self._dev_key = None, None

    @property
    def image_shape(self):
        return (self.grid[0], self.grid[1])

    def buffer(self, which):
        torch = _torch()
        lib = _lib.load()
        nbytes = c_int64()
        nx, nz = self.image_shape
        shape = (2 * (nx // 2) + 1, 1, self.n_t) if which == 0 else (nx, 1, nz)
        out = torch.empty(shape, dtype=torch.complex64, device=self.device)
        check(lib.pa_plan_buffer(self.handle, which, c_void_p(out.data_ptr()), out.numel() * 8, byref(nbytes),
                                 _stream_ptr(self.device)))
        return out


class Batch:
    """Many plans of uneven sizes reconstructed together (pa_batch_*),
    replayed as a CUDA graph.  mode 0: each instance's own single-plan
    launches as concurrent graph branches; mode 1: one launch per stage over
    all instances."""

    def __init__(self, plans, mode=0):
        torch = _torch()
        self.plans = list(plans)
        n = len(self.plans)
        arr = (c_void_p * n)(*[p.handle for p in self.plans])
        ptr = c_void_p()
        check(_lib.load().pa_batch_create(byref(ptr), n, arr, _stream_ptr(self.plans[0].device)))
        self._ptr = ptr
        self.device = self.plans[0].device
        check(_lib.load().pa_batch_set_mode(self._ptr, int(mode)))
        del torch

    def run(self, gs, fs):
        n = len(self.plans)
        if len(gs) != n or len(fs) != n:
            raise ValueError("one data and one image tensor per plan")
        for p, g, f in zip(self.plans, gs, fs):
            _check_tensor(g, p.data_shape, "g")
            _check_tensor(f, p.image_shape, "f")
        ga = (c_void_p * n)(*[g.data_ptr() for g in gs])
        fa = (c_void_p * n)(*[f.data_ptr() for f in fs])
        check(_lib.load().pa_batch_run(self._ptr, ga, fa, _stream_ptr(self.device)))
        return fs

    def close(self):
        if getattr(self, "_ptr", None) is not None and self._ptr.value:
            _lib.load().pa_batch_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    torch = _torch()

    class ReconstructFunction(torch.autograd.Function):
        """f = A(xy) g with gradients to the data g (the adjoint) and to the
        sensor positions xy (through the window derivative)."""

        @staticmethod
        def forward(ctx, g, xy, plan, voronoi=False):
            if xy.is_cuda:
                # positions on the device are re-binned on the device, without
                # a copy to the host, unless they are the very tensor (same
                # object, no in-place change since: same version counter) the
                # plan was last given
                key = getattr(plan, "_dev_key", None)
                if key is None or key[0] is not xy or key[1] != xy._version:
                    plan.update_positions(xy)
                    plan._dev_key = (xy, xy._version)
            else:
                xy_np = xy.detach().to("cpu", torch.float64).numpy()
                if not np.array_equal(xy_np, plan.positions):
                    plan.update_positions(xy_np)
            if voronoi:
                plan.set_weights(plan.voronoi_weights())
            ctx.plan = plan
            ctx.voronoi = voronoi
            ctx.xy_meta = (xy.dtype, xy.device)
            ctx.save_for_backward(g)
            return plan.reconstruct(g.contiguous())

        @staticmethod
        def backward(ctx, grad_f):
            (g,) = ctx.saved_tensors
            plan = ctx.plan
            grad_f = grad_f.contiguous()
            need_g, need_xy = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            grad_g = grad_xy = None
            if need_xy:
                grad_g, gxy = plan.position_grad(g.contiguous(), grad_f, want_grad_g=need_g)
                if ctx.voronoi:  # the weights follow the positions
                    plan.voronoi_grad(plan.weight_grad(g.contiguous(), grad_f), gxy)
                dtype, device = ctx.xy_meta
                grad_xy = gxy.to(device=device, dtype=dtype)
            elif need_g:
                grad_g = plan.adjoint(grad_f)
            return grad_g, grad_xy, None, None

    return ReconstructFunction


_RF = None


def ReconstructFunction():
    global _RF
    if _RF is None:
        _RF = _autograd()
    return _RF


def reconstruct(g, xy, plan, voronoi=False):
    """Differentiable reconstruction: f = A(xy) g.  With voronoi=True the
    detector weights are the Voronoi cells of xy (set on every call) and the
    position gradient includes their dependence on xy.

    xy on the host is compared with the plan's positions and re-binned on the
    host when it differs; xy on the GPU (float32 is enough: the cell
    coordinates are formed in FP64 on the device) is re-binned on the device
    unless it is the same tensor as on the last call with no in-place change
    since (its version counter; a change through .data bypasses the counter
    and is not seen)."""
    return ReconstructFunction().apply(g, xy, plan, voronoi)


# ------------------------------------------------------------ quality measures
def correlation(a, b):
    """Correlation coefficient of two CUDA float32 tensors with the same number
    of elements (pa_correlation)."""
    if a.numel() != b.numel():
        raise ValueError("correlation needs tensors of equal size")
    a = a.contiguous()
    b = b.contiguous()
    v = ctypes.c_double()
    check(_lib.load().pa_correlation(c_void_p(a.data_ptr()), c_void_p(b.data_ptr()), a.numel(), byref(v),
                                     _stream_ptr(a.device)))
    return v.value


def tenenbaum(u):
    """Normalised Tenenbaum sharpness of a CUDA float32 image [n0][n1] or stack
    [n0][n1][n2] of images over the first two axes (pa_tenenbaum)."""
    u = u.contiguous()
    if u.dim() == 2:
        n0, n1, n2 = u.shape[0], u.shape[1], 1
    elif u.dim() == 3:
        n0, n1, n2 = u.shape
    else:
        raise ValueError("tenenbaum takes a 2-D image or a 3-D stack")
    v = ctypes.c_double()
    check(_lib.load().pa_tenenbaum(c_void_p(u.data_ptr()), n0, n1, n2, byref(v), _stream_ptr(u.device)))
    return v.value
