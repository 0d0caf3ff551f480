"""pa_position_grad_noalloc: the position gradient whose scratch lives in a
static device array of the library, for callers that may not allocate device
memory when they need gradients (inside a CUDA-graph capture, or under a
fixed memory arena).  It must give the same result as pa_position_grad, on
consecutive calls, and refuse problems larger than its static array.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import ctypes
from ctypes import c_void_p

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_02946_gb300 import build, _lib
    build.build()
    return _lib.load()


def _ptr(t):
    return c_void_p(t.data_ptr())


def test_noalloc_gradient_matches_position_grad_on_consecutive_calls(lib):
    import paper_1501_02946_gb300 as pa
    P = synth.c1()
    plan = pa.Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    g = torch.tensor(P.g, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(31)
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        fb = torch.tensor(rng.normal(size=P.grid.shape), dtype=torch.float32, device="cuda")
        ref_g, ref_xy = plan.position_grad(g, fb)              # existing entry point
        out_g = torch.full_like(g, float("nan"))
        out_xy = torch.full((P.n_sensors, 2), float("nan"), device="cuda")
        rc = lib.pa_position_grad_noalloc(plan.handle, _ptr(g), _ptr(fb), _ptr(out_g), _ptr(out_xy), stream)
        assert rc == 0, lib.pa_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out_xy).all() and torch.isfinite(out_g).all()
        assert _rel(out_xy, ref_xy) <= TOL, f"call {call}"
        assert _rel(out_g, ref_g) <= TOL, f"call {call}"
    plan.close()


def test_noalloc_gradient_rejects_problems_beyond_its_array(lib):
    import paper_1501_02946_gb300 as pa
    rng = np.random.default_rng(4)
    grid = (64, 64, 16, 1e-4, 1e-4, 1e-4)
    M, nt = 70000, 1024                          # ceil(1024/32) * M > 2^21 partials
    xy = rng.uniform(-3.2e-3, 3.2e-3, size=(M, 2))
    plan = pa.Plan(xy, nt, 20e-9, 1500.0, grid)
    g = torch.zeros((M, nt), device="cuda")
    fb = torch.zeros(grid[:3], device="cuda")
    gxy = torch.zeros((M, 2), device="cuda")
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pa_position_grad_noalloc(plan.handle, _ptr(g), _ptr(fb), None, _ptr(gxy), stream)
    assert rc == 2
    assert b"static limit" in lib.pa_last_error()
    plan.close()
