"""pa_position_grad_noalloc: the position gradient whose scratch lives in a
static device array of the library instead of the plan's workspace.  It is
for callers that cannot let the library allocate device memory while they
run (an application that hands out all device memory from its own arena or
caching allocator, or a loop that must not stall on cudaMalloc/cudaFree).

The tests call it through the C ABI and check that it gives what
pa_position_grad gives, call after call, with two plans of different sizes
taking turns (so partial sums left in the shared array by a larger problem
must not leak into a smaller one), with and without the data gradient, and
with the device status word clear after each call; and that it refuses a
problem larger than its array.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
from ctypes import c_int, c_void_p, byref

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


def _warp_ner_problem():
    """32x32 jittered sensors, 256 samples, output 32x32x256: sizes whose plan
    runs the warp-per-column NER kernels and the pipelined interpolation."""
    rng = np.random.default_rng(41)
    grid = synth.Grid(32, 32, 256, 1e-4, 1e-4, 1e-4)
    xy = synth.jittered_lattice(rng, 32, 32, 1e-4, 1e-4)
    return synth.Problem("noalloc_warp", xy, np.full(1024, 1e-8), rng.normal(size=(1024, 256)), 20e-9,
                         synth.C_WATER, grid)


def test_noalloc_gradient_matches_position_grad_on_consecutive_calls(lib):
    import paper_1501_02946_gb300 as pa
    probs = [synth.c1(), _warp_ner_problem()]
    plans = [pa.Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h) for P in probs]
    assert not plans[0].warp_ner and plans[1].warp_ner
    gs = [torch.tensor(P.g, dtype=torch.float32, device="cuda") for P in probs]
    rng = np.random.default_rng(31)
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
    # the two plans take turns; every other call leaves out the data gradient
    for call, (k, want_g) in enumerate([(0, True), (1, False), (0, False), (1, True), (0, True)]):
        P, plan, g = probs[k], plans[k], gs[k]
        fb = torch.tensor(rng.normal(size=P.grid.shape), dtype=torch.float32, device="cuda")
        ref_g, ref_xy = plan.position_grad(g, fb)              # the allocating entry point
        out_g = torch.full_like(g, float("nan")) if want_g else None
        out_xy = torch.full((P.n_sensors, 2), float("nan"), device="cuda")
        rc = lib.pa_position_grad_noalloc(plan.handle, _ptr(g), _ptr(fb), _ptr(out_g) if want_g else None,
                                          _ptr(out_xy), stream)
        assert rc == 0, lib.pa_last_error()
        status = c_int(-1)
        assert lib.pa_status(plan.handle, byref(status), stream) == 0
        assert status.value == 0, f"call {call}: device status {status.value}"
        torch.cuda.synchronize()
        assert torch.isfinite(out_xy).all()
        assert _rel(out_xy, ref_xy) <= TOL, f"call {call}"
        if want_g:
            assert torch.isfinite(out_g).all()
            assert _rel(out_g, ref_g) <= TOL, f"call {call}"
    for plan in plans:
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
