"""A bounded wait that runs out, on the GPU, without a fault.

Through the C ABI test hook pa_plan_test_wait_fault, the pipelined
interpolation kernel posts the byte count of one work item on its mbarrier
but issues none of that item's copies (a barrier that nothing completes),
with a short poll limit.  The block that owns the item must give up, wait
(bounded) for the copies it did issue, record the wait-timeout bit in the
plan's status word and return: the call returns, pa_status reports the bit,
and the next call on the same plan, with the hook off, is exact again."""
from ctypes import c_void_p

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WAIT_TIMEOUT = 1   # PA_STATUS_WAIT_TIMEOUT


@pytest.fixture(scope="module")
def lib():
    from paper_1501_02946_gb300 import build, _lib
    build.build()
    return _lib.load()


def _rel(a, b):
    a, b = a.double().numpy(), b.double().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _problem(nside, nt, nz, seed):
    rng = np.random.default_rng(seed)
    grid = synth.Grid(nside, nside, nz, 1e-4, 1e-4, 1e-4)
    xy = synth.jittered_lattice(rng, nside, nside, 1e-4, 1e-4)
    X = nside * 1e-4
    return synth.Problem("timeout", xy, np.full(nside * nside, X * X / nside ** 2), rng.normal(size=(nside ** 2, nt)),
                         20e-9, synth.C_WATER, grid)


# 32x32x64, 128 samples: one interpolation item per block; 64x64x64, 512
# samples: 2048 items over the persistent blocks, so the dropped item (1000)
# has the copies of the block's next item in flight when its wait runs out
@pytest.mark.parametrize("nside,nt,nz,item", [(32, 128, 64, 0), (64, 512, 64, 1000)])
def test_wait_runs_out_reports_and_returns(lib, nside, nt, nz, item):
    import paper_1501_02946_gb300 as pa
    P = _problem(nside, nt, nz, 51)
    plan = pa.Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    fb = torch.tensor(np.random.default_rng(52).normal(size=P.grid.shape), dtype=torch.float32, device="cuda")
    g = torch.tensor(P.g, dtype=torch.float32, device="cuda")
    ref = plan.adjoint(fb).cpu()
    ref_xy = plan.position_grad(g, fb)[1].cpu()
    assert plan.status() == 0

    assert lib.pa_plan_test_wait_fault(plan.handle, item, 4096, _stream()) == 0, lib.pa_last_error()
    out = torch.full_like(g, float("nan"))
    plan.adjoint(fb, out=out)                  # returns; the output is incomplete
    torch.cuda.synchronize()
    assert plan.status() & WAIT_TIMEOUT
    plan.position_grad(g, fb)
    torch.cuda.synchronize()
    assert plan.status() & WAIT_TIMEOUT

    # hook off: the same results as before it (to the rounding of the NER
    # adjoint's shared-memory accumulation, whose order may vary)
    assert lib.pa_plan_test_wait_fault(plan.handle, -1, 0, _stream()) == 0
    assert _rel(plan.adjoint(fb).cpu(), ref) <= 1e-6
    assert _rel(plan.position_grad(g, fb)[1].cpu(), ref_xy) <= 1e-5
    assert plan.status() == 0
    plan.close()
