"""Back-to-back launches on one stream with no host synchronisation between
steps.  The pipeline kernels may be scheduled while the previous kernel of
the stream drains (programmatic dependent launch) and wait on the device for
its completion; these tests check that every step still sees the finished
results of the one before it and of the torch copies that refill its input:
the images of six steps issued back to back equal, bit for bit, the same
steps run one at a time with a synchronisation after each call, and so do
their adjoints up to the order of the NER adjoint's shared-memory sums."""
import numpy as np
import pytest
import torch

import synth

from test_gpu_parity import host, pa, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _problems():
    rng = np.random.default_rng(41)
    # 32x32 jittered sensors, Nt = Nz = 256: warp NER and every pipelined kernel
    warp = synth.Problem("warp_32x32x256", synth.jittered_lattice(rng, 32, 32, 1e-4, 1e-4),
                         np.full(1024, 1e-8), rng.normal(size=(1024, 256)), 20e-9, synth.C_WATER,
                         synth.Grid(32, 32, 256, 1e-4, 1e-4, 1e-4))
    return [synth.c1(), warp]


@pytest.mark.parametrize("which", [0, 1])
def test_back_to_back_steps_match_synchronised_steps(which):
    P = _problems()[which]
    plan = pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    if which == 1:
        assert plan.warp_ner
    rng = np.random.default_rng(42)
    srcs = [torch.tensor(rng.normal(size=P.g.shape), dtype=torch.float32, device="cuda") for _ in range(6)]
    # one call at a time, synchronised after each
    ref_f, ref_a = [], []
    for s in srcs:
        f = plan.reconstruct(s)
        torch.cuda.synchronize()
        a = plan.adjoint(f)
        torch.cuda.synchronize()
        ref_f.append(host(f))
        ref_a.append(host(a))
    # back to back: one input buffer refilled by a torch copy before every
    # step, one image buffer and one adjoint buffer reused by every step,
    # results copied out on the same stream
    g = torch.empty_like(srcs[0])
    f = torch.empty(P.grid.shape, dtype=torch.float32, device="cuda")
    a = torch.empty_like(g)
    outs_f = [torch.empty_like(f) for _ in srcs]
    outs_a = [torch.empty_like(a) for _ in srcs]
    for k, s in enumerate(srcs):
        g.copy_(s)
        plan.reconstruct(g, out=f)
        plan.adjoint(f, out=a)
        outs_f[k].copy_(f)
        outs_a[k].copy_(a)
    torch.cuda.synchronize()
    for k in range(len(srcs)):
        assert np.array_equal(host(outs_f[k]), ref_f[k]), k
        assert rel(host(outs_a[k]), ref_a[k]) <= 1e-6, k
    assert plan.status() == 0
    plan.close()
