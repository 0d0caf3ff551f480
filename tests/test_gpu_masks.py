"""Plans driven by the equi-steradian and equiangular masks: sensors on a
subset of the grid nodes with weights h_m ~ r^3 (a strongly non-uniform
density), against the direct FP64 sums."""
import numpy as np
import pytest
import torch

import synth
from oracle import ndft
from paper_1501_02946_gb300 import masks

from test_gpu_parity import TOL, close, dev, host, pa, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("nodes,nz,nt,n,r0", [(32, 40, 64, 300, 1.2e-3), (27, 35, 50, 180, 0.8e-3)])
def test_equisteradian_plan_matches_direct_sums(nodes, nz, nt, n, r0):
    pitch = 1e-4
    grid = synth.Grid(nodes, nodes, nz, pitch, pitch, pitch)
    xy, h = masks.equisteradian_mask(n, nodes, pitch, r0)
    rng = np.random.default_rng(nodes)
    g = rng.normal(size=(xy.shape[0], nt))
    dt, c = 20e-9, 1500.0
    plan = pa().Plan(xy, nt, dt, c, grid.as_tuple(), weights=h)
    assert not plan.is_lattice
    f = host(plan.reconstruct(dev(g)))
    ref = ndft.reconstruct(xy, h, g, dt, c, grid)
    close(f, ref, f"equi-steradian {nodes}^2 M={xy.shape[0]} forward")
    fb = rng.normal(size=grid.shape)
    gb = host(plan.adjoint(dev(fb)))
    close(gb, ndft.reconstruct_adjoint(xy, h, fb, dt, c, grid, nt), f"equi-steradian {nodes}^2 M={xy.shape[0]} adjoint")
    assert plan.status() == 0
