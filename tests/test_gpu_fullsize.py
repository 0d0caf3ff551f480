"""Checks at the full size of the largest workload (65536 sensors, 1024
samples, 256x256x512 voxels), in the launch configuration of a single-plan
call: sampled outputs of every stage against the FP64 oracle evaluated one
column or one voxel at a time, the adjoint at sampled sensors against the
oracle's transposed chain, and the adjoint identity of the whole chain."""
import numpy as np
import pytest
import torch

import synth
from oracle import ndft, nufft

from test_gpu_parity import TOL, close, dev, host, plan_of, rel, sample_sensors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def c3():
    P = synth.c3()
    plan = plan_of(P)
    plan.autotune()  # the launch shapes the benchmark times
    f = host(plan.reconstruct(dev(P.g)))
    G1 = plan.buffer(0).cpu().numpy().astype(np.complex128)  # [jx + hx][jy][n], jy = 0..hy
    Fz = plan.buffer(1).cpu().numpy().astype(np.complex128)  # [jx + hx][iy][z]
    return P, plan, f, G1, Fz


def test_c3_spatial_spectrum_columns(c3):
    """G1 on sampled columns (Nyquist rows and corners included) against the
    direct sum over all 65536 sensors."""
    P, _, _, G1, _ = c3
    hx, hy = P.grid.nx // 2, P.grid.ny // 2
    cols = [(0, 0), (1, 0), (-hx, 5), (hx - 1, 64), (-3, hy), (hx, hy), (-hx, hy), (50, 77), (hx, 0)]
    for jx, jy in cols:
        exp = ndft.data_transform(P.xy, P.h, P.g, P.grid, [jx], [jy])[0, 0]
        close(G1[jx + hx, jy], exp, f"G1({jx},{jy})")


def test_c3_depth_profile_columns(c3):
    """After NER, weight, Hermitian part and inverse DFT over depth: sampled
    columns against the oracle's single-column evaluation of the definition
    (from the data, not from the GPU's intermediate)."""
    P, _, _, _, Fz = c3
    hx, hy = P.grid.nx // 2, P.grid.ny // 2
    # (jx, stored row iy); iy = hy holds the unpaired jy = -ny/2 of even ny
    cols = [(0, 0), (5, 3), (-hx, 7), (-hx, 0), (17, hy), (-hx, hy), (0, hy), (hx - 1, hy - 1), (-60, 90)]
    for jx, iy in cols:
        jy = -hy if (P.grid.ny % 2 == 0 and iy == hy) else iy
        exp = ndft.column_depth_profile(P.xy, P.h, P.g, P.dt, P.c, P.grid, jx, jy)
        close(Fz[jx + hx, iy], exp, f"Fz({jx},{jy})")


def test_c3_image_voxels_from_stage_input(c3):
    """The x and y inverse transforms at full size: sampled voxels of f against
    the oracle's voxel evaluation from the GPU's own half spectrum."""
    P, _, f, _, Fz = c3
    rng = np.random.default_rng(7)
    nx, ny, nz = P.grid.shape
    pts = list(zip(rng.integers(0, nx, 24), rng.integers(0, ny, 24), rng.integers(0, nz, 24)))
    pts += [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2, ny // 2, nz // 2)]
    exp = ndft.half_spectrum_voxels(Fz, P.grid, pts)
    got = np.array([f[p, q, k] for p, q, k in pts])
    close(got, exp, "sampled voxels")


def test_c3_adjoint_sampled_sensors(c3):
    """The adjoint A^T fbar at 48 sampled sensors (wrapping footprints, the
    centre, random draws) against the oracle: G1bar from the oracle's
    transposed chain (image adjoint, weight, NER adjoint at width 16), then
    the transposed eq:NUDFT2 sum over every (jx, jy) at each sensor."""
    P, plan, _, _, _ = c3
    fb = np.random.default_rng(10).normal(size=P.grid.shape).astype(np.float32).astype(np.float64)
    gb = host(plan.adjoint(dev(fb)))
    assert plan.status() == 0
    G1bar = nufft.spectrum_cotangent(fb, P.dt, P.c, P.grid, P.n_t, rows=16)
    S = sample_sensors(P, 48, seed=1)
    ref = ndft.data_transform_adjoint(P.xy[S], P.h[S], G1bar, P.grid)
    close(gb[S], ref, f"C3 adjoint, {len(S)} sensors")


def test_c3_adjoint_identity(c3):
    """<A g, f'> = <g, A^T f'> for the whole chain at full size (FP32)."""
    P, plan, f, _, _ = c3
    rng = np.random.default_rng(8)
    fb = rng.normal(size=P.grid.shape)
    gb = host(plan.adjoint(dev(fb)))
    lhs = float(np.vdot(f, fb))
    rhs = float(np.vdot(P.g.astype(np.float32).astype(np.float64), gb))
    err = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    print(f"C3 dot test: {err:.3e}")
    assert err <= 1e-5
