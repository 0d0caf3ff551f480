"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance: relative L2 error <= 1e-4 against the FP64 oracle for every
reconstruction, adjoint and position gradient, and element by element
max |GPU - oracle| <= 1e-3 max |oracle| (so that an error confined to a few
elements -- one wrong Nyquist column, one bad tile halo -- cannot hide in the
norm); the FP32 NUFFT with a width-8 Kaiser-Bessel window is expected near
1e-6.  Dot-product tests of the GPU operator and its adjoint: <= 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import ndft, nufft

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1501_02946_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def pa():
    import paper_1501_02946_gb300 as m
    return m


def rel(a, b):
    """Relative L2 error; complex arrays are compared in full."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a = np.asarray(a, dtype=np.complex128 if cplx else np.float64)
    b = np.asarray(b, dtype=np.complex128 if cplx else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def close(got, ref, what, tol=TOL):
    """GPU result against the oracle: relative L2 error <= tol and max
    |got - ref| <= 10 tol max |ref| (1e-3 for the default 1e-4).  Returns
    the relative L2 error."""
    cplx = np.iscomplexobj(got) or np.iscomplexobj(ref)
    got = np.asarray(got, dtype=np.complex128 if cplx else np.float64)
    ref = np.asarray(ref, dtype=np.complex128 if cplx else np.float64)
    err = rel(got, ref)
    peak = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print(f"{what}: rel L2 = {err:.3e}, max abs err / max |ref| = {peak:.3e}")
    assert err <= tol, f"{what}: rel L2 {err:.3e}"
    assert peak <= 10 * tol, f"{what}: max abs err / max |ref| {peak:.3e}"
    return err


def sample_sensors(P, n, seed=0):
    """n sensor indices of a problem: sensors whose window footprint wraps
    round the periodic grid (within 4 oversampled cells of an edge), the ones
    nearest the centre, and a seeded random draw from each half of the sensor
    list (for the 128x128 workload: the jittered lattice, then the
    centre-dense half)."""
    X, Y = P.grid.nx * P.grid.dx, P.grid.ny * P.grid.dy
    ux = (P.xy[:, 0] / X + 0.5) % 1.0
    uy = (P.xy[:, 1] / Y + 0.5) % 1.0
    edge = np.minimum(np.minimum(ux, 1 - ux) * 2 * P.grid.nx, np.minimum(uy, 1 - uy) * 2 * P.grid.ny)
    rng = np.random.default_rng(seed)
    k = n // 4
    picks = list(np.argsort(edge)[:k])
    picks += list(np.argsort(np.hypot(P.xy[:, 0], P.xy[:, 1]))[:k])
    M = P.n_sensors
    picks += list(rng.choice(M // 2, k, replace=False))
    picks += list(M // 2 + rng.choice(M - M // 2, n - 3 * k, replace=False))
    return np.unique(np.array(picks))


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def plan_of(P, width=8, sigma=2):
    return pa().Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h, sigma=sigma, width=width)


def custom_problem(nsx, nsy, grid, n_t, dt=20e-9, seed=0, jitter=0.4):
    rng = np.random.default_rng(seed)
    xy = synth.jittered_lattice(rng, nsx, nsy, grid.dx, grid.dy, jitter)
    g = rng.normal(size=(xy.shape[0], n_t))
    X, Y = grid.nx * grid.dx, grid.ny * grid.dy
    return synth.Problem("custom", xy, np.full(xy.shape[0], X * Y / xy.shape[0]), g, dt, 1500.0, grid)


# ----------------------------------------------------------------- forward
@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_forward_matches_direct_sum(name):
    P = getattr(synth, name)()
    ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    plan = plan_of(P)
    f = host(plan.reconstruct(dev(P.g)))
    close(f, ref, f"{name} forward vs O1")
    assert plan.status() == 0


@pytest.mark.parametrize("grid,n_t,ns", [
    (synth.Grid(15, 21, 25, 1e-4, 1e-4, 1e-4), 45, (15, 21)),
    (synth.Grid(12, 9, 10, 1e-4, 1.5e-4, 1e-4), 36, (12, 9)),
    (synth.Grid(10, 14, 27, 1.2e-4, 1e-4, 0.8e-4), 50, (9, 13)),
    (synth.Grid(16, 8, 12, 1e-4, 1e-4, 1e-4), 35, (20, 11)),
])
def test_forward_odd_and_ragged_sizes(grid, n_t, ns):
    P = custom_problem(ns[0], ns[1], grid, n_t)
    ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    f = host(plan_of(P).reconstruct(dev(P.g)))
    close(f, ref, f"{grid.shape} nt={n_t} forward vs O1")


@pytest.mark.parametrize("width", [6, 12, 16])
def test_forward_other_widths(width):
    P = synth.c1()
    ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    close(host(plan_of(P, width=width).reconstruct(dev(P.g))), ref, f"width {width} forward vs O1",
          tol=3e-4 if width == 6 else TOL)


def test_sigma_three():
    P = synth.c1()
    ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    close(host(plan_of(P, sigma=3).reconstruct(dev(P.g))), ref, "sigma 3 forward vs O1")


# ----------------------------------------------------------- stage parity
def test_spatial_spectrum_stage():
    """G1 after the NED step against eq:NUDFT2 evaluated directly."""
    P = synth.c1()
    plan = plan_of(P)
    plan.reconstruct(dev(P.g))
    G1 = plan.buffer(0).cpu().numpy().astype(np.complex128)
    nx, ny = P.grid.nx, P.grid.ny
    hx, hy = nx // 2, ny // 2
    # the GPU keeps jx = -hx..hx and jy = 0..hy (the Hermitian half plus +N/2)
    exp = ndft.data_transform(P.xy, P.h, P.g, P.grid, np.arange(-hx, hx + 1), np.arange(0, hy + 1))
    close(G1, exp, "G1 vs eq:NUDFT2")


def test_time_frequency_stage():
    """Spectrum after NER, weight, Hermitian symmetrisation and inverse DFT
    over depth, against the direct sums of eq:disc_rec."""
    P = synth.c1()
    plan = plan_of(P)
    plan.reconstruct(dev(P.g))
    Fz = plan.buffer(1).cpu().numpy().astype(np.complex128)
    _, aux = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid, full=True)
    F = aux["F"]
    nx, ny, nz = P.grid.shape
    hx, hy, hz = nx // 2, ny // 2, nz // 2
    ia = (2 * hx - np.arange(nx)) % nx
    ib = (2 * hy - np.arange(ny)) % ny
    ic = (2 * hz - np.arange(nz)) % nz
    Fneg = F[np.ix_(ia, ib, ic)]
    Fsym = 0.5 * (F + np.conj(Fneg))
    l = ndft.freqs(nz)
    z = np.arange(nz)
    E = np.exp(2j * np.pi * np.outer(l, z) / nz)            # [l][z]
    # jy = 0..hy: array indices hy..ny-1, then (even ny) the Nyquist slot at index 0
    half = Fsym[:, hy:, :] if ny % 2 else np.concatenate([Fsym[:, hy:, :], Fsym[:, :1, :]], axis=1)
    exp = np.einsum("abl,lz->abz", half, E) / (nx * ny * nz)
    close(Fz, exp, "Fz vs direct sums")


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_adjoint_matches_direct_transpose(name):
    P = getattr(synth, name)()
    rng = np.random.default_rng(3)
    fb = rng.normal(size=P.grid.shape)
    ref = ndft.reconstruct_adjoint(P.xy, P.h, fb, P.dt, P.c, P.grid, P.n_t)
    got = host(plan_of(P).adjoint(dev(fb)))
    close(got, ref, f"{name} adjoint vs O1 transpose")


def _dot_test(P, plan, seed=4):
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(P.n_sensors, P.n_t))
    fb = rng.normal(size=P.grid.shape)
    Ag = host(plan.reconstruct(dev(g)))
    Atf = host(plan.adjoint(dev(fb)))
    g32 = g.astype(np.float32).astype(np.float64)
    f32 = fb.astype(np.float32).astype(np.float64)
    return abs(np.sum(Ag * f32) - np.sum(g32 * Atf)) / (np.linalg.norm(Ag) * np.linalg.norm(f32))


@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_dot_product_small(name):
    P = getattr(synth, name)()
    d = _dot_test(P, plan_of(P))
    print(f"{name}: dot test {d:.3e}")
    assert d <= 1e-5


def test_dot_product_odd_sizes():
    P = custom_problem(15, 21, synth.Grid(15, 21, 25, 1e-4, 1e-4, 1e-4), 45)
    assert _dot_test(P, plan_of(P)) <= 1e-5
    P = custom_problem(12, 9, synth.Grid(12, 9, 10, 1e-4, 1.5e-4, 1e-4), 36)
    assert _dot_test(P, plan_of(P)) <= 1e-5


# ------------------------------------------------------ position gradient
@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_position_gradient_matches_analytic(name):
    P = getattr(synth, name)()
    rng = np.random.default_rng(8)
    fb = rng.normal(size=P.grid.shape)
    ref = ndft.position_grad(P.xy, P.h, P.g, fb, P.dt, P.c, P.grid)
    plan = plan_of(P)
    gg, gxy = plan.position_grad(dev(P.g), dev(fb))
    close(host(gxy), ref, f"{name} position gradient vs O1")
    ref_g = ndft.reconstruct_adjoint(P.xy, P.h, fb, P.dt, P.c, P.grid, P.n_t)
    close(host(gg), ref_g, f"{name} data gradient vs O1")


def test_autograd_function():
    P = synth.c1()
    plan = plan_of(P)
    g = dev(P.g).requires_grad_(True)
    xy = torch.tensor(P.xy, dtype=torch.float64, requires_grad=True)
    f = pa().reconstruct(g, xy, plan)
    rng = np.random.default_rng(12)
    fb = dev(rng.normal(size=P.grid.shape))
    (f * fb).sum().backward()
    gg, gxy = plan.position_grad(dev(P.g), fb)
    assert rel(host(g.grad), host(gg)) <= 1e-6
    assert rel(xy.grad.numpy(), host(gxy)) <= 1e-6
    ref = ndft.position_grad(P.xy, P.h, P.g, host(fb), P.dt, P.c, P.grid)
    close(xy.grad.numpy(), ref, "autograd position gradient vs O1")


def test_update_positions_matches_new_plan():
    P = synth.c1()
    plan = plan_of(P)
    rng = np.random.default_rng(21)
    xy2 = P.xy + rng.normal(scale=2e-5, size=P.xy.shape)
    plan.update_positions(xy2)
    a = host(plan.reconstruct(dev(P.g)))
    b = host(pa().Plan(xy2, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h).reconstruct(dev(P.g)))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name", ["c1", "tiny"])
def test_update_positions_on_device_matches_host(name):
    """Re-binning on the device (float32 positions, FP64 cell coordinates)
    gives the tables of a host re-binning of the same positions: identical
    sensor order and entry lists, taps to float rounding, the same image to
    1e-6 and the same adjoint and position gradient."""
    P = getattr(synth, name)()
    rng = np.random.default_rng(22)
    xy2 = (P.xy + rng.normal(scale=3e-5, size=P.xy.shape)).astype(np.float32)
    # a few positions outside the period, reduced on the device
    X = P.grid.nx * P.grid.dx
    xy2[:3, 0] += np.float32(2 * X)
    plan_d = plan_of(P)
    plan_d.update_positions(torch.tensor(xy2, device="cuda"))
    plan_h = plan_of(P)
    plan_h.update_positions(xy2.astype(np.float64))
    g = dev(P.g)
    a, b = host(plan_d.reconstruct(g)), host(plan_h.reconstruct(g))
    err = rel(a, b)
    print(f"{name}: device vs host re-binning rel L2 = {err:.3e}")
    assert err <= 1e-6
    fb = dev(np.random.default_rng(23).normal(size=P.grid.shape))
    assert rel(host(plan_d.adjoint(fb)), host(plan_h.adjoint(fb))) <= 1e-6
    gd = host(plan_d.position_grad(g, fb)[1])
    gh = host(plan_h.position_grad(g, fb)[1])
    assert rel(gd, gh) <= 1e-5


def test_position_updates_that_grow_the_entry_lists():
    """Host and device position updates in turn, where a host update makes
    the spread entry lists grow (sensors whose base cells all sit at the
    last row of a strip meet two strips, lattice sensors three): every step
    gives the image of a fresh plan with those positions, and the device
    re-binning scratch and the lattice tables stay valid across the growth."""
    grid = synth.Grid(32, 32, 64, 1e-4, 1e-4, 1e-4)
    X = grid.nx * grid.dx
    rng = np.random.default_rng(25)
    n = 32
    # oversampled cell coordinate U = 64 x / X + 32 with floor(U) = 3 mod 4
    k = np.arange(n)
    U = (4 * (k % 16) + 3.25)[:, None] + np.zeros((1, n))
    V = (4 * (k % 16) + 3.5)[None, :] + np.zeros((n, 1))
    xy_few = np.stack([(U.ravel() - 32) * X / 64, (V.ravel() - 32) * X / 64], axis=1)
    xy_lat = synth.lattice_positions(32, 32, grid.dx, grid.dy)
    h = np.full(n * n, X * X / (n * n))
    g = rng.normal(size=(n * n, 64))
    gd = dev(g)

    def fresh(xy):
        return host(pa().Plan(xy, 64, 20e-9, 1500.0, grid.as_tuple(), weights=h).reconstruct(gd))

    plan = pa().Plan(xy_few, 64, 20e-9, 1500.0, grid.as_tuple(), weights=h)
    n0 = plan.info()
    xy_j = (xy_few + rng.uniform(-1e-6, 1e-6, xy_few.shape)).astype(np.float32)
    plan.update_positions(torch.tensor(xy_j, device="cuda"))          # device: re-binning scratch
    assert rel(host(plan.reconstruct(gd)), fresh(xy_j.astype(np.float64))) <= 1e-6
    plan.update_positions(xy_lat)                                       # host: the entry lists grow
    assert plan.is_lattice
    assert np.array_equal(host(plan.reconstruct(gd)), fresh(xy_lat))
    plan.update_positions(torch.tensor(xy_j, device="cuda"))          # device again, after the growth
    assert rel(host(plan.reconstruct(gd)), fresh(xy_j.astype(np.float64))) <= 1e-6
    plan.update_positions(xy_lat)
    assert np.array_equal(host(plan.reconstruct(gd)), fresh(xy_lat))
    assert plan.status() == 0
    assert n0["n_sensors"] == n * n
    plan.close()


def test_update_positions_on_device_rejects_nonfinite():
    P = synth.c1()
    plan = plan_of(P)
    xy = torch.tensor(P.xy.astype(np.float32), device="cuda")
    xy[5, 1] = float("nan")
    with pytest.raises(Exception):
        plan.update_positions(xy)
    # the status word is left as it was
    assert plan.status() == 0


@pytest.mark.parametrize("name", ["c1", "tiny"])
def test_autotune_keeps_results(name):
    """Every launch shape the autotuner may pick sums the forward in the same
    order (bit-identical image); the adjoint's shared-memory accumulation
    follows the NER block shape (equal to float rounding)."""
    P = getattr(synth, name)()
    plan = plan_of(P)
    g = dev(P.g)
    fb = dev(np.random.default_rng(24).normal(size=P.grid.shape))
    before = (host(plan.reconstruct(g)), host(plan.adjoint(fb)), host(plan.position_grad(g, fb)[1]))
    choice = plan.autotune()
    print(name, choice)
    assert choice["spread_samples_per_lane"] in (4, 8)
    assert choice["ner_columns_per_block"] in (2, 4)
    assert choice["ner_threads"] in (128, 256)
    assert choice["interp_tile_columns"] in (8, 16, 32)
    after = (host(plan.reconstruct(g)), host(plan.adjoint(fb)), host(plan.position_grad(g, fb)[1]))
    assert np.array_equal(before[0], after[0])
    assert rel(after[1], before[1]) <= 1e-6
    assert rel(after[2], before[2]) <= 1e-5


def test_profile_selected_stages():
    """Events around every launch, around the selected stages only, or none;
    the results do not depend on it."""
    P = synth.c1()
    plan = plan_of(P)
    g = dev(P.g)
    f0 = host(plan.reconstruct(g))
    plan.profile(True)
    f1 = plan.reconstruct(g)
    plan.adjoint(f1)
    every = plan.profile_read()
    assert {"ned_spread", "ner_fused", "ner_adj", "ned_interp"} <= set(every)
    plan.profile(True, stages=["ned_interp"])
    plan.reconstruct(g)
    plan.adjoint(f1)
    sel = plan.profile_read()
    assert set(sel) == {"ned_interp"}
    assert sel["ned_interp"][1] == 1 and sel["ned_interp"][0] > 0
    plan.profile(False)
    plan.reconstruct(g)
    assert plan.profile_read() == {}
    assert np.array_equal(f0, host(f1))
    with pytest.raises(ValueError):
        plan.profile(True, stages=["no_such_stage"])


# ---------------------------------------------------------- edge cases
def test_positions_wrap_by_period():
    P = synth.c1()
    X = P.grid.nx * P.grid.dx
    a = host(plan_of(P).reconstruct(dev(P.g)))
    Q = synth.Problem("w", P.xy + np.array([X, -3 * X]), P.h, P.g, P.dt, P.c, P.grid)
    b = host(plan_of(Q).reconstruct(dev(P.g)))
    assert rel(b, a) <= 1e-5


def test_single_sensor_and_one_cell():
    grid = synth.Grid(8, 8, 16, 1e-4, 1e-4, 1e-4)
    rng = np.random.default_rng(2)
    for xy in (np.array([[1.3e-5, -2.2e-4]]), np.full((40, 2), 3.1e-5) + rng.uniform(0, 1e-6, (40, 2))):
        g = rng.normal(size=(xy.shape[0], 32))
        h = np.full(xy.shape[0], 6.4e-7 / xy.shape[0])
        ref = ndft.reconstruct(xy, h, g, 40e-9, 1500.0, grid)
        got = host(pa().Plan(xy, 32, 40e-9, 1500.0, grid.as_tuple(), weights=h).reconstruct(dev(g)))
        close(got, ref, f"{xy.shape[0]} sensor(s) in one cell, forward vs O1")


def test_zero_data_gives_zero_image():
    P = synth.tiny()
    f = host(plan_of(P).reconstruct(dev(np.zeros_like(P.g))))
    assert np.all(f == 0.0)


# ------------------------------------------------------ baseline and batch
def test_cubic_baseline_is_less_accurate():
    P = synth.c1()
    ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    plan = plan_of(P)
    e_nufft = rel(host(plan.reconstruct(dev(P.g))), ref)
    e_cubic = rel(host(plan.reconstruct_cubic(dev(P.g))), ref)
    print(f"cubic baseline rel L2 = {e_cubic:.3e} (NUFFT {e_nufft:.3e})")
    assert e_nufft < e_cubic < 1.0


def test_staged_spread_rows_past_the_buffer():
    """Four sensors per output cell (one per oversampled cell): every spread
    block's union of g rows (about 165) is longer than the rows its shared
    buffer holds (sized so that four blocks share an SM), so most rows come
    from global memory.  The forward equals the unstaged spread's (the batch's
    stage mode) bit for bit, and the oracle."""
    rng = np.random.default_rng(31)
    n, nt = 32, 64
    grid = synth.Grid(n, n, 64, 1e-4, 1e-4, 1e-4)
    xy = synth.jittered_lattice(rng, 2 * n, 2 * n, grid.dx / 2, grid.dy / 2)
    X = n * grid.dx
    P = synth.Problem("dense", xy, np.full(xy.shape[0], X * X / xy.shape[0]), rng.normal(size=(xy.shape[0], nt)),
                      20e-9, 1500.0, grid)
    plan = plan_of(P)
    g = dev(P.g)
    f = host(plan.reconstruct(g))
    assert plan.status() == 0
    fs = torch.empty(plan.image_shape, device="cuda")
    pa().Batch([plan], mode=1).run([g], [fs])
    assert np.array_equal(host(fs), f)
    close(f, ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid), "dense sensors forward vs O1")


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_matches_single_plans(mode):
    rng = np.random.default_rng(5)
    probs = [synth.batch_instance(rng, n, t, n_balls=2) for n, t in ((16, 32), (21, 48), (12, 64), (20, 40))]
    plans = [plan_of(P) for P in probs]
    gs = [dev(P.g) for P in probs]
    singles = [host(p.reconstruct(g)) for p, g in zip(plans, gs)]
    B = pa().Batch(plans, mode=mode)
    fs = [torch.empty(p.image_shape, device="cuda") for p in plans]
    for _ in range(3):  # first run captures the graph, later runs replay it
        for f in fs:
            f.zero_()
        B.run(gs, fs)
        for f, s in zip(fs, singles):
            assert np.array_equal(host(f), s)
    for k, (P, f) in enumerate(zip(probs, fs)):
        ref = ndft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
        close(host(f), ref, f"batch mode {mode} instance {k} vs O1")


def test_batch_with_fast_path_sizes():
    """Instances whose single plans take the warp NER and tensor-map kernels:
    mode 0 replays exactly those launches (bit-identical), mode 1 runs the
    general stage kernels over all instances (same operator to rounding)."""
    rng = np.random.default_rng(6)
    probs = [synth.batch_instance(rng, n, t, n_balls=2) for n, t in ((64, 256), (70, 128), (32, 512), (64, 128))]
    plans = [plan_of(P) for P in probs]
    gs = [dev(P.g) for P in probs]
    singles = [host(p.reconstruct(g)) for p, g in zip(plans, gs)]
    refs = [nufft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid) for P in probs]   # O2, width 16
    for mode in (0, 1):
        B = pa().Batch(plans, mode=mode)
        fs = [torch.empty(p.image_shape, device="cuda") for p in plans]
        for _ in range(2):
            B.run(gs, fs)
            for f, s in zip(fs, singles):
                if mode == 0:
                    assert np.array_equal(host(f), s)
                else:
                    assert rel(host(f), s) <= 1e-5
        for k, (f, ref) in enumerate(zip(fs, refs)):
            close(host(f), ref, f"batch mode {mode} instance {k} {probs[k].grid.shape} vs O2")
        B.close()


# ----------------------------------------------------------- full size
@pytest.fixture(scope="module")
def c2():
    return synth.c2()


def test_c2_forward_matches_nufft_oracle(c2):
    P = c2
    ref = nufft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid, 2, 12)
    f = host(plan_of(P).reconstruct(dev(P.g)))
    close(f, ref, "C2 forward vs O2(w=12)")


def test_c2_adjoint_and_dot(c2):
    P = c2
    plan = plan_of(P)
    rng = np.random.default_rng(6)
    fb = rng.normal(size=P.grid.shape)
    ref = nufft.reconstruct_adjoint(P.xy, P.h, fb, P.dt, P.c, P.grid, P.n_t, 2, 12)
    close(host(plan.adjoint(dev(fb))), ref, "C2 adjoint vs O2(w=12)")
    assert _dot_test(P, plan) <= 1e-5


def test_c2_position_gradient_sampled_sensors(c2):
    """The position gradient (and the data gradient) of the autotuned plan the
    benchmark times, at the full 128x128x256 size, on sampled sensors
    (footprints that wrap round the grid, the centre-dense region, random
    draws from both halves) against the oracle: the cotangent G1bar of the
    spatial spectrum from the oracle's transposed chain (image adjoint,
    weight, NER adjoint at width 16), then the analytic derivative of
    eq:NUDFT2 at each sampled sensor."""
    P = c2
    plan = plan_of(P)
    plan.autotune()
    assert plan.warp_ner
    fb = np.random.default_rng(9).normal(size=P.grid.shape).astype(np.float32).astype(np.float64)
    gg, gxy = plan.position_grad(dev(P.g), dev(fb))
    G1bar = nufft.spectrum_cotangent(fb, P.dt, P.c, P.grid, P.n_t, rows=32)
    S = sample_sensors(P, 80)
    g32 = P.g.astype(np.float32).astype(np.float64)
    ref_xy = ndft.position_grad_from_cotangent(P.xy[S], P.h[S], g32[S], G1bar, P.grid)
    close(host(gxy)[S], ref_xy, f"C2 position gradient, {len(S)} sensors")
    ref_g = ndft.data_transform_adjoint(P.xy[S], P.h[S], G1bar, P.grid)
    close(host(gg)[S], ref_g, f"C2 data gradient, {len(S)} sensors")
    assert plan.status() == 0


def test_c2_autotuned_plan_matches_default(c2):
    """The benchmark times an autotuned plan: whichever launch shapes the
    tuner keeps at the full 128x128x256 size, the forward is bit-identical to
    the default plan's (checked against O2 above) and the adjoint and the
    position gradient agree to float rounding."""
    P = c2
    plan_d, plan_t = plan_of(P), plan_of(P)
    choice = plan_t.autotune()
    print("C2 tuned shapes:", choice)
    g = dev(P.g)
    fb = dev(np.random.default_rng(7).normal(size=P.grid.shape))
    assert np.array_equal(host(plan_t.reconstruct(g)), host(plan_d.reconstruct(g)))
    assert rel(host(plan_t.adjoint(fb)), host(plan_d.adjoint(fb))) <= 1e-6
    assert rel(host(plan_t.position_grad(g, fb)[1]), host(plan_d.position_grad(g, fb)[1])) <= 1e-5
    assert plan_t.status() == 0
