#!/usr/bin/env python3
"""Throughput of the GB300 NEDNER-NUFFT: one step = one forward
reconstruction and one adjoint (f = A g, then A^T f) of the large single
reconstruction (65536 dart-thrown sensors over 25.6 mm, 1024 samples at
10 ns, 256x256x512 voxels).

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): each rank runs its own
replica of the workload ("replicas only": a single reconstruction does not
shard without a collective), timing is the max over ranks and `value` counts
the voxels of all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the NUFFT algorithm in numpy) on
the host cores instead, on a bounded sample of the same workload (tiles of
the aperture, one oracle process per core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxels/s (NEDNER-NUFFT fwd+adjoint, FP32, ≤1e-4 rel L2 vs FP64) and HBM roofline %"
UNIT = "voxels/s"
WORKLOAD = ("256x256 non-equispaced sensors: 65536 random-uniform over 25.6 mm (dart throwing, minimum "
            "spacing 40 um), 1024 samples at 10 ns, 20 balls + 6 vessels (chains of balls, 638 sources), "
            "output 256x256x512 at 100 um, sigma 2, width 8")
WORKLOAD_C2 = ("128x128 non-equispaced sensors over 12.8 mm (8192 jittered lattice + 8192 centre-dense), "
               "512 samples at 20 ns, 20 balls + 1% noise, output 128x128x256 at 100 um, sigma 2, width 8")
STAGES = ["ned_spread", "ned_rowfft", "ned_colfft", "ner_fused", "image_x", "image_y_c2r", "image_y_adj",
          "image_x_adj", "ner_adj", "ned_colfft_adj", "ned_rowifft", "ned_interp"]


def stage_bytes(M, Nt, Nx, Ny, Nz, sigma=2):
    """Algorithmic bytes per launch of each kernel: its input read once and
    its output written once (complex64 = 8 B, float32 = 4 B)."""
    Mx = sigma * Nx
    nX1, nY1 = 2 * (Nx // 2) + 1, Ny // 2 + 1
    g = 4 * M * Nt
    T = 8 * Mx * nY1 * Nt
    G1 = 8 * nX1 * nY1 * Nt
    F = 8 * Nx * nY1 * Nz
    f = 4 * Nx * Ny * Nz
    G0 = 4 * Mx * (sigma * Ny) * Nt
    return {"ned_spread": g + G0, "ned_rowfft": G0 + T, "ned_colfft": T + G1, "ner_fused": G1 + F, "image_x": 2 * F,
            "image_y_c2r": F + f, "image_y_adj": f + F, "image_x_adj": 2 * F, "ner_adj": F + G1,
            "ned_colfft_adj": G1 + T, "ned_rowifft": T + G0,
            "ned_interp": G0 + g}


def pipeline_min_bytes(M, Nt, Nx, Ny, Nz):
    """Minimum HBM bytes of one forward (and, mirrored, one adjoint): read g,
    write f, round-trip the spatial spectrum and the image spectrum once."""
    nY1 = Ny // 2 + 1
    return 4 * M * Nt + 4 * Nx * Ny * Nz + 2 * 8 * Nx * nY1 * Nt + 2 * 8 * Nx * nY1 * Nz


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1501_02946_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as fh:
                h.update(fn.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(stage):
    """DRAM bytes per launch of `stage` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    v = d.get("bytes_per_launch", {}).get(stage)
    return None if v is None else float(v)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def tile_problem(P, s, i, j):
    """Tile (i, j) of an s x s tiling of a workload's aperture: the sensors in
    that (X/s) x (Y/s) square, moved so the tile is centred on (0, 0), with
    the matching (nx/s) x (ny/s) x nz output grid and uniform weights."""
    import numpy as np
    import synth
    if s == 1:
        return P
    gr = P.grid
    X, Y = gr.nx * gr.dx, gr.ny * gr.dy
    x0, y0 = -X / 2 + i * X / s, -Y / 2 + j * Y / s
    keep = (P.xy[:, 0] >= x0) & (P.xy[:, 0] < x0 + X / s) & (P.xy[:, 1] >= y0) & (P.xy[:, 1] < y0 + Y / s)
    grid = synth.Grid(gr.nx // s, gr.ny // s, gr.nz, gr.dx, gr.dy, gr.dz)
    M = int(keep.sum())
    xy = P.xy[keep] - np.array([x0 + X / (2 * s), y0 + Y / (2 * s)])
    h = np.full(M, (X / s) * (Y / s) / M)
    return synth.Problem(P.name + f"_tile{s}_{i}_{j}", xy, h, P.g[keep], P.dt, P.c, grid)


def _oracle_worker(args):
    """One FP64 forward + adjoint of the NUFFT oracle (as it stands) on one
    tile, in a worker process with one BLAS/FFT thread.  Returns the seconds
    it took, its voxels, and (if asked) the forward image."""
    xy, h, g, dt, c, grid_t, want_f = args
    import synth
    from oracle import nufft
    grid = synth.Grid(*grid_t)
    t0 = time.perf_counter()
    f = nufft.reconstruct(xy, h, g, dt, c, grid)
    nufft.reconstruct_adjoint(xy, h, f, dt, c, grid, g.shape[1])
    return time.perf_counter() - t0, grid.nx * grid.ny * grid.nz, (f if want_f else None)


def oracle_pool(n):
    """A pool of n spawned oracle workers, each with one BLAS/FFT thread (the
    environment is set before the workers start; spawn, so that no worker is
    forked from a process that holds a CUDA context)."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(n)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_tiles(P, s, k0, n, want_first=False):
    """Arguments of n oracle tasks: tiles k0, k0 + 1, .. (mod s*s) of an s x s
    tiling of P."""
    out = []
    for k in range(k0, k0 + n):
        i, j = divmod(k % (s * s), s)
        T = tile_problem(P, s, i, j)
        out.append((T.xy, T.h, T.g, T.dt, T.c, T.grid.as_tuple(), want_first and k == k0))
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    """The FP64 oracle on the host cores: every step runs one tile of the
    workload's aperture per core at once (tiles cycle through the tiling);
    value = the tiles' voxels / the step's wall time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    P = synth.c3()
    cores = min(host_cores(), 32)
    n = args.steps + args.warmup
    # tile size: 64x64x512 tiles take about 20 s each on one core, 32x32x512
    # about a fifth of that; keep the whole run within about three minutes
    s = 4 if n * 20.0 <= 180.0 else 8
    pool = oracle_pool(cores)
    times, vox = [], 0
    try:
        for k in range(n):
            tasks = oracle_tiles(P, s, k * cores, cores)
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, tasks)
            t = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(t)
                vox = sum(r[1] for r in res)
    finally:
        pool.close()
        pool.join()
    ms = 1e3 * sum(times) / len(times)
    value = vox / (ms / 1e3)
    sample = (f"{cores} tiles of {256 // s}x{256 // s}x512 per step (a {s}x{s} tiling of the 256x256 aperture, "
              f"each tile's sensors re-centred, 1024 samples), one tile per core at once, one FP64 "
              f"forward+adjoint per tile")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample, "oracle": "FP64 NUFFT (numpy), width 16"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def cpu_baseline(P, pa, dev):
    """The oracle on all host cores: one 64x64x512 tile of the workload per
    core, run at once (one step's worth of a 4x4 tiling, cycling); plus the
    accuracy of the GPU forward and of the cubic baseline on the first tile
    against the oracle's FP64 forward image."""
    import numpy as np
    import torch
    cores = min(host_cores(), 32)
    s = 4
    tasks = oracle_tiles(P, s, 0, cores, want_first=True)
    pool = oracle_pool(cores)
    try:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, tasks)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    vox = sum(r[1] for r in res)
    xy, h, g, dt, c, grid_t, _ = tasks[0]
    ref = res[0][2]
    tile = pa.Plan(xy, g.shape[1], dt, c, grid_t, weights=h)
    gd = torch.tensor(g, dtype=torch.float32, device=dev)
    f_n = tile.reconstruct(gd).double().cpu().numpy()
    f_c = tile.reconstruct_cubic(gd).double().cpu().numpy()
    tile.close()
    nrm = np.linalg.norm(ref)
    acc = {"tile": f"{grid_t[0]}x{grid_t[1]}x{grid_t[2]}, {g.shape[0]} sensors, 1024 samples",
           "nedner_rel_l2_vs_fp64_oracle": float(np.linalg.norm(f_n - ref) / nrm),
           "cubic_rel_l2_vs_fp64_oracle": float(np.linalg.norm(f_c - ref) / nrm)}
    sample = (f"{cores} tiles of 64x64x512 (a 4x4 tiling of the 256x256 aperture, each tile's sensors "
              f"re-centred, 1024 samples), one FP64 forward+adjoint per tile, one tile per core at once")
    return {"value": vox / wall, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": wall, "per_tile_seconds": [r[0] for r in res]}, acc


def batch_timings(pa, synth, dev, steps, warmup, tune=True):
    """The uneven batch (64 instances, N uniform over the 7-smooth integers in
    [64, 256], T in {256, 512, 1024}, output N x N x 2T), seeded random data:
    pa_batch_run in its two modes against 64 sequential single-plan calls."""
    import numpy as np
    import torch
    shapes = synth.batch_shapes()
    rng = np.random.default_rng(1505)
    plans, gs, fs = [], [], []
    voxels = 0
    for n_side, n_t in shapes:
        xy = synth.jittered_lattice(rng, n_side, n_side, 1e-4, 1e-4)
        grid = (n_side, n_side, 2 * n_t, 1e-4, 1e-4, 1e-4)
        p = pa.Plan(xy, n_t, 20e-9, synth.C_WATER, grid)
        if tune:
            p.autotune()
        plans.append(p)
        gs.append(torch.randn(n_side * n_side, n_t, device=dev, dtype=torch.float32))
        fs.append(torch.empty(n_side, n_side, 2 * n_t, device=dev, dtype=torch.float32))
        voxels += n_side * n_side * 2 * n_t
    batch = pa.Batch(plans)
    batch_st = pa.Batch(plans, mode=1)
    stream = torch.cuda.current_stream(dev)

    def seq():
        for p, g, f in zip(plans, gs, fs):
            p.reconstruct(g, out=f)

    res = {}
    for name, fn in (("batch_graph", lambda: batch.run(gs, fs)),
                     ("batch_graph_stage_launches", lambda: batch_st.run(gs, fs)),
                     ("sequential_64", seq)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.median(a.elapsed_time(b) for a, b in evs)
        res[name] = {"ms": ms, "voxels_per_s": voxels / (ms / 1e3)}
    batch.close()
    batch_st.close()
    for p in plans:
        p.close()
    best = min(res["batch_graph"]["ms"], res["batch_graph_stage_launches"]["ms"])
    return {"workload": "64 instances, N in 7-smooth [64, 256], T in {256, 512, 1024}, output N x N x 2T, "
                        "forward; plans autotuned" if tune else "64 instances (untuned plans)",
            "total_voxels": voxels, "median_of": steps, **res,
            "speedup_vs_sequential": res["sequential_64"]["ms"] / best}
def timed_median(fn, k, flush, stream, dev):
    """Median of k CUDA-event timings of fn() (L2 flushed before each, outside
    the events), after two untimed calls."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for _ in range(2):
        fn()
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize(dev)
    return statistics.median(a.elapsed_time(b) for a, b in evs)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1501_02946_gb300 as pa
    import synth

    if args.case == "columns128":
        # the large workload's sample count, depth and kernel instantiations on
        # a 128x128 grid (16384 dart-thrown sensors, random data): a case small
        # enough for a profiler's full metric set
        import numpy as np
        rng = np.random.default_rng(7)
        xy = synth.dart_throwing(rng, 128 * 128, 128 * 0.5e-4, 4e-5)
        grid = synth.Grid(128, 128, 512, 1e-4, 1e-4, 1e-4)
        P = synth.Problem("columns128", xy, np.full(xy.shape[0], (128e-4) ** 2 / xy.shape[0]),
                          rng.normal(size=(xy.shape[0], 1024)), 10e-9, synth.C_WATER, grid)
    elif args.case == "rows256":
        # the large workload's grid, sensors and depth with 256 samples: its
        # spatial and image transform lengths (512-point row and column FFTs,
        # 256-point image transforms) at a quarter of its G0
        import numpy as np
        P0 = synth.c3()
        P = synth.Problem("rows256", P0.xy, P0.h, np.random.default_rng(7).normal(size=(P0.xy.shape[0], 256)),
                          P0.dt, P0.c, P0.grid)
    else:
        P = synth.c3()
    Nx, Ny, Nz = P.grid.shape
    voxels = Nx * Ny * Nz
    plan = pa.Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    # plan setup, outside the timed region; a profiled step keeps the default
    # shapes (what the tuner keeps at this size) so that a profiler's slowdown
    # of the tuning launches cannot change them
    shapes = plan.autotune() if not args.profile_step else "default"
    g = torch.tensor(P.g, dtype=torch.float32, device=dev)
    f = torch.empty(P.grid.shape, dtype=torch.float32, device=dev)
    g2 = torch.empty_like(g)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.reconstruct(g, out=f)
        plan.adjoint(f, out=g2)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if args.profile_step:
        # one forward + adjoint between cudaProfilerStart/Stop, for
        # `ncu --profile-from-start off`; no timing line
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
        print(json.dumps({"profiled": "one forward + adjoint step", "launch_shapes": shapes}))
        return 0
    # per-stage times: one profiled pass of the same steps, events around
    # every launch (they sit between the kernels and lengthen the step, so
    # this pass is not the timed one)
    plan.profile(True)
    plan.profile_read()
    ev_p = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev_p[k][0].record(stream)
        step()
        ev_p[k][1].record(stream)
    torch.cuda.synchronize(dev)
    profiled_ms = sum(a.elapsed_time(b) for a, b in ev_p) / args.steps
    prof = plan.profile_read()
    # the timed region: events around the dominant kernel's launches only
    dom = max(prof, key=lambda k: prof[k][0])
    plan.profile(True, stages=[dom])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(dev.index if world == 1 else int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (256 MiB written), outside the events
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    gpu_ms = sum(a.elapsed_time(b) for a, b in ev)
    prof_dom = plan.profile_read()[dom]
    plan.profile(False)
    if world > 1:
        t = torch.tensor([gpu_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        gpu_ms = float(t.item())
    ms_per_step = gpu_ms / args.steps
    value = world * voxels / (ms_per_step / 1e3)

    # roofline of the dominant kernel (largest device time in the profiled
    # pass); its launch time comes from the events of the timed region
    peaks, peak_kind = measured_peaks()
    sb = stage_bytes(P.n_sensors, P.n_t, Nx, Ny, Nz)
    dom_ms = prof_dom[0] / prof_dom[1]
    achieved = sb[dom] / (dom_ms / 1e3) / 1e9
    hbm = float(peaks["hbm_gbs"])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": ncu_traffic(dom), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": sb[dom], "launch_ms": dom_ms,
                "launch_timing": "CUDA events around this kernel's launches inside the timed region"}
    stages = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                  "gbs": sb[k] / (v[0] / v[1] / 1e3) / 1e9 if k in sb else None,
                  "frac_of_hbm": sb[k] / (v[0] / v[1] / 1e3) / 1e9 / hbm if k in sb else None,
                  "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()}
    pipe = 2 * pipeline_min_bytes(P.n_sensors, P.n_t, Nx, Ny, Nz)
    pipeline = {"min_bytes_per_step": pipe, "achieved_gbs": pipe / (ms_per_step / 1e3) / 1e9,
                "frac": pipe / (ms_per_step / 1e3) / 1e9 / hbm}

    k_parts = max(3, min(args.steps, 10))

    def timed(fn):
        return timed_median(fn, k_parts, flush, stream, dev)

    # forward alone, adjoint alone, the cubic-in-omega baseline forward and
    # the position gradient of the same plan
    fwd_ms = timed(lambda: plan.reconstruct(g, out=f))
    adj_ms = timed(lambda: plan.adjoint(f, out=g2))
    cub_ms = timed(lambda: plan.reconstruct_cubic(g, out=f))
    f_cub = plan.reconstruct_cubic(g).double()
    f_ned = plan.reconstruct(g, out=f).double()
    cub_vs_ned = float(torch.linalg.norm(f_cub - f_ned) / torch.linalg.norm(f_ned))
    del f_cub, f_ned
    fb3 = torch.randn(P.grid.shape, device=dev, dtype=torch.float32)
    pg3_ms = timed(lambda: plan.position_grad(g, fb3))
    del fb3
    # library comparison (bench only): cuFFT (through torch.fft) doing the
    # row and column transforms of the same oversampled grid, without the
    # deconvolution, truncation and pair packing that the kernels fuse
    Mx, My = 2 * Nx, 2 * Ny
    g0 = torch.randn(Mx, My, P.n_t, device=dev, dtype=torch.float32)

    def cufft_rows_cols():
        t = torch.fft.rfft(g0, dim=1)[:, : Ny // 2 + 1, :]
        return torch.fft.fft(t, dim=0)
    cufft_ms = timed(cufft_rows_cols)
    del g0
    own_rc = (prof["ned_rowfft"][0] / prof["ned_rowfft"][1] + prof["ned_colfft"][0] / prof["ned_colfft"][1]
              if "ned_rowfft" in prof and "ned_colfft" in prof else None)

    # the 128x128 sensor workload (the single reconstruction at 128x128x256)
    Q = synth.c2()
    voxels2 = int(np.prod(Q.grid.shape))
    plan2 = pa.Plan(Q.xy, Q.n_t, Q.dt, Q.c, Q.grid.as_tuple(), weights=Q.h)
    plan2.autotune()
    q_g = torch.tensor(Q.g, dtype=torch.float32, device=dev)
    q_f = torch.empty(Q.grid.shape, dtype=torch.float32, device=dev)
    q_g2 = torch.empty_like(q_g)

    def step2():
        plan2.reconstruct(q_g, out=q_f)
        plan2.adjoint(q_f, out=q_g2)
    c2_ms = timed(step2)
    c2_fwd_ms = timed(lambda: plan2.reconstruct(q_g, out=q_f))
    c2_adj_ms = timed(lambda: plan2.adjoint(q_f, out=q_g2))
    c2_cub_ms = timed(lambda: plan2.reconstruct_cubic(q_g, out=q_f))
    # the same output grid and samples with the sensors on the output lattice
    # (the lattice spatial step: no window spreading)
    xy_l = synth.lattice_positions(128, 128, Q.grid.dx, Q.grid.dy)
    plan_l = pa.Plan(xy_l, Q.n_t, Q.dt, Q.c, Q.grid.as_tuple())
    g_l = torch.randn(128 * 128, Q.n_t, device=dev, dtype=torch.float32)

    def lattice_step():
        plan_l.reconstruct(g_l, out=q_f)
        plan_l.adjoint(q_f, out=g_l)
    lat_ms = timed(lattice_step) if plan_l.is_lattice else None
    plan_l.close()
    del g_l
    # the d = 2 operator: 256 sensors on a 51.2 mm line (jittered, centre-dense),
    # 1024 samples at 20 ns, image 512 x 512 at 100 um
    rng2 = np.random.default_rng(1507)
    nx2, nz2, nt2, m2 = 512, 512, 1024, 256
    X2 = nx2 * 1e-4
    x2 = np.sort(np.concatenate([rng2.uniform(-X2 / 2, X2 / 2, m2 // 2),
                                 rng2.normal(0.0, X2 / 8, m2 // 2).clip(-X2 / 2, X2 / 2 - 1e-7)]))
    plan_2 = pa.Plan2D(x2, nt2, 20e-9, Q.c, (nx2, nz2, 1e-4, 1e-4))
    g_2 = torch.randn(m2, nt2, device=dev, dtype=torch.float32)
    f_2 = torch.empty(nx2, nz2, device=dev, dtype=torch.float32)

    def d2_step():
        plan_2.reconstruct(g_2, out=f_2)
        plan_2.adjoint(f_2, out=g_2)
    d2_ms = timed(d2_step)
    plan_2.close()
    del g_2, f_2
    # the position gradient (data gradient A^T fbar included) alone, and the
    # variational workload at 128x128x256: L = ||A(xy) g - target||^2 +
    # 1e-3 TV_eps(A(xy) g), eps = 1e-8 (isotropic, forward differences),
    # target = the phantom's balls sampled at the voxel centres, backpropagated
    # to g and xy through the autograd function (loss terms in torch, FP64 sums;
    # positions as a CUDA tensor, re-binned on the device when they change)
    fb_v = torch.randn(Q.grid.shape, device=dev, dtype=torch.float32)
    pg_ms = timed(lambda: plan2.position_grad(q_g, fb_v))
    target_d = torch.tensor(Q.voxelised(), dtype=torch.float32, device=dev)
    xy_v = torch.tensor(Q.xy, dtype=torch.float32, device=dev, requires_grad=True)
    g_v = q_g.detach().clone().requires_grad_(True)

    def var_loss(fv):
        fv = fv.to(torch.float64)
        d0 = torch.diff(fv, dim=0, append=fv[-1:])
        d1 = torch.diff(fv, dim=1, append=fv[:, -1:])
        d2 = torch.diff(fv, dim=2, append=fv[:, :, -1:])
        r = fv - target_d
        return (r * r).sum() + 1e-3 * torch.sqrt(d0 * d0 + d1 * d1 + d2 * d2 + 1e-8).sum()

    def var_step():
        g_v.grad = None
        xy_v.grad = None
        var_loss(pa.reconstruct(g_v, xy_v, plan2)).backward()
    var_ms = timed(var_step)
    del fb_v, target_d, g_v
    plan2.close()
    del q_g, q_f, q_g2
    torch.cuda.empty_cache()
    batch = batch_timings(pa, synth, dev, steps=5, warmup=3) if not args.no_batch else None
    parts = {"forward": {"ms": fwd_ms, "voxels_per_s": voxels / (fwd_ms / 1e3)},
             "adjoint": {"ms": adj_ms, "voxels_per_s": voxels / (adj_ms / 1e3)},
             "cubic_baseline_forward": {"ms": cub_ms, "voxels_per_s": voxels / (cub_ms / 1e3),
                                        "rel_l2_vs_nedner_forward": cub_vs_ned},
             "position_grad": {"ms": pg3_ms, "voxels_per_s": voxels / (pg3_ms / 1e3),
                               "what": "pa_position_grad: A^T fbar and dL/dxy of <fbar, A(xy) g>"},
             "cufft_row_col_transforms_ms": cufft_ms, "own_row_col_transforms_ms": own_rc,
             "c2_fwd_adj": {"workload": WORKLOAD_C2, "ms": c2_ms, "voxels_per_s": voxels2 / (c2_ms / 1e3),
                            "forward_ms": c2_fwd_ms, "adjoint_ms": c2_adj_ms, "cubic_forward_ms": c2_cub_ms,
                            "position_grad_ms": pg_ms,
                            "variational_fwd_bwd_ms": var_ms,
                            "variational_what": "L = ||A(xy) g - target||^2 + 1e-3 TV_eps(A(xy) g); forward, "
                                                "loss and backward to g and xy through the autograd function",
                            "lattice_sensors_fwd_adj_ms": lat_ms},
             "d2_fwd_adj": {"ms": d2_ms, "pixels_per_s": nx2 * nz2 / (d2_ms / 1e3),
                            "workload": f"d = 2: {m2} sensors on a {X2 * 1e3:.1f} mm line, {nt2} samples at 20 ns, "
                                        f"image {nx2}x{nz2} at 100 um"},
             "batch": batch,
             "median_of": k_parts}

    # end to end through the public API with host buffers: every step copies
    # its input g from pinned host memory and its results (f and the adjoint's
    # g') back.  Serial: copy, compute, copy on one stream.  Pipelined (the
    # reported value): three device buffer sets and three streams, so the H2D
    # copy of step k + 1 and the D2H copies of step k overlap the compute.
    g_h = torch.tensor(P.g, dtype=torch.float32).pin_memory()
    f_h = torch.empty(P.grid.shape, dtype=torch.float32).pin_memory()
    g2_h = torch.empty(g_h.shape, dtype=torch.float32).pin_memory()
    n_e2e = min(args.steps, 10)
    for _ in range(2):
        g.copy_(g_h, non_blocking=True)
        step()
        f_h.copy_(f, non_blocking=True)
        g2_h.copy_(g2, non_blocking=True)
    torch.cuda.synchronize(dev)
    # each end-to-end figure is the median of E2E_REPEATS runs of n_e2e steps:
    # the host copies share the machine's host memory with other jobs, and a
    # single copy has been seen to stall for several milliseconds
    E2E_REPEATS = 3
    serial_runs = []
    for _ in range(E2E_REPEATS):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            g.copy_(g_h, non_blocking=True)
            step()
            f_h.copy_(f, non_blocking=True)
            g2_h.copy_(g2, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        serial_runs.append(e0.elapsed_time(e1) / n_e2e)
    e2e_serial_ms = sorted(serial_runs)[E2E_REPEATS // 2]

    NB = 3  # device buffer sets
    bufs = [(g, f, g2)] + [(torch.empty_like(g), torch.empty_like(f), torch.empty_like(g2)) for _ in range(NB - 1)]
    s_h2d, s_d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_h2d = [torch.cuda.Event() for _ in range(NB)]
    ev_cmp = [torch.cuda.Event() for _ in range(NB)]
    ev_d2h = [torch.cuda.Event() for _ in range(NB)]

    def h2d(k):
        b = k % NB
        with torch.cuda.stream(s_h2d):
            if k >= NB:
                s_h2d.wait_event(ev_d2h[b])  # set b's previous step is copied out
            bufs[b][0].copy_(g_h, non_blocking=True)
            ev_h2d[b].record(s_h2d)

    def pipelined(n):
        # the input copy of step k + 1 is issued before step k's compute and
        # output copies, so that it never queues behind them (copies of both
        # directions may share a copy engine, which runs them in issue order)
        h2d(0)
        for k in range(n):
            b = k % NB
            gb, fb, g2b = bufs[b]
            if k + 1 < n:
                h2d(k + 1)
            stream.wait_event(ev_h2d[b])
            plan.reconstruct(gb, out=fb)
            plan.adjoint(fb, out=g2b)
            ev_cmp[b].record(stream)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(ev_cmp[b])
                f_h.copy_(fb, non_blocking=True)
                g2_h.copy_(g2b, non_blocking=True)
                ev_d2h[b].record(s_d2h)

    pipelined(4)
    torch.cuda.synchronize(dev)
    pipe_runs = []
    for _ in range(E2E_REPEATS):
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(s_h2d)
        pipelined(n_e2e)
        p1.record(s_d2h)
        torch.cuda.synchronize(dev)
        pipe_runs.append(p0.elapsed_time(p1) / n_e2e)
    e2e_ms = sorted(pipe_runs)[E2E_REPEATS // 2]
    if world > 1:
        t = torch.tensor([e2e_ms, e2e_serial_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms, e2e_serial_ms = float(t[0].item()), float(t[1].item())
    e2e = {"value": world * voxels / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": g_h.numel() * 4,
           "d2h_bytes_per_step": (f_h.numel() + g2_h.numel()) * 4, "ms_per_step": e2e_ms,
           "overlap": "pipelined: H2D of step k+1 and D2H of step k overlap the compute (three buffer sets, "
                      "three streams); serial_* is copy, compute, copy on one stream",
           "serial_ms_per_step": e2e_serial_ms, "serial_value": world * voxels / (e2e_serial_ms / 1e3),
           "repeats": {"steps_each": n_e2e, "ms_per_step": [round(x, 4) for x in pipe_runs],
                       "serial_ms_per_step": [round(x, 4) for x in serial_runs], "reported": "median"}}
    del bufs

    cpu, acc = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, acc = cpu_baseline(P, pa, dev)
        parts["cubic_baseline_forward"]["accuracy_on_a_tile"] = acc

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "step": "forward + adjoint (A g, then A^T of the result)",
                      "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                      "parallelism": f"replicas x{world}", "wall_s": t_wall, "launch_shapes": shapes},
           "roofline": roofline, "pipeline_roofline": pipeline, "stages": stages,
           "stages_timing": "a profiled pass of the same steps before the timed region (events around every launch)",
           "profiled_pass_ms_per_step": profiled_ms,
           "parts": parts,
           "cpu_baseline": cpu,
           "e2e": e2e, "gpu_launches": sum(v[1] for v in prof.values()), "clocks": clocks}
    if rank == 0:
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """The uneven batch alone (see batch_timings)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1501_02946_gb300 as pa
    import synth
    dev = torch.device("cuda", 0)
    res = batch_timings(pa, synth, dev, args.steps, args.warmup)
    out = {"metric": "voxels/s (uneven batch of 64 forward reconstructions)",
           "value": res["batch_graph"]["voxels_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["batch_graph"]["ms"], "higher_is_better": True,
           "dtype": "f32", "data": "synthetic (seeded random)", "config": {"workload": res["workload"]},
           "comparison": res}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="leave the uneven batch out of the parts")
    ap.add_argument("--batch", action="store_true", help="time the uneven 64-instance batch alone")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one step between cudaProfilerStart/Stop (for ncu --profile-from-start off) and exit")
    ap.add_argument("--case", choices=["workload", "columns128", "rows256"], default="workload",
                    help="with --profile-step: the workload; its sample count and depth on a 128x128 grid "
                         "(columns128); or its grid with 256 samples (rows256)")
    args = ap.parse_args()
    if args.case != "workload" and not args.profile_step:
        ap.error("--case selects the profiled step's problem; it needs --profile-step")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
