#!/usr/bin/env python3
"""Throughput of the GB300 NEDNER-NUFFT: one step = one forward
reconstruction and one adjoint (f = A g, then A^T f) of the 128x128 sensor
workload (16384 non-equispaced sensors, 512 samples, 128x128x256 voxels).

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): each rank runs its own
replica of the workload ("replicas only": a single reconstruction does not
shard without a collective), timing is the max over ranks and `value` counts
the voxels of all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the NUFFT algorithm in numpy) on
the host cores instead, on a bounded sample of the same workload.
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
WORKLOAD = ("128x128 non-equispaced sensors over 12.8 mm (8192 jittered lattice + 8192 centre-dense), "
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


def cpu_oracle_step(P, fb_seed=0):
    """One forward + adjoint of the FP64 NUFFT oracle (as it stands)."""
    import numpy as np
    from oracle import nufft
    t0 = time.perf_counter()
    f = nufft.reconstruct(P.xy, P.h, P.g, P.dt, P.c, P.grid)
    nufft.reconstruct_adjoint(P.xy, P.h, f, P.dt, P.c, P.grid, P.n_t)
    return time.perf_counter() - t0


def cropped(P, s):
    """Sub-aperture sample of a workload: the sensors within the central
    (X/s) x (Y/s) square and the matching (nx/s) x (ny/s) x nz output grid."""
    import numpy as np
    import synth
    if s == 1:
        return P
    gr = P.grid
    hx, hy = gr.nx * gr.dx / (2 * s), gr.ny * gr.dy / (2 * s)
    keep = (P.xy[:, 0] >= -hx) & (P.xy[:, 0] < hx) & (P.xy[:, 1] >= -hy) & (P.xy[:, 1] < hy)
    grid = synth.Grid(gr.nx // s, gr.ny // s, gr.nz, gr.dx, gr.dy, gr.dz)
    M = int(keep.sum())
    h = np.full(M, (2 * hx) * (2 * hy) / M)
    return synth.Problem(P.name + f"_crop{s}", P.xy[keep], h, P.g[keep], P.dt, P.c, grid)


def cpu_baseline_subprocess(s=1):
    """Time the oracle single-threaded in a fresh interpreter (BLAS/FFT threads
    pinned to 1 so `cores` is exact)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench, synth; "
            "P = bench.cropped(synth.c2(), %d); t = bench.cpu_oracle_step(P); "
            "print(json.dumps({'t': t, 'voxels': P.grid.nx * P.grid.ny * P.grid.nz, 'M': P.n_sensors}))"
            % (ROOT, s))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("cpu baseline failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # the oracle runs on one host thread (numpy's FFT is single-threaded;
    # pin BLAS pools before numpy loads so that `cores` is exact)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    import synth
    # sample per step: a central sub-aperture crop sized so that the whole
    # (steps + warmup) run stays within about three minutes
    t_full_est = 25.0
    n = args.steps + args.warmup
    s = 1
    while s < 8 and n * t_full_est / (s * s) > 180.0:
        s *= 2
    P = cropped(synth.c2(), s)
    times = []
    for i in range(n):
        t = cpu_oracle_step(P)
        if i >= args.warmup:
            times.append(t)
    voxels = P.grid.nx * P.grid.ny * P.grid.nz
    ms = 1e3 * sum(times) / len(times)
    value = voxels / (ms / 1e3)
    sample = (f"central {P.grid.nx}x{P.grid.ny} of 128x128 sub-aperture ({P.n_sensors} sensors), "
              f"512 samples, depth 256; one FP64 forward+adjoint per step")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample, "oracle": "FP64 NUFFT (numpy), width 16"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


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

    P = synth.c2()
    Nx, Ny, Nz = P.grid.shape
    voxels = Nx * Ny * Nz
    plan = pa.Plan(P.xy, P.n_t, P.dt, P.c, P.grid.as_tuple(), weights=P.h)
    shapes = plan.autotune()  # plan setup, outside the timed region
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
                  "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()}
    pipe = 2 * pipeline_min_bytes(P.n_sensors, P.n_t, Nx, Ny, Nz)
    pipeline = {"min_bytes_per_step": pipe, "achieved_gbs": pipe / (ms_per_step / 1e3) / 1e9,
                "frac": pipe / (ms_per_step / 1e3) / 1e9 / hbm}

    # forward alone, adjoint alone and the cubic-in-omega baseline forward
    # (same plan, same L2 flush, CUDA events around each call)
    def timed_calls(fn, k):
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
    k_parts = max(3, min(args.steps, 10))
    fwd_ms = timed_calls(lambda: plan.reconstruct(g, out=f), k_parts)
    adj_ms = timed_calls(lambda: plan.adjoint(f, out=g2), k_parts)
    cub_ms = timed_calls(lambda: plan.reconstruct_cubic(g, out=f), k_parts)
    plan.reconstruct(g, out=f)
    # library comparison (bench only): cuFFT (through torch.fft) doing the
    # row and column transforms of the same oversampled grid, without the
    # deconvolution, truncation and pair packing that the kernels fuse
    Mx, My = 2 * Nx, 2 * Ny
    g0 = torch.randn(Mx, My, P.n_t, device=dev, dtype=torch.float32)
    def cufft_rows_cols():
        t = torch.fft.rfft(g0, dim=1)[:, : Ny // 2 + 1, :]
        return torch.fft.fft(t, dim=0)
    cufft_ms = timed_calls(cufft_rows_cols, k_parts)
    del g0
    # the same output grid and samples with the sensors on the output lattice
    # (the lattice spatial step: no window spreading)
    import numpy as np
    xy_l = synth.lattice_positions(Nx, Ny, P.grid.dx, P.grid.dy)
    plan_l = pa.Plan(xy_l, P.n_t, P.dt, P.c, P.grid.as_tuple())
    g_l = torch.randn(Nx * Ny, P.n_t, device=dev, dtype=torch.float32)
    def lattice_step():
        plan_l.reconstruct(g_l, out=f)
        plan_l.adjoint(f, out=g_l)
    lat_ms = timed_calls(lattice_step, k_parts) if plan_l.is_lattice else None
    plan_l.close()
    del g_l
    # the d = 2 operator: 256 sensors on a 51.2 mm line (jittered, centre-dense),
    # 1024 samples at 20 ns, image 512 x 512 at 100 um
    rng2 = np.random.default_rng(1507)
    nx2, nz2, nt2, m2 = 512, 512, 1024, 256
    X2 = nx2 * 1e-4
    x2 = np.sort(np.concatenate([rng2.uniform(-X2 / 2, X2 / 2, m2 // 2),
                                 rng2.normal(0.0, X2 / 8, m2 // 2).clip(-X2 / 2, X2 / 2 - 1e-7)]))
    plan_2 = pa.Plan2D(x2, nt2, 20e-9, P.c, (nx2, nz2, 1e-4, 1e-4))
    g_2 = torch.randn(m2, nt2, device=dev, dtype=torch.float32)
    f_2 = torch.empty(nx2, nz2, device=dev, dtype=torch.float32)
    def d2_step():
        plan_2.reconstruct(g_2, out=f_2)
        plan_2.adjoint(f_2, out=g_2)
    d2_ms = timed_calls(d2_step, k_parts)
    plan_2.close()
    del g_2, f_2
    # the position gradient (data gradient A^T fbar included) alone, and the
    # variational workload on the same plan: L = ||A(xy) g - target||^2 +
    # 1e-3 TV_eps(A(xy) g), eps = 1e-8 (isotropic, forward differences),
    # target = the phantom's balls sampled at the voxel centres, backpropagated
    # to g and xy through the autograd function (loss terms in torch, FP64 sums)
    fb_v = torch.randn(P.grid.shape, device=dev, dtype=torch.float32)
    pg_ms = timed_calls(lambda: plan.position_grad(g, fb_v), k_parts)
    target_d = torch.tensor(P.voxelised(), dtype=torch.float32, device=dev)
    xy_v = torch.tensor(P.xy, dtype=torch.float64, requires_grad=True)
    g_v = g.detach().clone().requires_grad_(True)

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
        var_loss(pa.reconstruct(g_v, xy_v, plan)).backward()
    var_ms = timed_calls(var_step, k_parts)
    del fb_v, target_d, g_v
    parts = {"forward": {"ms": fwd_ms, "voxels_per_s": voxels / (fwd_ms / 1e3)},
             "adjoint": {"ms": adj_ms, "voxels_per_s": voxels / (adj_ms / 1e3)},
             "cubic_baseline_forward": {"ms": cub_ms, "voxels_per_s": voxels / (cub_ms / 1e3)},
             "cufft_row_col_transforms_ms": cufft_ms,
             "lattice_sensors_fwd_adj": None if lat_ms is None else
             {"ms": lat_ms, "voxels_per_s": voxels / (lat_ms / 1e3),
              "workload": f"{Nx}x{Ny} sensors on the output lattice, same samples and output"},
             "d2_fwd_adj": {"ms": d2_ms, "pixels_per_s": nx2 * nz2 / (d2_ms / 1e3),
                            "workload": f"d = 2: {m2} sensors on a {X2 * 1e3:.1f} mm line, {nt2} samples at 20 ns, "
                                        f"image {nx2}x{nz2} at 100 um"},
             "position_grad": {"ms": pg_ms, "voxels_per_s": voxels / (pg_ms / 1e3),
                               "what": "pa_position_grad: A^T fbar and dL/dxy of <fbar, A(xy) g>"},
             "variational_fwd_bwd": {"ms": var_ms, "voxels_per_s": voxels / (var_ms / 1e3),
                                     "what": "L = ||A(xy) g - target||^2 + 1e-3 TV_eps(A(xy) g); forward, loss and "
                                             "backward to g and xy through the autograd function"},
             "own_row_col_transforms_ms": (prof["ned_rowfft"][0] / prof["ned_rowfft"][1]
                                           + prof["ned_colfft"][0] / prof["ned_colfft"][1])
             if "ned_rowfft" in prof and "ned_colfft" in prof else None,
             "median_of": k_parts}

    # end to end through the public API with host buffers: every step copies
    # its input g from pinned host memory and its results (f and the adjoint's
    # g') back.  Serial: copy, compute, copy on one stream.  Pipelined (the
    # reported value): two device buffer sets and three streams, so the H2D
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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_e2e):
        g.copy_(g_h, non_blocking=True)
        step()
        f_h.copy_(f, non_blocking=True)
        g2_h.copy_(g2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_serial_ms = e0.elapsed_time(e1) / n_e2e

    bufs = [(g, f, g2), (torch.empty_like(g), torch.empty_like(f), torch.empty_like(g2))]
    s_h2d, s_d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_h2d = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_d2h = [torch.cuda.Event() for _ in range(2)]

    def pipelined(n):
        for k in range(n):
            b = k & 1
            gb, fb, g2b = bufs[b]
            with torch.cuda.stream(s_h2d):
                if k >= 2:
                    s_h2d.wait_event(ev_d2h[b])  # set b's previous step is copied out
                gb.copy_(g_h, non_blocking=True)
                ev_h2d[b].record(s_h2d)
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
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(s_h2d)
    pipelined(n_e2e)
    p1.record(s_d2h)
    torch.cuda.synchronize(dev)
    e2e_ms = p0.elapsed_time(p1) / n_e2e
    if world > 1:
        t = torch.tensor([e2e_ms, e2e_serial_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms, e2e_serial_ms = float(t[0].item()), float(t[1].item())
    e2e = {"value": world * voxels / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": g_h.numel() * 4,
           "d2h_bytes_per_step": (f_h.numel() + g2_h.numel()) * 4, "ms_per_step": e2e_ms,
           "overlap": "H2D of step k+1 and D2H of step k overlap the compute (two buffer sets, three streams)",
           "serial_ms_per_step": e2e_serial_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_baseline_subprocess(1)
        cpu = {"value": r["voxels"] / r["t"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one FP64 forward+adjoint of the full workload (NUFFT oracle, width 16), "
                         "single thread", "seconds": r["t"]}

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
    """The uneven batch (64 instances, N uniform over the 7-smooth integers in
    [64, 256], T in {256, 512, 1024}, output N x N x 2T): pa_batch_run
    (the instances' launches as concurrent branches of a CUDA graph; and the
    mode with one launch per stage over all instances) against 64 sequential
    single-plan reconstructions.  Seeded random data (timing only)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1501_02946_gb300 as pa
    import synth

    dev = torch.device("cuda", 0)
    shapes = synth.batch_shapes()
    rng = np.random.default_rng(1505)
    plans, gs, fs = [], [], []
    voxels = 0
    for k, (n_side, n_t) in enumerate(shapes):
        xy = synth.jittered_lattice(rng, n_side, n_side, 1e-4, 1e-4)
        grid = (n_side, n_side, 2 * n_t, 1e-4, 1e-4, 1e-4)
        plans.append(pa.Plan(xy, n_t, 20e-9, synth.C_WATER, grid))
        gs.append(torch.randn(n_side * n_side, n_t, device=dev, dtype=torch.float32))
        fs.append(torch.empty(n_side, n_side, 2 * n_t, device=dev, dtype=torch.float32))
        voxels += n_side * n_side * 2 * n_t
    batch = pa.Batch(plans)               # concurrent per-instance branches
    batch_st = pa.Batch(plans, mode=1)    # one launch per stage over all instances
    stream = torch.cuda.current_stream(dev)

    def seq():
        for p, g, f in zip(plans, gs, fs):
            p.reconstruct(g, out=f)

    def bat():
        batch.run(gs, fs)

    def bat_st():
        batch_st.run(gs, fs)

    res = {}
    for name, fn in (("batch_graph", bat), ("batch_graph_stage_launches", bat_st), ("sequential_64", seq)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.median(a.elapsed_time(b) for a, b in evs)
        res[name] = {"ms": ms, "voxels_per_s": voxels / (ms / 1e3)}
    out = {"metric": "voxels/s (uneven batch of 64 forward reconstructions)", "value": res["batch_graph"]["voxels_per_s"],
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": res["batch_graph"]["ms"], "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded random)",
           "config": {"workload": "64 instances, N in 7-smooth [64, 256], T in {256, 512, 1024}, output N x N x 2T",
                      "total_voxels": voxels, "shapes": shapes},
           "comparison": res, "speedup_vs_sequential": res["sequential_64"]["ms"] / res["batch_graph"]["ms"]}
    print(json.dumps(out))
    batch.close()
    batch_st.close()
    for p in plans:
        p.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", action="store_true", help="time the uneven 64-instance batch instead")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one step between cudaProfilerStart/Stop (for ncu --profile-from-start off) and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
