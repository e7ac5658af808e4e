"""Benchmark of the GB300 WECT library (one JSON line on rank 0).

Default workload: the WECT of the cubical complex of a 128^3 voxel volume (smoothed Gaussian
random field quantised to u8), d = 256 Fibonacci directions, T = 128 thresholds over
[-sqrt3, sqrt3].  One step = set the vertex weights (device copy + check) and compute the
transform: every row of the hot path (weights, threshold table, fused stencil scatter,
prefix scan).  The metric is simplex.direction evaluations per second: (cells of the complex)
x d per step, summed over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--headline-only]

The same JSON line also carries the metric's other two parts, each timed with CUDA events in a
clock-sampled window of its own: "batched_vs_loop" (4096 blob images, d = 64, T = 64: one
graph-captured persistent launch with the autotuned tile shape against the per-image launch
loop) and "fwd_bwd_ratio" (256
volumes of 64^3, d = 128, T = 128: autograd forward + MSE + backward against the forward), and
"ecf_intensity" (the intensity-filter ECF of uniform 2048^2 .. 8192^2 images and 128^3 .. 512^3
volumes at T = 1000 and 10000).

Multi-GPU (torchrun, one process per GPU): every rank transforms its own volume (the path
partitions into independent complexes, no collective on the data path); timing is the max
over ranks.  --impl reference times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

METRIC = "WECT simplex·direction evals/s on 1 GB300; % HBM peak; fwd+bwd/fwd time"
UNIT = "simplex·direction evals/s"
L2_FLUSH_BYTES = 256 << 20


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            j = json.load(fh)
        return j, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region (and the soak before it) runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "nvidia-smi every 100 ms over >= 1.5 s of identical steps ending with the timed region"}


# ------------------------------------------------------------------ oracle baseline


def oracle_sample(wl, ndirs: int):
    """Time the CPU oracle (single thread, as it stands) on ndirs directions of the workload."""
    import numpy as np

    from oracle import oracle as O

    O.build()
    vw = wl.grid.ravel().astype(np.int64)
    t0 = time.perf_counter()
    O.wect_cubical(wl.dims, vw, wl.dirs[:ndirs], wl.T, wl.lo, wl.hi)
    return time.perf_counter() - t0


# The oracle over all host cores: independent processes (spawn start, safe after CUDA
# initialisation), one direction of the workload each.  The oracle itself is unchanged and
# single-threaded; the directions are independent, so this is its parallel-over-directions run.
_OW = None


def _oracle_worker_init(dims, grid, dirs, T, lo, hi):
    global _OW
    import numpy as np

    from oracle import oracle as O

    O.build()
    _OW = (O, list(dims), np.ascontiguousarray(grid).ravel().astype(np.int64), np.ascontiguousarray(dirs), T, lo, hi)


def _oracle_worker(k):
    O, dims, vw, dirs, T, lo, hi = _OW
    return O.wect_cubical(dims, vw, dirs[k:k + 1], T, lo, hi)[0]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """nproc spawned processes holding the workload; sample() times one direction per process."""

    def __init__(self, wl, nproc: int):
        import multiprocessing as mp

        from oracle import oracle as O

        O.build()       # once, before the workers load it
        self.nproc = nproc
        self.d = len(wl.dirs)
        self.pool = mp.get_context("spawn").Pool(nproc, initializer=_oracle_worker_init,
                                                 initargs=(wl.dims, wl.grid, wl.dirs, wl.T, wl.lo, wl.hi))
        self.pool.map(_oracle_worker_noop, range(nproc), chunksize=1)
        self.next = 0

    def sample(self) -> float:
        ks = [(self.next + i) % self.d for i in range(self.nproc)]
        self.next = (self.next + self.nproc) % self.d
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, ks, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def _oracle_worker_noop(k):
    return k


def cells_of(dims):
    c = 1
    for L in dims:
        c *= 2 * L - 1
    return c


# ------------------------------------------------------------------ traffic from the committed profile


# The committed ncu summary of each stencil kernel on the 128^3 workload, and the sources the
# kernel is compiled from (the counters are stale once any of them changed).
_PROFILES = {
    "cubical_fwd_kernel": ("cubical_fwd_voxel3d_128.md", ("wect_cubical.cu", "wect_cubical_common.cuh",
                                                          "wect_device.cuh")),
    "cubical_run_kernel": ("cubical_run_voxel3d_128.md", ("wect_cubical_run.cu", "wect_cubical_common.cuh",
                                                          "wect_device.cuh")),
}


def _sources_sha(names):
    import hashlib

    csrc = os.path.join(ROOT, "paper_2511_03909_gb300", "csrc")
    hs = hashlib.sha256()
    for name in names:
        hs.update(open(os.path.join(csrc, name), "rb").read())
    return hs.hexdigest()[:16]


def _traffic_per_launch(kernel):
    """DRAM bytes per launch of the kernel from its committed ncu summary, or None when the
    kernel's sources changed since the counters were taken."""
    try:
        prof, names = _PROFILES[kernel]
        h = _sources_sha(names)
        for ln in open(os.path.join(ROOT, "profiles", prof)):
            if ln.startswith("traffic_bytes_per_launch:"):
                _, val, _, sha = ln.split()
                return float(val) if sha == h else None
    except Exception:
        return None
    return None


# ------------------------------------------------------------------ reference arm


def run_reference(args):
    ws, rank, local = _dist_env()
    if rank != 0:
        return 0
    import synthetic as S

    wl = S.voxel3d_128()
    cells = cells_of(wl.dims)
    nproc = host_cores()
    pool = OraclePool(wl, nproc)
    for _ in range(args.warmup):
        pool.sample()
    ts = [pool.sample() for _ in range(args.steps)]
    pool.close()
    sec = sum(ts) / len(ts)
    val = cells * nproc / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": wl.name, "cells": cells, "d": len(wl.dirs), "T": wl.T,
                   "sample": f"{nproc} of {len(wl.dirs)} directions per step"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": nproc, "kind": "oracle",
                         "sample": f"{nproc} directions of the 128^3 workload per step, one per process over "
                                   f"{nproc} host cores (the C oracle is single-threaded)"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2511_03909_gb300 as P
    import synthetic as S

    ws, rank, local = _dist_env()
    dist = ws > 1
    if dist:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P._build.build()
    P.load()

    wl = S.voxel3d_128()
    cells = cells_of(wl.dims)
    d, T = len(wl.dirs), wl.T
    evals_per_step = cells * d
    grid_h = torch.from_numpy(wl.grid).pin_memory()
    dirs_h = torch.from_numpy(wl.dirs).pin_memory()
    grid_d = grid_h.to(dev)
    dirs_d = dirs_h.to(dev)
    out = torch.empty((d, T), dtype=torch.int64, device=dev)
    out_h = torch.empty((d, T), dtype=torch.int64).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    cx = P.CubicalComplex(grid_d)

    def step():
        cx.set_weights(grid_d)
        cx.wect(dirs_d, T, wl.lo, wl.hi, out=out)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    barrier()

    # ---- clock window: nvidia-smi samples every 100 ms cannot resolve a timed region of a few
    # milliseconds, so the sampler runs over a soak of identical steps (>= 1.5 s) that ends
    # with the timed region.
    clocks = ClockSampler(local)
    clocks.start()
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 1.5:
        for _ in range(50):
            flush.zero_()
            step()
        torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = P.launch_count()
    barrier()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                    # L2 flush outside the timed events
        ev[i][0].record()
        step()
        ev[i][1].record()
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = P.launch_count() - l0
    # the stencil kernel's own duration: the same K steps again with the library's event hook
    # around each forward launch on its stream (kept out of the step timing above: events
    # between the step's kernels would take away their programmatic overlap)
    P.profile_enable(True)
    P.profile_read()
    for i in range(args.steps):
        flush.zero_()
        step()
    barrier()
    kern_ms, kern_n = P.profile_read()
    P.profile_enable(False)
    ck = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    value = evals_per_step * ws / (ms / 1e3)

    # ---- end to end through the public API with host buffers: wect_compute_host reads the
    # page-locked weights and directions and writes the page-locked table itself, so every
    # host<->device byte of the step moves inside the timed region
    def step_host():
        cx.wect_host(grid_h, dirs_h, T, wl.lo, wl.hi, out=out_h, sync=False)

    for _ in range(3):
        flush.zero_()
        step_host()
    barrier()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        e2e_ev[i][0].record()
        step_host()
        e2e_ev[i][1].record()
    barrier()
    assert torch.equal(out_h, out.cpu()), "host entry and device entry disagree"

    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / args.steps
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = evals_per_step * ws / (e2e_ms / 1e3)

    # ---- correctness of the timed output on sampled directions (device result vs oracle)
    # is covered by the GPU tests; here only the invariant last column is checked.
    o = out.cpu().numpy()
    assert np.all(o[:, -1] == o[0, -1]), "last column must be the weighted Euler characteristic"

    if rank != 0:
        if dist:
            tdist.destroy_process_group()
        return 0

    peaks, src = _peaks()
    # roofline of the dominant kernel (the stencil kernel of the transform).  Unit of work: one
    # vertex.direction update of the method (the height fma, the rounding to a bin, the integer
    # add into the histogram: 3 lane operations); peak lane-op rate = 152 SMs x 128 lanes x the SM
    # clock.  The run-based kernel reaches the same sums with fewer operations on long rows (one
    # update per bin boundary), so against this roof it is a throughput ratio.  Floors of the
    # unit of work: HBM (inputs read once, table written once), the lane-op roof, and the shared
    # atomic pipe (one 32-bit red.shared per update at ~25 per clock per SM, measured with a
    # probe kernel on this GPU).
    kernel = P.last_stencil_kernel()
    nv = int(np.prod(wl.dims))
    kernel_ms = kern_ms / max(kern_n, 1)
    units = nv * d
    ops = 3.0 * units
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_ops = 152 * 128 * sm_mhz * 1e6
    achieved = ops / (kernel_ms / 1e3)
    hbm_bytes = nv * 1 + d * T * 8 + d * 3 * 8
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    floors = {"hbm_us": hbm_bytes / (hbm_peak * 1e9) * 1e6, "alu_us": ops / peak_ops * 1e6,
              "smem_atomic_us": units / (25.0 * 152 * sm_mhz * 1e6) * 1e6}
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
            "frac": achieved / peak_ops, "traffic": _traffic_per_launch(kernel),
            "kernel": kernel, "kernel_ms": kernel_ms, "units_per_launch": units,
            "unit_of_work": "vertex.direction update, 3 lane ops",
            "kernel_timing": "CUDA events around each forward launch on its stream, over a second pass of the K "
                             "timed steps (launched in plain stream order while timed)",
            "peak_source": f"152 SMs x 128 lanes x {sm_mhz:.0f} MHz ({src} sm_max_mhz)",
            "floors_us": floors, "floor_us": max(floors.values()),
            "frac_of_floor": max(floors.values()) / (kernel_ms * 1e3),
            "hbm_gbs": hbm_bytes / (kernel_ms / 1e3) / 1e9,
            "hbm_frac": hbm_bytes / (kernel_ms / 1e3) / 1e9 / hbm_peak}

    # CPU baseline: the oracle on a bounded sample (a few directions) of the same workload
    cpu = None
    if not args.no_cpu_baseline:
        ndirs = 3
        sec = oracle_sample(wl, ndirs)
        nproc = host_cores()
        pool = OraclePool(wl, nproc)
        pool.sample()                   # the first round also finishes the workers' start-up
        secp = pool.sample()
        pool.close()
        cpu = {"value": cells * nproc / secp, "unit": UNIT, "cores": nproc, "kind": "oracle",
               "sample": f"{nproc} of {d} directions of the 128^3 workload, one per process over {nproc} host "
                         f"cores ({secp:.1f} s; the C oracle is single-threaded)",
               "single_core": {"value": cells * ndirs / sec,
                               "sample": f"{ndirs} of {d} directions in one process ({sec:.1f} s)"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": wl.name, "cells": cells, "vertices": nv, "d": d, "T": T,
                   "range": [wl.lo, wl.hi], "weights": "u8 smoothed Gaussian field (seed 2)",
                   "l2": "flushed between steps (256 MiB device write outside the timed events)",
                   "parallelism": f"replicas x{ws} (one volume per GPU)"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(grid_h.numel() + dirs_h.numel() * 8),
                "d2h_bytes_per_step": int(out.numel() * 8), "ms_per_step": e2e_ms,
                "call": "wect_compute_host with page-locked weights, directions and table (read and written "
                        "by the library's kernels through their device mapping)"},
        "gpu_launches": int(launches),
        "clocks": ck,
        "wall_s": t_wall,
    }
    if not args.headline_only:
        line.update(secondary(P, S, dev, args.steps, flush, local))
    print(json.dumps(line), flush=True)
    if dist:
        tdist.destroy_process_group()
    return 0


def _section(fn, steps, flush, local, soak_s=1.5, warmup=3):
    """Time fn with CUDA events on the current stream after warm-up, flushing L2 before every
    timed call outside the events, with nvidia-smi clocks sampled over a soak of identical calls
    that ends with the timed calls.  Returns (mean ms, clocks)."""
    import torch

    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    ck = ClockSampler(local)
    ck.start()
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < soak_s:
        flush.zero_()
        fn()
        torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    clocks = ck.stop()
    return sum(a.elapsed_time(b) for a, b in ev) / steps, clocks


def secondary(P, S, dev, steps, flush, local):
    """The metric's other two parts and the ECF throughput rows, each with its own clock window:
    the 4096-image batch as one graph-captured persistent launch against the per-image launch
    loop, forward + backward against forward on the differentiation workload (autograd + MSE),
    and the intensity-filter ECF of uniform images and volumes at T = 1000 and 10000."""
    import torch

    res = {}
    # batched images: 4096 2D blob images, d=64, T=64
    wl = S.image_batch()
    dirs = torch.from_numpy(wl.dirs).to(dev)
    b = P.CubicalBatch([torch.from_numpy(x).to(dev) for x in wl.grids])
    out = torch.empty((len(wl.grids), len(wl.dirs), wl.T), dtype=torch.int64, device=dev)
    b.autotune(dirs, wl.T, wl.lo, wl.hi)            # the tile shape of the batched launch
    shape = b.tuned_shape(len(wl.dirs), wl.T)
    t_batch, ck_b = _section(lambda: b.wect(dirs, wl.T, wl.lo, wl.hi, out=out), steps, flush, local)
    t_loop, ck_l = _section(lambda: b.wect(dirs, wl.T, wl.lo, wl.hi, out=out, loop=True), min(steps, 5), flush, local,
                            warmup=1)
    cells = sum((2 * x.shape[0] - 1) * (2 * x.shape[1] - 1) for x in wl.grids)
    res["batched_vs_loop"] = {"workload": wl.name, "batched_ms": t_batch, "loop_ms": t_loop,
                              "ratio": t_loop / t_batch, "batched_evals_per_s": cells * len(wl.dirs) / (t_batch / 1e3),
                              "tuned_shape": {"directions_per_lane": shape[0], "tile": shape[1], "run_kernel": shape[2],
                                              "cta_threads": shape[3]} if shape else None,
                              "clocks_batched": ck_b, "clocks_loop": ck_l}
    del b, out
    # differentiation: 256 volumes 64^3 f32, d=128, T=128, MSE against a target batch
    wv = S.volume_batch_diff()
    dirs = torch.from_numpy(wv.dirs).to(dev)
    flat = torch.from_numpy(wv.grids.reshape(-1)).to(dev)
    bt = P.CubicalBatch(flat=torch.from_numpy(wv.target.reshape(-1)).to(dev), dims=[wv.dims] * len(wv.grids),
                        frac_bits=24)
    Bt = bt.wect(dirs, wv.T, wv.lo, wv.hi).to(torch.float64) * 2.0 ** -24
    del bt
    bb = P.CubicalBatch(flat=flat, dims=[wv.dims] * len(wv.grids), frac_bits=24)
    w = flat.clone().requires_grad_(True)

    def fwd():
        with torch.no_grad():
            W = P.WECTFunction.apply(bb, w, dirs, wv.T, wv.lo, wv.hi)
            return ((W - Bt) ** 2).mean()

    def fwd_bwd():
        w.grad = None
        W = P.WECTFunction.apply(bb, w, dirs, wv.T, wv.lo, wv.hi)
        loss = ((W - Bt) ** 2).mean()
        loss.backward()

    tf, ck_f = _section(fwd, steps, flush, local)
    tfb, ck_fb = _section(fwd_bwd, steps, flush, local)
    cells = len(wv.grids) * cells_of(wv.dims)
    res["fwd_bwd_ratio"] = {"workload": wv.name, "fwd_ms": tf, "fwd_bwd_ms": tfb, "ratio": tfb / tf,
                            "fwd_evals_per_s": cells * len(wv.dirs) / (tf / 1e3),
                            "step": "WECTFunction forward + MSE (+ loss.backward() through the library adjoint)",
                            "clocks_fwd": ck_f, "clocks_fwd_bwd": ck_fb}
    del bb, w, flat, Bt
    # intensity-filter ECF of uniform images and volumes (the paper's ECF throughput workloads):
    # vertices per second, T = 1000 and 10000, filter resident on the device
    g = torch.Generator(device=dev).manual_seed(7)
    ecf = {}
    for dims in ([2048] * 2, [4096] * 2, [8192] * 2, [128] * 3, [256] * 3, [512] * 3):
        nv = 1
        for L in dims:
            nv *= L
        f = torch.rand(nv, generator=g, device=dev, dtype=torch.float64)
        cx = P.CubicalComplex(None, dims=dims)
        o = torch.empty(10000, dtype=torch.int64, device=dev)
        for T in (1000, 10000):
            ms, ck = _section(lambda: cx.ecf(f, T, 0.0, 1.0, out=o[:T]), steps, flush, local, soak_s=0.5)
            ecf[f"{'x'.join(map(str, dims))}_T{T}"] = {"ms": ms, "gvertices_per_s": nv / ms / 1e6,
                                                        "sm_mhz": ck.get("sm_mhz"), "reasons": ck.get("reasons")}
        del cx, f
    res["ecf_intensity"] = ecf
    return res


def run_case(name):
    """Run one small workload a few times, untimed, for ncu captures of kernels the headline
    step does not launch (the adjoint, the run-based stencil, the simplicial gather, the batch,
    the ECF)."""
    import torch

    sys.path.insert(0, ROOT)
    import paper_2511_03909_gb300 as P
    import synthetic as S

    dev = torch.device("cuda:0")
    if name == "adjoint16":
        # 16 volumes 64^3 f32 (2^-24 fixed point), d = 128 Fibonacci, T = 128: three adjoint calls
        wv = S.volume_batch_diff(count=16)
        dirs = torch.from_numpy(wv.dirs).to(dev)
        bt = P.CubicalBatch(flat=torch.from_numpy(wv.target.reshape(-1)).to(dev), dims=[wv.dims] * 16, frac_bits=24)
        bb = P.CubicalBatch(flat=torch.from_numpy(wv.grids.reshape(-1)).to(dev), dims=[wv.dims] * 16, frac_bits=24)
        D = (bb.wect(dirs, wv.T, wv.lo, wv.hi) - bt.wect(dirs, wv.T, wv.lo, wv.hi)).contiguous()
        for _ in range(3):
            g = bb.backward(dirs, wv.T, wv.lo, wv.hi, D, 2.0 ** -23 / D.numel())
        torch.cuda.synchronize()
        print("adjoint16 ok", float(g.abs().sum()))
    elif name == "run128":
        # the 128^3 u8 volume, d = 256 Fibonacci, T = 128, through the run-based stencil kernel
        # (forced with the kernel-selection hook): three calls
        wl = S.voxel3d_128()
        cx = P.CubicalComplex(torch.from_numpy(wl.grid).to(dev))
        dirs = torch.from_numpy(wl.dirs).to(dev)
        P.stencil_variant(2)
        try:
            for _ in range(3):
                W = cx.wect(dirs, wl.T, wl.lo, wl.hi)
            torch.cuda.synchronize()
            kernel = P.last_stencil_kernel()
        finally:
            P.stencil_variant(0)
        print("run128 ok", kernel, int(W[:, -1].sum()))
    elif name == "mesh64":
        # the 1024^2 mesh with d = 64 directions (two 32-direction tiles), T = 512, range [-1.5, 1.5]
        wl = S.mesh2d_1024(d=64)
        cx = wl.complex
        h = P.SimplicialComplex(torch.from_numpy(cx.coords).to(dev), [torch.from_numpy(x).to(dev) for x in cx.simplices],
                                torch.from_numpy(cx.weights).to(dev), frac_bits=24)
        dirs = torch.from_numpy(wl.dirs).to(dev)
        for _ in range(2):
            W = h.wect(dirs, wl.T, -1.5, 1.5)
        torch.cuda.synchronize()
        print("mesh64 ok", int(W[:, -1].abs().sum()))
    elif name == "batch4096":
        # the 4096-image batch (d = 64, T = 64, [-sqrt2, sqrt2]): two graph replays, then one
        # per-image launch loop
        wl = S.image_batch()
        dirs = torch.from_numpy(wl.dirs).to(dev)
        b = P.CubicalBatch([torch.from_numpy(x).to(dev) for x in wl.grids])
        out = torch.empty((len(wl.grids), 64, 64), dtype=torch.int64, device=dev)
        for _ in range(2):
            b.wect(dirs, wl.T, wl.lo, wl.hi, out=out)
        b.wect(dirs, wl.T, wl.lo, wl.hi, out=out, loop=True)
        torch.cuda.synchronize()
        print("batch4096 ok", int(out[:, :, -1].sum()))
    elif name == "ecf4096":
        # intensity-filter ECF of a uniform 4096^2 image, T = 1000, [0, 1]: three calls
        g = torch.Generator(device=dev).manual_seed(7)
        f = torch.rand(4096 * 4096, generator=g, device=dev, dtype=torch.float64)
        cx = P.CubicalComplex(None, dims=[4096, 4096])
        for _ in range(3):
            o = cx.ecf(f, 1000, 0.0, 1.0)
        torch.cuda.synchronize()
        print("ecf4096 ok", int(o[-1]))
    elif name == "wecf64":
        # 64 uniform vertex filters on the 128^3 cubical complex of the voxel workload, T = 128,
        # [-1, 1], weighted: three calls
        wl = S.voxel3d_128()
        cx = P.CubicalComplex(torch.from_numpy(wl.grid).to(dev))
        g = torch.Generator(device=dev).manual_seed(3)
        F = torch.rand((64, cx.nv), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        for _ in range(3):
            o = cx.wecf(F, 128, -1.0, 1.0)
        torch.cuda.synchronize()
        print("wecf64 ok", int(o[:, -1].sum()))
    else:
        raise SystemExit(f"unknown case {name}")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the batched-vs-loop, forward+backward and ECF sections")
    ap.add_argument("--case", choices=["adjoint16", "run128", "mesh64", "batch4096", "ecf4096", "wecf64"],
                    help="run one untimed workload for an ncu capture (no JSON line)")
    args = ap.parse_args()
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
