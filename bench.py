#!/usr/bin/env python
"""Throughput of plane-wise multi-view Richardson-Lucy on GB300.

One step = the whole hot path over one synthetic volume: reslice every view
stack into planes on the GPU, start every plane from its mean, run 10 MV-RL
iterations over all planes.  Default workload (one per GPU, weak scaling):
4 views of 1024^3 uint16 Gaussian-blob stacks (density 5e-5 per voxel,
Poisson noise) at 0/90/180/270 degrees, 41x41 Gaussian PSFs sigma (1.8, 10)
px, views updating the estimate in sequence, zero boundary, eps 1e-6.

Prints one JSON line (rank 0).  `value` counts voxel-view-iterations per
second over all GPUs (planes x pixels x iterations x views / time); inputs
are device-resident and larger than L2 (16 GiB of stacks and planes per
step).  `e2e` is the same metric through mvd_run_host with pinned host
buffers, copies included.  `--impl reference` times the FP64 CPU oracle on
a sample of the same workload instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/s per view for MV-RL vs plain per-plane path; % HBM roofline"
UNIT = "voxel-view-iterations/s"

_VOL1024 = dict(Z=1024, Y=1024, X=1024, K=41, sigma_axial=10.0, sigma_lateral=1.8, angles=(0.0, 90.0, 180.0, 270.0),
                density=5e-5, iters=10, seed=0, order="sequential")
_VOL512 = dict(Z=512, Y=512, X=512, K=31, sigma_axial=8.0, sigma_lateral=1.5, angles=(0.0, 90.0), density=1e-4,
               iters=10, seed=0, order="simultaneous")
WORKLOADS = {
    "volume1024x4": dict(_VOL1024,
                         label="4 views, 1024^3 uint16 stacks resliced on the GPU to 1024 planes of 1024x1024, "
                               "41x41 PSFs sigma (1.8, 10) px at 0/90/180/270 degrees, views in sequence, "
                               "10 iterations"),
    "slab1024x4": dict(_VOL1024, Y=64,
                       label="4 views, 1024x64x1024 uint16 slab: 64 planes of 1024x1024 of the 4-view 1024^3 "
                             "workload (profiling case)"),
    "volume512": dict(_VOL512,
                      label="2 views, 512^3 uint16 stacks resliced on the GPU to 512 planes of 512x512, "
                            "31x31 PSFs sigma (1.5, 8) px turned by 90 degrees, 10 iterations"),
    "slab512": dict(_VOL512, Y=128,
                    label="2 views, 512x128x512 uint16 slab: 128 planes of 512x512 (profiling case, "
                          "one quarter of the 512^3 volume)"),
    "volume128": dict(_VOL512, Z=128, Y=128, X=128, label="2 views, 128^3 uint16 (quick check)"),
}
DEFAULT_WORKLOAD = "volume1024x4"

# HBM copy bandwidth measured on GB300 (STREAM-style copy); MEASURED_PEAKS.json,
# when present, overrides it.
HBM_PEAK_GBS = 6767.4
# FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 flop x the maximum SM clock
# (2070 MHz on GB300 unless MEASURED_PEAKS.json gives another).
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# of the current kernels on the workload's profiling slab, scaled to a full
# launch by the planes processed (traffic is proportional to the planes);
# None where no capture of the current kernels exists.  The captures are
# summarised under profiles/ (fused_kernels_volume1024x4.md); the 512^3
# workload has no capture of the current kernels.
NCU_TRAFFIC_PER_LAUNCH = {
    "volume1024x4": {"blur_ratio": 1.0073e10, "correlate_update": 1.2251e10},
    "volume512": {"blur_ratio": None, "correlate_update": None},
}
# The fused kernels' source files and the first 16 hex digits of the SHA-256
# of their concatenation when those counters were taken: once any of them
# changes, the line reports traffic null until a new capture is recorded.
FUSED_KERNEL_SOURCES = ("fused.cu", "fused_common.cuh", "tma.cuh", "mvd_internal.h")
NCU_TRAFFIC_SOURCE_SHA16 = "e61f00f827214c9e"


def fused_sources_sha16():
    import hashlib
    h = hashlib.sha256()
    for f in FUSED_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1503_07998_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel):
    """Captured DRAM bytes per launch of `kernel`, or None when there is no
    capture of the kernels as they are now."""
    t = NCU_TRAFFIC_PER_LAUNCH.get(workload, {}).get(kernel)
    if t is None or fused_sources_sha16() != NCU_TRAFFIC_SOURCE_SHA16:
        return None
    return t


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _peaks():
    m = _measured_peaks()
    if "hbm_gbs" in m:
        return float(m["hbm_gbs"]), "measured"
    return HBM_PEAK_GBS, "fallback"


def alu_peak_tflops(sms: int):
    """FP32 FMA peak from the device's SM count and the maximum SM clock."""
    mhz = float(_measured_peaks().get("sm_max_mhz", SM_MAX_MHZ))
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, \
        f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz:.0f} MHz"


def kernel_budget(order: str, V: int, es: int, K: int):
    """Algorithmic bytes and FLOP per pixel of one launch of the fused kernels.

    A launch covers every pixel of every plane once, for the views it takes
    part in: all V (simultaneous product) or one (views in sequence).  Per
    pixel and view in that launch, kernel A reads the estimate once for all
    its views (4 B), reads the data (es B) and writes the ratio (4 B); kernel
    B reads the ratio (4 B) and reads and writes the estimate once (8 B).
    FLOP: a rank-1 separable K x K PSF is two 1D passes of K taps, 2 FLOP per
    tap, per view, in each kernel (8 V K per voxel-iteration in all)."""
    vl = 1 if order == "sequential" else V
    return {"blur_ratio": (4 + (es + 4) * vl, 4 * K * vl),
            "correlate_update": (4 * vl + 8, 4 * K * vl)}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        """Start sampling every 50 ms and wait (at most 3 s) for the first row,
        so that a short timed region that follows still gets samples."""
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.index)], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + 3.0
        while time.time() < t_end and self._rows() < 1 and self.proc.poll() is None:
            time.sleep(0.01)

    def _rows(self) -> int:
        try:
            with open(self.file.name) as f:
                return sum(1 for r in f if r.strip())
        except OSError:
            return 0

    def mark(self) -> int:
        """Rows written so far; stop(skip=mark()) keeps only later samples."""
        return self._rows() if self.proc is not None else 0

    def stop(self, skip: int = 0, upto=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        with open(self.file.name) as f:
            rows = [r.strip().split(", ") for r in f if r.strip()][skip:upto]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- oracle (CPU)
def _oracle_plane(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import oracle
    phi, psfs, iters, order = args
    t0 = time.perf_counter()
    psi = oracle.rl_planes(phi[:, None].astype(np.float64), psfs, iters, boundary="zero", eps=1e-6, route="fft",
                           order=order)
    return time.perf_counter() - t0, psi[0]


def _warm_worker(_):
    """Start-up work of a pool worker (imports), kept out of the timed sample."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy  # noqa: F401
    import oracle  # noqa: F401
    return os.getpid()


def oracle_sample(pool, planes_np, psfs, iters, order):
    """Oracle over the sampled planes [V][S][H][W], one plane per worker.
    Returns (wall seconds, results [S][H][W] FP64)."""
    import numpy as np
    t0 = time.perf_counter()
    out = pool.map(_oracle_plane, [(planes_np[:, s], psfs, iters, order) for s in range(planes_np.shape[1])])
    return time.perf_counter() - t0, np.stack([o[1] for o in out])


def n_workers():
    """Every host core this process may run on."""
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    return max(1, n)


def sample_planes(stacks, idx):
    """Planes y in idx of every view, [V][S][Z][X] numpy, cut from the
    synthetic stacks [V][Z][Y][X] by torch slicing (plane y of view v is
    stacks[v, :, y, :]); the library's reslice kernel is not involved."""
    import numpy as np
    import torch
    return np.stack([stacks[:, :, int(y), :].to(torch.int32).cpu().numpy() for y in idx], axis=1)


def error_vs_oracle(got, ref):
    """rel-L2 and per-pixel errors of a route's sampled planes against the
    FP64 oracle: ||g-o||/||o||; max |g-o| / max(|o|, tau), tau = 1e-3 max|o|;
    and the unfloored per-pixel maximum."""
    import numpy as np
    g = np.asarray(got, dtype=np.float64)
    o = np.asarray(ref, dtype=np.float64)
    tau = 1e-3 * float(np.abs(o).max())
    d = np.abs(g - o)
    return {"rel_l2": float(np.linalg.norm(g - o) / np.linalg.norm(o)),
            "per_pixel": float((d / np.maximum(np.abs(o), tau)).max()),
            "per_pixel_unfloored": float((d / np.maximum(np.abs(o), 1e-300)).max()),
            "planes": int(g.shape[0]), "finite": bool(np.all(np.isfinite(g)))}


# ----------------------------------------------------------------- helpers
def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world):
    if world == 1:
        return x
    from paper_1503_07998_gb300 import shard
    return shard.max_over_ranks(x)


def make_inputs(wl, seed, device):
    from paper_1503_07998_gb300 import synth
    return synth.volume_stacks(wl["Z"], wl["Y"], wl["X"], wl["K"], wl["sigma_axial"], wl["sigma_lateral"],
                               wl["angles"], wl["density"], seed=seed, device=device)


def workload_config(wl, world):
    """The `config` object of both arms (the same keys and values)."""
    V = len(wl["angles"])
    stack_mib = V * wl["Z"] * wl["Y"] * wl["X"] * 2 / 2**20
    return {"workload": wl["label"], "views": V, "volume": [wl["Z"], wl["Y"], wl["X"]], "psf": wl["K"],
            "sigma_px": [wl["sigma_lateral"], wl["sigma_axial"]], "angles_deg": list(wl["angles"]),
            "iters": wl["iters"], "order": wl["order"], "boundary": "zero", "planes_per_gpu": wl["Y"],
            "data_dtype": "u16",
            "l2": (f"inputs larger than L2: {stack_mib:.0f} MiB of stacks + {stack_mib:.0f} MiB of planes per step"
                   if 2 * stack_mib > 129 else f"inputs smaller than L2 ({2 * stack_mib:.0f} MiB): a quick check, "
                                               "not a bench line"),
            "parallelism": f"{world} GPU(s), one independent volume per GPU, no collective"}


def kernel_roofline(prof, name, units_per_launch, bytes_per_unit, flops_per_unit, hbm_peak, alu_peak):
    total_ms, n = prof.get(name, (0.0, 0))
    if not n:
        return None
    t = total_ms / n / 1e3
    gbs = units_per_launch * bytes_per_unit / t / 1e9
    tfl = units_per_launch * flops_per_unit / t / 1e12
    return {"avg_ms": total_ms / n, "launches": n, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
            "tflops": tfl, "alu_frac": tfl / alu_peak,
            "bytes_per_unit": bytes_per_unit, "flops_per_unit": flops_per_unit,
            "units_per_launch": units_per_launch}


def timed_call(stream, fn, prof_ctx=None):
    """Device time of fn() with CUDA events on the launching stream."""
    import torch
    from paper_1503_07998_gb300 import mvd
    if prof_ctx is not None:
        mvd.mvd_profile_enable(prof_ctx, True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    prof = None
    if prof_ctx is not None:
        prof = mvd.mvd_profile_read(prof_ctx)
        mvd.mvd_profile_enable(prof_ctx, False)
    return a.elapsed_time(b), prof


# ----------------------------------------------------------------- arms
def run_reference(args, wl):
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return 0
    import numpy as np
    import torch
    S = n_workers()
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(S)
    pool.map(_warm_worker, range(S))
    dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    stacks, psfs = make_inputs(wl, wl["seed"], dev)
    V = stacks.shape[0]
    idx = np.linspace(0, wl["Y"] - 1, S).round().astype(int)
    planes = sample_planes(stacks, idx)
    del stacks
    for _ in range(args.warmup):
        oracle_sample(pool, planes, psfs, wl["iters"], wl["order"])
    times = [oracle_sample(pool, planes, psfs, wl["iters"], wl["order"])[0] for _ in range(args.steps)]
    pool.close()
    t = sum(times) / len(times)
    units = S * wl["Z"] * wl["X"] * wl["iters"] * V
    value = units / t
    sample = (f"{S} of the {wl['Y']} planes (one per process, all {S} host cores), FP64 Fourier route, "
              f"{wl['iters']} iterations, views {wl['order']}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": S, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_mvd(args, wl):
    import numpy as np
    import torch
    S = n_workers()
    world, rank, local = dist_setup(args.gpus)
    from paper_1503_07998_gb300 import mvd
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak, alu_src = alu_peak_tflops(sms)
    hbm_peak, hbm_src = _peaks()
    stacks, psfs = make_inputs(wl, wl["seed"] + rank, dev)
    V, Z, Y, X = stacks.shape
    K, iters, order = wl["K"], wl["iters"], wl["order"]
    ctx = mvd.mvd_create(V, psfs, K, Z, X, iters, "zero", 1e-6)
    mvd.mvd_set_update_order(ctx, order)
    planes = torch.empty((V, Y, Z, X), dtype=stacks.dtype, device=dev)
    est = torch.empty((Y, Z, X), dtype=torch.float32, device=dev)
    # planes whose results are compared with the FP64 oracle (cut from the
    # synthetic stacks, not from the library's reslice)
    idx = np.linspace(0, Y - 1, S).round().astype(int) if rank == 0 else np.zeros(0, dtype=int)
    sampled = {}

    def keep(name):
        if rank == 0 and not args.no_cpu:
            sampled[name] = np.stack([est[int(y)].cpu().numpy() for y in idx])

    def step(marks=None):
        if marks:
            marks[0].record(stream)
        mvd.mvd_reslice(ctx, stacks, planes)
        if marks:
            marks[1].record(stream)
        mvd.mvd_deconvolve_planes(ctx, planes, est, init_mean=True)
        if marks:
            marks[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    mvd.mvd_profile_enable(ctx, True)
    n0 = mvd.mvd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # per-step marks (reslice, deconvolution) for the medians; recording an
    # event costs nothing measurable next to a step
    step_marks = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier(world)
    first_row = clocks.mark()
    ev0.record(stream)
    for i in range(args.steps):
        step(step_marks[i])
    ev1.record(stream)
    torch.cuda.synchronize()
    last_row = max(clocks.mark(), first_row + 1)   # at least the first sample after the start
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    timing = {"steps_timed": args.steps,
              "step_ms_median": statistics.median(m[0].elapsed_time(m[2]) for m in step_marks),
              "reslice_ms_median": statistics.median(m[0].elapsed_time(m[1]) for m in step_marks),
              "deconvolve_ms_median": statistics.median(m[1].elapsed_time(m[2]) for m in step_marks)}
    launches = mvd.mvd_launch_count() - n0
    prof = mvd.mvd_profile_read(ctx)
    mvd.mvd_profile_enable(ctx, False)
    clk = clocks.stop(first_row, last_row)
    ms_max = reduce_max(ms, world)
    units_per_step = Y * Z * X * iters * V
    value = units_per_step * world * args.steps / (ms_max / 1e3)
    keep("fused")

    # roofline of the dominant kernel, on the algorithmic counts
    es = 2 if stacks.dtype == torch.uint16 else 4
    px = Y * Z * X                                   # pixels of one launch
    budget = kernel_budget(order, V, es, K)
    kr = {n: kernel_roofline(prof, n, px, b, f, hbm_peak, alu_peak) for n, (b, f) in budget.items()}
    kr["reslice"] = kernel_roofline(prof, "reslice", px * V, 2 * es, 0, hbm_peak, alu_peak)
    kr["plane_means"] = kernel_roofline(prof, "plane_means", px * V, es, 0, hbm_peak, alu_peak)
    dom = max((k for k in kr if kr[k]), key=lambda k: kr[k]["avg_ms"] * kr[k]["launches"])
    d = kr[dom]
    if d["alu_frac"] >= d["hbm_frac"]:
        roof = {"bound": "alu", "achieved": d["tflops"], "peak": alu_peak, "unit": "TFLOP/s",
                "frac": d["alu_frac"], "peak_source": alu_src}
    else:
        roof = {"bound": "hbm", "achieved": d["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": d["hbm_frac"], "peak_source": hbm_src}
    roof.update({"kernel": dom, "traffic": ncu_traffic(args.workload, dom),
                 "algorithmic_bytes_per_launch": px * d["bytes_per_unit"],
                 "algorithmic_flops_per_launch": px * d["flops_per_unit"],
                 "hbm_gbs": d["hbm_gbs"], "hbm_frac": d["hbm_frac"], "hbm_peak": hbm_peak,
                 "tflops": d["tflops"], "alu_frac": d["alu_frac"], "alu_peak": alu_peak,
                 "avg_launch_ms": d["avg_ms"], "launches": d["launches"],
                 "share_of_timed_region": d["avg_ms"] * d["launches"] / ms})

    def leg(name):   # the comparison legs this run includes
        return not args.no_plain and (args.legs == "all" or name in args.legs.split(","))

    # plain per-plane path on a slice of the planes (same context and factors)
    plain = None
    if leg("plain"):
        sub = min(Y, 32)
        mvd.mvd_set_algo(ctx, "plain")
        e2 = est[:sub].contiguous()
        p2 = planes[:, :sub].contiguous()
        mvd.mvd_deconvolve_planes(ctx, p2, e2)
        torch.cuda.synchronize()
        pms, _ = timed_call(stream, lambda: mvd.mvd_deconvolve_planes(ctx, p2, e2))
        mvd.mvd_set_algo(ctx, "fused")
        fused_ms = sum(v[0] for k, v in prof.items() if k in ("blur_ratio", "correlate_update", "plane_means"))
        fused_ms_per_plane = fused_ms / args.steps / Y
        plain_val = sub * Z * X * iters * V / (pms / 1e3)
        plain = {"value": plain_val, "unit": UNIT, "planes": sub,
                 "speedup_of_fused": (pms / sub) / fused_ms_per_plane}
        del e2, p2

    # the Fourier route on the same planes (same context, one call = 10 iterations)
    fft_route = None
    if leg("fft"):
        try:
            mvd.mvd_set_algo(ctx, "fft")
            mvd.mvd_deconvolve_planes(ctx, planes, est)
            torch.cuda.synchronize()
            fms, fprof = timed_call(stream, lambda: mvd.mvd_deconvolve_planes(ctx, planes, est), ctx)
            keep("fft")
            fft_route = {"value": units_per_step / (fms / 1e3), "unit": UNIT, "ms": fms,
                         "note": "deconvolution only (no reslice), hand-written mixed-radix FFT route",
                         "kernels": {k: {"total_ms": v[0], "launches": v[1]} for k, v in fprof.items()}}
        except mvd.MvdError as e:
            fft_route = {"unavailable": str(e)}
        finally:
            mvd.mvd_set_algo(ctx, "fused")

    # the plane-resident route on the same planes (planes up to 512 x 512)
    resident = None
    if leg("resident"):
        try:
            mvd.mvd_set_algo(ctx, "resident")
            mvd.mvd_deconvolve_planes(ctx, planes, est)
            torch.cuda.synchronize()
            rms, _ = timed_call(stream, lambda: mvd.mvd_deconvolve_planes(ctx, planes, est), ctx)
            keep("resident")
            resident = {"value": units_per_step / (rms / 1e3), "unit": UNIT, "ms": rms,
                        "note": "deconvolution only (no reslice); one thread-block cluster per plane keeps the "
                                "estimate, ratio and product in shared memory for all iterations, phi read once "
                                "per iteration and view",
                        "hbm_bytes_per_vi_algorithmic": (es * iters * V + 4 + 4) / (iters * V)}
        except mvd.MvdError as e:
            resident = {"unavailable": str(e)}
        finally:
            mvd.mvd_set_algo(ctx, "fused")

    # the optional tensor-core routes (BF16x3 and TF32 tcgen05 passes) on the
    # same planes
    tc_routes = {}
    for algo, prefix, precision in (
            ("tensor", "tc", "BF16x3 tcgen05 passes, FP32 accumulate; ratio and update FP32"),
            ("tf32", "tf32", "TF32 tcgen05 passes (operands rounded to TF32), FP32 accumulate; ratio and update FP32")):
        if not leg(algo):
            continue
        try:
            mvd.mvd_set_algo(ctx, algo)
            mvd.mvd_deconvolve_planes(ctx, planes, est)
            torch.cuda.synchronize()
            tms, tprof = timed_call(stream, lambda: mvd.mvd_deconvolve_planes(ctx, planes, est), ctx)
            keep(algo)
            # launches sharing one rank-1 factorisation run on the warp-specialised
            # tensor kernels (tcw_*), the others on tc_* / tf32_*
            tk = {}
            for n, (b, f) in budget.items():
                for name in (prefix + "_" + n, "tcw_" + n):
                    r = kernel_roofline(tprof, name, px, b, f, hbm_peak, alu_peak)
                    if r:
                        tk[name] = r
            tc_routes[algo] = {"value": units_per_step / (tms / 1e3), "unit": UNIT, "ms": tms,
                               "precision": precision, "note": "deconvolution only (no reslice)", "kernels": tk}
        except mvd.MvdError as e:
            tc_routes[algo] = {"unavailable": str(e)}
        finally:
            mvd.mvd_set_algo(ctx, "fused")
    tensor_route = tc_routes.get("tensor")
    tf32_route = tc_routes.get("tf32")

    # weighted MV-RL on the padded domain: the planes embedded with zero
    # weights in an R-wide border (data + PSF size), deconvolved there, cropped
    weighted = None
    if leg("weighted"):
        R = ((X + K - 1 + 15) // 16 * 16 - X) // 2    # >= (K-1)/2, padded width a 16-multiple
        pctx = mvd.mvd_create(V, psfs, K, Z + 2 * R, X + 2 * R, iters, "zero", 1e-6)
        mvd.mvd_set_update_order(pctx, order)
        try:
            def padded_run():
                pd, pw = mvd.mvd_embed_padded(planes, R)
                mvd.mvd_set_weights(pctx, pw)
                pest = torch.empty((Y, Z + 2 * R, X + 2 * R), device=dev)
                mvd.mvd_deconvolve_planes(pctx, pd, pest)
                return mvd.mvd_crop_planes(pest, R), (pd, pw, pest)
            out, kept = padded_run()
            torch.cuda.synchronize()
            del out, kept
            res = {}
            wms, wprof = timed_call(stream, lambda: res.setdefault("r", padded_run()), pctx)
            weighted = {"value": units_per_step / (wms / 1e3), "unit": UNIT, "ms": wms,
                        "note": f"padded-domain estimate ({Z + 2 * R}x{X + 2 * R} planes, zero weights in a {R}-pixel "
                                "border, one weight plane per view), embed + weight normalisers + iterations + crop; "
                                "value counts the data voxels",
                        "kernels": {k: {"total_ms": v[0], "launches": v[1]} for k, v in wprof.items()}}
            del res
        finally:
            pctx.close()

    # 3D MV-RL (PSF a_v(y) P_v(z, x), axial sigma = the lateral width) on the
    # same planes, and what the plane-wise approximation loses against it on
    # 3D-blurred synthetic volumes with known truth
    vol3d = None
    if leg("vol3d") and rank == 0:
        from paper_1503_07998_gb300 import synth
        ax = synth.gaussian_1d(11, wl["sigma_lateral"]).astype(np.float32)
        mvd.mvd_set_axial_psfs(ctx, np.stack([ax] * V))
        try:
            mvd.mvd_deconvolve_planes(ctx, planes, est)
            torch.cuda.synchronize()
            vms, vprof = timed_call(stream, lambda: mvd.mvd_deconvolve_planes(ctx, planes, est), ctx)
        finally:
            mvd.mvd_set_axial_psfs(ctx, None)
        study = []
        for sy in (1.5, 3.0, 6.0):
            cs = synth.volume3d_case(48, 128, 128, 31, 8.0, 1.5, sy, n_blobs=200, seed=7)
            sctx = mvd.mvd_create(2, cs["psfs"], 31, 128, 128, iters, "zero", 1e-6)
            try:
                dd = torch.from_numpy(cs["phi"].astype(np.int32)).to(torch.uint16).to(dev)
                e = torch.empty((48, 128, 128), device=dev)
                errs = {}
                for name, axial in (("planewise", None), ("3d", cs["axial"])):
                    mvd.mvd_set_axial_psfs(sctx, axial)
                    mvd.mvd_deconvolve_planes(sctx, dd, e)
                    torch.cuda.synchronize()
                    errs[name] = float(np.linalg.norm(e.cpu().numpy() - cs["truth"]) / np.linalg.norm(cs["truth"]))
                study.append({"sigma_y": sy, "rel_l2_to_truth": errs})
            finally:
                sctx.close()
        vol3d = {"value": units_per_step / (vms / 1e3), "unit": UNIT, "ms": vms,
                 "note": f"3D route on the same planes (axial Gaussian sigma {wl['sigma_lateral']}, 11 taps): "
                         "fused in-plane passes + axial passes; deconvolution only",
                 "kernels": {k: {"total_ms": v[0], "launches": v[1]} for k, v in vprof.items()},
                 "study": {"config": "2 views, 48 planes of 128x128, 200 blobs, K=31 sigma (1.5, 8), 10 iterations, "
                                     "data blurred in 3D with an axial Gaussian of sigma_y, Poisson noise",
                           "results": study}}

    # PSF calibration gradient: 2 views, 64 planes of 256x256, free 31x31
    # PSFs started at sigma (1.2, 5) px on data made with (1.5, 7) px,
    # 10 unrolled iterations, checkpoint every 2
    grad = None
    if leg("grad") and rank == 0:
        from paper_1503_07998_gb300 import synth
        gs, _ = synth.volume_stacks(256, 64, 256, 31, 7.0, 1.5, (0.0, 90.0), 2e-3, seed=5, device=dev)
        gplanes = torch.empty((2, 64, 256, 256), dtype=gs.dtype, device=dev)
        init = np.stack([synth.gaussian_psf(31, 5.0, 1.2, a) for a in (0.0, 90.0)])
        gctx = mvd.mvd_create(2, init, 31, 256, 256, 10, "zero", 1e-6)
        try:
            mvd.mvd_reslice(gctx, gs, gplanes)
            mvd.mvd_psf_grad(gctx, gplanes, 2)
            reps = 3
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(reps):
                loss, _ = mvd.mvd_psf_grad(gctx, gplanes, 2)
            ev1.record()
            torch.cuda.synchronize()
            gms = ev0.elapsed_time(ev1) / reps
            # algorithmic FLOPs of one gradient: every K x K stencil and every
            # K^2-lag sum is 2 K^2 flop per pixel; forward 2TV stencils,
            # terminal fit 2V stencils + V lag sums, recomputed segments 2TV
            # stencils, reverse sweep 2TV stencils + 2TV lag sums
            T_, V_, K_, n_ = 10, 2, 31, 64 * 256 * 256
            n_stencil, n_lag = 6 * T_ * V_ + 2 * V_, 2 * T_ * V_ + V_
            gflop = (n_stencil + n_lag) * 2 * K_ * K_ * n_
            tfl = gflop / (gms * 1e-3) / 1e12
            grad = {"ms_per_gradient": gms, "loss": loss,
                    "config": "2 views, 64 planes 256x256, K=31 free PSFs, 10 iterations, checkpoint every 2",
                    "unrolled_voxel_view_iterations_per_s": n_ * T_ * V_ / (gms * 1e-3),
                    "roofline": {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s",
                                 "frac": tfl / alu_peak, "peak_source": alu_src,
                                 "flops_per_gradient": gflop,
                                 "count": f"{n_stencil} K x K stencils + {n_lag} K^2-lag sums, 2 K^2 flop per pixel each"}}
        finally:
            gctx.close()
            del gs, gplanes

    # end to end through host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        host_in = torch.empty(stacks.shape, dtype=stacks.dtype, pin_memory=True)
        host_in.copy_(stacks)
        host_out = torch.empty((Y, Z, X), dtype=torch.float32, pin_memory=True)
        mvd.mvd_run_host(ctx, host_in, host_out)
        torch.cuda.synchronize()
        barrier(world)
        ne = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(ne):
            mvd.mvd_run_host(ctx, host_in, host_out)
        torch.cuda.synchronize()
        te = reduce_max((time.perf_counter() - t0) / ne, world)
        e2e = {"value": units_per_step * world / te, "unit": UNIT,
               "h2d_bytes_per_step": int(host_in.numel() * host_in.element_size()),
               "d2h_bytes_per_step": int(host_out.numel() * host_out.element_size()),
               "ms_per_step": te * 1e3, "steps_timed": ne}
        del host_in, host_out

    cpu = None
    errors = None
    if not args.no_cpu and world == 1 and rank == 0:
        # spawned workers (safe after CUDA initialisation), created only now:
        # a pool held through the timed regions slowed the host pipeline's
        # end-to-end time by a quarter
        pool = mp.get_context("spawn").Pool(S)
        pool.map(_warm_worker, range(S))
        sp = sample_planes(stacks, idx)
        t, ref = oracle_sample(pool, sp, psfs, iters, order)
        pool.close()
        cpu = {"value": S * Z * X * iters * V / t, "unit": UNIT, "cores": S, "kind": "oracle",
               "sample": f"{S} of the {Y} planes (one per process, all {S} host cores), FP64 Fourier route, "
                         f"{iters} iterations, views {order}"}
        errors = {name: error_vs_oracle(got, ref) for name, got in sampled.items()}

    ctx.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(wl, world),
                "voxel_iterations_per_s": value / V,
                "timing": timing,
                "roofline": roof, "kernels": kr, "cpu_baseline": cpu, "e2e": e2e,
                "error_vs_oracle": errors,
                "gpu_launches": int(launches), "clocks": clk, "sms": sms, "plain_per_plane": plain,
                "fft_route": fft_route, "resident_route": resident, "tensor_route": tensor_route,
                "tf32_route": tf32_route,
                "weighted_padded": weighted, "vol3d": vol3d, "psf_grad": grad,
                "paper_context": "GTX TITAN Black, 2 views, 1024^3 padded, 10 it: 21.1 s = 1.02e9 voxel-view-it/s "
                                 "(Supp. Table 1); another machine, not the target"}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mvd", choices=["mvd", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["batch64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="none of the comparison legs")
    ap.add_argument("--batch-volumes", default="",
                    help="batch64 only: comma list of the volumes (0-63) to run instead of all 64")
    ap.add_argument("--batch-schedule", default="auto", choices=["auto", "graph", "queue"],
                    help="batch64 only: the schedule (auto: mvd_batch_tune picks)")
    ap.add_argument("--legs", default="all",
                    help="comparison legs to run: all, or a comma list of plain,fft,resident,tensor,tf32,weighted,vol3d,grad")
    args = ap.parse_args()
    if args.warmup < 3:
        print("note: at least 3 warm-up steps are used", file=sys.stderr)
        args.warmup = 3
    if args.workload == "batch64":
        return run_batch(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_mvd(args, wl)


def run_batch(args):
    """64 independent volumes of uneven shape (planes 96-768 px square, 16-256
    planes, 2-6 views at k*180/V degrees, odd PSFs 9-41 px with sigma
    (U(1, 2), U(4, 12)) px, 5-20 iterations, blob density 5e-5, seeded per
    volume) run as one captured CUDA graph after autotuning."""
    import torch
    world, rank, _ = dist_setup(args.gpus)
    from paper_1503_07998_gb300 import mvd, shard, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    # the same 64 volumes on every world size; each rank takes its share
    subset = [int(i) for i in args.batch_volumes.split(",")] if args.batch_volumes else list(range(64))
    mine = [subset[i] for i in shard.volumes_of_rank(len(subset), rank, world)]
    allv = [v for i, v in enumerate(synth.uneven_volumes(64, seed=1000, shapes_only=True)) if i in set(subset)]
    vols = synth.uneven_volumes(64, seed=1000, device=dev, only=mine)
    ests = [torch.empty((v["P"], v["H"], v["W"]), device=dev) for v in vols]
    batch = mvd.mvd_batch_create([{"stacks": v["stacks"], "psfs": v["psfs"], "iters": v["iters"], "estimate": e}
                                  for v, e in zip(vols, ests)], order="sequential")
    t0 = time.perf_counter()
    if args.batch_schedule == "auto":
        mvd.mvd_batch_tune(batch)
    else:
        mvd.mvd_batch_set_schedule(batch, args.batch_schedule)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        mvd.mvd_batch_run(batch)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = mvd.mvd_launch_count()
    barrier(world)
    first_row = clocks.mark()
    e0.record(stream)
    for _ in range(args.steps):
        mvd.mvd_batch_run(batch)
    e1.record(stream)
    torch.cuda.synchronize()
    last_row = max(clocks.mark(), first_row + 1)
    barrier(world)
    clk = clocks.stop(first_row, last_row)
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, world)
    units = sum(v["P"] * v["H"] * v["W"] * v["iters"] * v["views"] for v in allv)
    info = mvd.mvd_batch_info(batch)
    info.update(mvd.mvd_batch_queue_info(batch))
    mvd.mvd_batch_device_status(batch)
    # the schedule the tuner did not keep, timed the same way (one step)
    chosen = info["schedule"]
    other = "graph" if chosen == "queue" else "queue"
    schedules = {chosen: ms}
    try:
        mvd.mvd_batch_set_schedule(batch, other)
        mvd.mvd_batch_run(batch)
        torch.cuda.synchronize()
        oms, _ = timed_call(stream, lambda: mvd.mvd_batch_run(batch))
        mvd.mvd_batch_device_status(batch)
        schedules[other] = oms
        schedules[other + "_info"] = mvd.mvd_batch_queue_info(batch)
    except mvd.MvdError as e:
        schedules[other] = {"unavailable": str(e)}
    mvd.mvd_batch_set_schedule(batch, chosen)
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("64 uneven volumes per GPU, one captured CUDA graph, fused-route volumes on "
                                    "the persistent queue when the tuner keeps it (see run_batch)")
                       if len(subset) == 64 else f"volumes {subset} of the 64-volume batch (see run_batch)",
                       "schedule": args.batch_schedule,
                       "voxels": int(sum(v["P"] * v["H"] * v["W"] for v in allv)),
                       "voxel_view_iterations": int(units), "order": "sequential",
                       "l2": "inputs larger than L2",
                       "parallelism": f"{world} GPU(s), volumes dealt round robin, no collective"},
            "batch": info, "schedules_ms": schedules, "tune_s": tune_s, "clocks": clk,
            "gpu_launches": int(mvd.mvd_launch_count() - n0)}
    batch.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
