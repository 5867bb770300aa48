#!/usr/bin/env python3
"""Throughput benchmark of the sphere tracer on synthetic scenes.

Default (N=1): the Mandelbulb n = 8 at 1920x1080 with one shadow ray per hit
and the cut plane z = 0.1 (camera frame 10 of the orbit), rendered through the
C ABI.  One step = one full frame (every pixel: camera ray, interval, march,
normal, shadow ray, shading, stores).  Prints one JSON line.

  python bench.py [--steps K] [--warmup W] [--workload NAME] [--path plain|persistent]
  python -m torch.distributed.run --nproc-per-node N bench.py --gpus N   (weak scaling:
        every rank renders its own frame of the orbit; no data-path collective)
  python bench.py --impl reference    (the CPU oracle on the host cores, same metric)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2102_01747_gb300 import workloads as W  # noqa: E402

# FP32 operations per unit of work, used for the roofline's achieved FLOP/s
# (units counted per frame by the counting kernel).  Julia degree 2: the orbit
# step of julia_de2 written out (2 FMUL for |z'|^2, 1 FADD for 2x, 3 FFMA for
# the imaginary parts, 1 FMUL + 2 FFMA + 2 FADD for the real part, 1 FMUL +
# 3 FFMA for |z|^2; FFMA = 2) = 24 flops per orbit iteration.  Mandelbulb:
# FP32 operations the float math library executes for one trip of bulb_de
# (sqrt, pow, acos, atan2, two sincos, pow) plus the arithmetic around them;
# provisional estimate until ncu's SASS counters (2*FFMA + FADD + FMUL) are
# divided by the counted orbit iterations.
FLOPS_PER_ITER = {("julia", 2): 24.0, ("julia", 3): 31.0, ("bulb", 8): 178.0}
FP32_LANES_PER_SM = 128  # FFMA lanes per SM (4 sub-partitions x 32)


def workload(name: str, rank: int = 0):
    if name == "bulb_1080p":
        return W.bulb_1080p(10 + rank), "Mandelbulb n=8 1920x1080, 12 iterations, bailout 2, shadow ray, cut z=0.1, frame %d" % (10 + rank)
    if name == "bulb_small":
        return W.bulb_1080p(10 + rank, 480, 270), "Mandelbulb n=8 480x270 (same scene, small case)"
    if name == "julia_256":
        return W.julia_256(), "quaternion Julia q^2+c, c=(-0.2,0.6,0.2,0), 256x256, 11 iterations"
    if name == "stress_bulb_4k":
        return W.stress_bulb_4k(60 + rank), "Mandelbulb n=8 3840x2160 4 spp, iteration cap 12 (frame 60)"
    if name == "stress_julia_4k":
        return W.stress_julia_4k(), "quaternion Julia 3840x2160 with shadow rays"
    raise SystemExit("unknown workload " + name)


def flops_per_iter(scene) -> float:
    key = (scene["kind"], scene["p"] if scene["kind"] == "julia" else scene["n"])
    return FLOPS_PER_ITER.get(key, FLOPS_PER_ITER[("bulb", 8)] if scene["kind"] == "bulb" else 24.0)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [l.split(",") for l in open(self.path) if l.count(",") >= 8]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def fp32_peak_tflops(clock_mhz: float, sms: int) -> float:
    return sms * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12


def run_reference(args, scene, desc, rank, world):
    """CPU oracle (float build) on the host cores, same metric and units."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    n = scene["camera"]["width"] * scene["camera"]["height"]
    # a bounded sample: every k-th pixel row-interleaved, sized to a few seconds per step
    stride = max(1, n // 400_000)
    import numpy as np

    px = np.arange(0, n, stride, dtype=np.int64)
    for _ in range(args.warmup):
        oracle.render(scene, pixels=px[: min(len(px), 20000)], precision="f32", threads=threads)
    t0 = time.perf_counter()
    rays = 0
    for _ in range(args.steps):
        r = oracle.render(scene, pixels=px, precision="f32", threads=threads)
        rays += len(px) * scene["camera"]["spp"] + int(r["stats"][:, 4].sum())
    dt = time.perf_counter() - t0
    value = rays / dt / 1e6
    sample = "every %d-th pixel of the frame (%d pixels per step)" % (stride, len(px))
    print(json.dumps({
        "impl": "reference", "metric": "Mrays/s", "value": value, "unit": "Mrays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(scene, budget_s: float = 12.0):
    """The float oracle on all host cores over a bounded pixel sample."""
    import numpy as np

    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    n = scene["camera"]["width"] * scene["camera"]["height"]
    stride = 64
    t0 = time.perf_counter()
    px = np.arange(0, n, stride, dtype=np.int64)
    r = oracle.render(scene, pixels=px, precision="f32", threads=threads)
    dt = time.perf_counter() - t0
    # grow the sample to the time budget (bounded)
    if dt < budget_s / 4 and stride > 1:
        stride = max(1, int(stride * dt / (budget_s / 2)))
        px = np.arange(0, n, stride, dtype=np.int64)
        t0 = time.perf_counter()
        r = oracle.render(scene, pixels=px, precision="f32", threads=threads)
        dt = time.perf_counter() - t0
    rays = len(px) * scene["camera"]["spp"] + int(r["stats"][:, 4].sum())
    return {"value": rays / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
            "sample": "every %d-th pixel of the same frame (%d pixels, %.1f s)" % (stride, len(px), dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bulb_1080p")
    ap.add_argument("--path", default="plain", choices=["plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    scene, desc = workload(args.workload, rank)

    if args.impl == "reference":
        run_reference(args, scene, desc, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2102_01747_gb300 import api, build as B

    B.build()
    from paper_2102_01747_gb300 import _ffi

    _ffi.load()
    stream = torch.cuda.current_stream(dev)
    H, Wd = scene["camera"]["height"], scene["camera"]["width"]
    spp = scene["camera"]["spp"]

    # counting pass (untimed): rays, DE calls and orbit iterations of one frame
    cnt = api.render(scene, rgba8=False, depth=False, stats=True)
    torch.cuda.synchronize()
    stats = [int(v) for v in cnt["stats"].cpu().tolist()]
    rays_per_frame = stats[0] + stats[1]
    de_per_frame = stats[2] + stats[3] + stats[4]
    iters_per_frame = stats[5]

    out = api.alloc_image(scene, rgba8=True, depth=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step():
        api.render(scene, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flushed between timed frames (outside the events)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    times_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(times_ms) / 1e3
    if dist:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    kernel_ms = statistics.mean(times_ms)
    rays_total = rays_per_frame * args.steps * world
    value = rays_total / total_s / 1e6

    # end to end through the public API with host buffers: the scene parameters
    # go in with the call, the image (rgba8 + depth) comes back to pinned memory
    host_rgba = torch.empty((H, Wd), dtype=torch.int32, pin_memory=True)
    host_depth = torch.empty((H, Wd), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o = api.render(scene, out=out)
        host_rgba.copy_(o["rgba8"], non_blocking=True)
        host_depth.copy_(o["depth"], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = rays_per_frame * args.steps / e2e_s / 1e6

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    c = clk.summary()
    max_mhz = c.get("sm_max_mhz") or 2070.0
    peak = fp32_peak_tflops(max_mhz, sms)
    fpi = flops_per_iter(scene)
    achieved = fpi * iters_per_frame / (kernel_ms / 1e3) / 1e12

    if rank != 0:
        return
    res = {
        "metric": "Mrays/s", "value": value, "unit": "Mrays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "path": args.path, "width": Wd, "height": H, "spp": spp,
                   "l2": "flushed between timed frames (256 MB write)",
                   "parallelism": "replicas (one frame per rank)" if world > 1 else "single GPU"},
        "de_evals_per_s": de_per_frame * args.steps * world / total_s,
        "orbit_iters_per_s": iters_per_frame * args.steps * world / total_s,
        "per_frame": {"rays": rays_per_frame, "primary_rays": stats[0], "shadow_rays": stats[1],
                      "de_calls": de_per_frame, "orbit_iters": iters_per_frame},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "plain_kernel<%s>" % scene["kind"],
                     "flops_per_orbit_iter": fpi,
                     "peak_basis": "FP32 FFMA: %d SMs x %d lanes x 2 x %.0f MHz" % (sms, FP32_LANES_PER_SM, max_mhz),
                     "frac_at_observed_clock": (achieved / fp32_peak_tflops(c["sm_mhz"], sms)) if c.get("sm_mhz") else None},
        "e2e": {"value": e2e_value, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": H * Wd * 8,
                "note": "inputs are scene parameters passed by value in the call (kernel parameters)"},
        "gpu_launches": args.steps,
        "clocks": c,
    }
    if world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(scene)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
