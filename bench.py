#!/usr/bin/env python3
"""Throughput benchmark of the sphere tracer on synthetic scenes.

Default (N=1): the Mandelbulb n = 8 at 1920x1080 with one shadow ray per hit
and the cut plane z = 0.1 (camera frame 10 of the orbit), rendered through the
C ABI.  One step = one full frame (every pixel: camera ray, interval, march,
normal, shadow ray, shading, stores).  Prints one JSON line.

  python bench.py [--steps K] [--warmup W] [--workload NAME] [--path plain|batch]
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2102_01747_gb300 import workloads as W  # noqa: E402

# FP32 operations per orbit iteration, the unit of work of the roofline's
# achieved FLOP/s (units counted per step by the counting kernel).  Each figure
# is the FP32 work the one-ray-per-thread kernel executes per orbit iteration,
# everything included (orbit step, DE epilogue, march update, stencils, camera
# ray, shading): ncu's SASS counters 2*FFMA + FADD + FMUL over one launch
# divided by the iterations counted on the same scene (Mandelbulb n = 8 at
# 1920x1080, the orbit loop unrolled 4 times: 7.363 G / 50.88 M = 144.7;
# Julia p = 2 at 256x256: 356.3 M / 10.27 M = 34.7; Mandelbulb powers 2..10
# at 960x540, the same scene and camera, one request each).  The degree-3
# Julia figure is the degree-2 one scaled by the ratio of their orbit-step
# arithmetic (28 / 24); Mandelbulb powers 11..16 take the n = 10 figure.
FLOPS_PER_ITER = {("julia", 2): 34.7, ("julia", 3): 40.5,
                  ("bulb", 2): 131.0, ("bulb", 3): 135.7, ("bulb", 4): 139.2, ("bulb", 5): 142.8,
                  ("bulb", 6): 144.2, ("bulb", 7): 145.7, ("bulb", 8): 144.7, ("bulb", 9): 149.2,
                  ("bulb", 10): 150.0}
# The algorithmic count of the same work: the operations of the listings'
# formulas as written, each math-library call (sqrt, pow, acos, atan2, sin,
# cos, log) counted as one operation, nothing for the library's internals.
# Per orbit iteration: Julia p = 2, dz2 *= 4 m2 (2), z^2 + c (15), m2 (7);
# p = 3, dz2 *= 9 m2^2 (3), z^3 + c (18), m2 (7); Mandelbulb, r = sqrt(m) (1),
# dz = n r^(n-1) dz + 1 (4 with the pow), b = n acos(y/r) (3),
# a = n atan2(x, z) (2), two sines and two cosines (4), r^n (1), the point
# r^n (sin b sin a, cos b, sin b cos a) + c (8), m = |w|^2 (5).  Per DE call:
# the march point ro + t rd (6), the start |p|^2 (Julia 7, Mandelbulb 5), the
# distance 0.25 log(m) sqrt(...) (Julia 5, Mandelbulb 5) and the step
# t += min(d, max_step) (1).
ALG_PER_ITER = {("julia", 2): 24, ("julia", 3): 28, "bulb": 29}
ALG_PER_DE = {"julia": 19, "bulb": 17}
# DRAM bytes of one launch of the dominant kernel (by the kernel the tuned
# configuration launches), from the ncu capture of the same command
# (dram__bytes_read.sum + dram__bytes_write.sum); the frame's 16.6 MB of
# stores are still in the 129 MB L2 when the kernel ends.
TRAFFIC = {("bulb_1080p", "plain_kernel"): 58880 + 512}
# The kernel sources the two tables above were counted on (sha256 over these
# files in this order): when the sources change, the bench reports the
# figures as stale and the traffic as null until they are counted again.
COUNTED_SOURCES = ("fr_device.cuh", "fr_math.cuh", "fr_trace.cuh", "fr_plain.cuh", "fr_plain.cu", "fr_launch.h")
COUNTED_SHA = "273055e64402ef6e83b575aa52c654ab07f46c72ffc51245c32c84c13e18737b"
FP32_LANES_PER_SM = 128  # FFMA lanes per SM (4 sub-partitions x 32), checked by the FFMA probe


def kernel_sources_sha() -> str:
    import hashlib

    h = hashlib.sha256()
    for name in COUNTED_SOURCES:
        with open(os.path.join(ROOT, "paper_2102_01747_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def workload(name: str, rank: int = 0):
    """(list of scenes rendered per step, description).  Under torchrun every rank
    renders its own frame of the orbit (weak scaling)."""
    if name == "bulb_1080p":
        return [W.bulb_1080p(10 + rank)], ("Mandelbulb n=8 1920x1080, 12 iterations, bailout 2, "
                                           "shadow ray, cut z=0.1, frame %d" % (10 + rank))
    if name == "bulb_1080p_orbit8":
        return [W.bulb_1080p(10 + 8 * rank + k) for k in range(8)], (
            "Mandelbulb n=8 1920x1080, 8 consecutive frames of the camera orbit (from frame %d) in one "
            "fr_render_batch call" % (10 + 8 * rank))
    if name == "bulb_powers":
        sc = []
        for n in range(2, 11):
            s = W.bulb_1080p(10 + rank, 960, 540)
            s["n"] = n
            sc.append(s)
        return sc, "Mandelbulb powers n = 2..10, 960x540 each (bulb_1080p scene), one request per power"
    if name == "bulb_small":
        return [W.bulb_1080p(10 + rank, 480, 270)], "Mandelbulb n=8 480x270 (same scene, small case)"
    if name == "julia_256":
        return [W.julia_256()], "quaternion Julia q^2+c, c=(-0.2,0.6,0.2,0), 256x256, 11 iterations"
    if name == "batch_mixed":
        sc = W.batch_mixed(W.BASE_SEED + rank)
        return sc, "64 mixed requests (Julia / Mandelbulb), sides 128..2048 log-uniform, %d pixels" % (
            W.total_pixels(sc))
    if name == "batch_small":
        sc = W.batch_mixed(W.BASE_SEED + rank, 64, 5.0, 8.0)
        return sc, "64 mixed requests, sides 32..256 (small case)"
    if name == "bulb_1080p_phong":
        return [W.phong(W.bulb_1080p(10 + rank))], (
            "Mandelbulb n=8 1920x1080 (bulb_1080p scene) with Phong lighting and one Fresnel-weighted "
            "mirror ray per hit, frame %d" % (10 + rank))
    if name == "stress_bulb_4k":
        return [W.stress_bulb_4k(60 + rank)], "Mandelbulb n=8 3840x2160 4 spp, iteration cap 12 (frame 60)"
    if name == "stress_julia_4k":
        return [W.stress_julia_4k()], "quaternion Julia 3840x2160 with shadow rays"
    if name == "bulb_1080p_analytic":
        return [dict(W.bulb_1080p(10 + rank), normal_mode="analytic")], (
            "Mandelbulb n=8 1920x1080 (bulb_1080p scene), analytic normal (Sec. 2) instead of the tetrahedral "
            "stencil, frame %d" % (10 + rank))
    if name == "julia_4k_analytic":
        return [dict(W.stress_julia_4k(), normal_mode="analytic")], (
            "quaternion Julia 3840x2160 with shadow rays, analytic normal (Sec. 2) instead of central differences")
    if name == "diff_julia":
        s, start = W.diff_julia(W.BASE_SEED + rank)
        return [s], "differentiable Julia 512x512: forward with saved state + implicit-diff adjoint"
    if name == "stress_anim":
        return [W.stress_bulb_4k(k) for k in range(0, 120, 40)], (
            "Mandelbulb n=8 3840x2160 4 spp, 120 frames, iteration cap 4..20")
    raise SystemExit("unknown workload " + name)


def flops_per_iter(scene) -> float:
    key = (scene["kind"], scene["p"] if scene["kind"] == "julia" else min(scene["n"], 10))
    return FLOPS_PER_ITER[key]


def alg_flops(scene, counts) -> float:
    """Algorithmic FP32 operations of one render of `scene` from its counters."""
    it = ALG_PER_ITER[("julia", scene["p"])] if scene["kind"] == "julia" else ALG_PER_ITER["bulb"]
    de = counts[2] + counts[3] + counts[4] + counts[7]
    return it * counts[5] + ALG_PER_DE[scene["kind"]] * de


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
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _stride_words(stride):
    return "every pixel" if stride == 1 else "every %d-th pixel" % stride


def _oracle_sample(scenes, stride):
    """Pixel sample of the step's scenes: every stride-th pixel of each."""
    import numpy as np

    return [np.arange(0, s["camera"]["width"] * s["camera"]["height"], stride, dtype=np.int64)
            for s in scenes]


def _oracle_rays(oracle, scenes, samples, threads, des=None):
    """Rays the oracle traced for the sampled pixels; DE calls are added to des[0]."""
    rays = 0
    for s, px in zip(scenes, samples):
        r = oracle.render(s, pixels=px, precision="f32", threads=threads)
        st = r["stats"]
        rays += len(px) * s["camera"]["spp"] + int(st[:, 4].sum()) + int(st[:, 6].sum())
        if des is not None:  # primary, normal, shadow and reflection DE calls
            des[0] += int(st[:, 0].sum() + st[:, 1].sum() + st[:, 2].sum() + st[:, 5].sum())
    return rays


def run_reference(args, scenes, desc, rank, world):
    """The CPU oracle (float build) on the host cores: same metric and units,
    each step a bounded pixel sample of the same workload."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    n = sum(s["camera"]["width"] * s["camera"]["height"] for s in scenes)
    stride = max(1, n // 2_000_000)
    samples = _oracle_sample(scenes, stride)
    for _ in range(args.warmup):  # untimed warm-up steps on the same sample
        _oracle_rays(oracle, scenes, samples, threads)
    t0 = time.perf_counter()
    rays, des = 0, [0]
    for _ in range(args.steps):
        rays += _oracle_rays(oracle, scenes, samples, threads, des)
    dt = time.perf_counter() - t0
    value = rays / dt / 1e6
    sample = "%s of each image (%d pixels per step)" % (_stride_words(stride), sum(map(len, samples)))
    print(json.dumps({
        "impl": "reference", "metric": "Mrays/s", "value": value, "unit": "Mrays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "de_evals_per_s": des[0] / dt},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(scenes, budget_s: float = 12.0):
    """The float oracle on all host cores over a bounded pixel sample of the
    same workload, grown until it takes about budget_s."""
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    stride = 256
    while True:
        samples = _oracle_sample(scenes, stride)
        des = [0]
        t0 = time.perf_counter()
        rays = _oracle_rays(oracle, scenes, samples, threads, des)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 3 or stride == 1:
            break
        stride = max(1, int(stride * dt / budget_s) if dt > 0 else 1)
    reps = 1
    while dt * (reps + 1) / reps < budget_s and reps < 20 and dt < budget_s:
        t1 = time.perf_counter()
        rays += _oracle_rays(oracle, scenes, samples, threads, des)
        dt += time.perf_counter() - t1
        reps += 1
    out = {"value": rays / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
           "de_evals_per_s": des[0] / dt,
           "sample": "%s of each image, %d pass%s, %.1f s" % (_stride_words(stride), reps, "" if reps == 1 else "es", dt)}
    # the same oracle on one thread, over a sparser sample of the same images
    one_stride = stride * max(1, threads)
    while True:
        samples = _oracle_sample(scenes, one_stride)
        t0 = time.perf_counter()
        rays1 = _oracle_rays(oracle, scenes, samples, 1)
        dt1 = time.perf_counter() - t0
        if dt1 >= budget_s / 8 or one_stride == 1:
            break
        one_stride = max(1, int(one_stride * dt1 / (budget_s / 4)) if dt1 > 0 else 1)
    out["one_thread"] = {"value": rays1 / dt1 / 1e6, "unit": "Mrays/s", "cores": 1,
                         "sample": "%s of each image, %.1f s" % (_stride_words(one_stride), dt1)}
    return out


class Renderer:
    """Prebuilt C structs for a list of scenes and their outputs, so that a timed
    step is only the C calls (no Python marshalling of parameters)."""

    def __init__(self, api, F, scenes, outs, path, stream, ws=None):
        self.F, self.path, self.stream = F, path, stream
        self.n = len(scenes)
        if path == "plain":
            self.calls = []
            for s, o in zip(scenes, outs):
                fn = F.fr_render_julia if s["kind"] == "julia" else F.fr_render_mandelbulb
                prm = api.julia_params(s) if s["kind"] == "julia" else api.bulb_params(s)
                self.calls.append((fn, prm, api.plane_struct(s), api.camera_struct(s),
                                   api.light_struct(s), api.image_struct(o)))
        else:
            self.arr = api.request_array(scenes, outs)
            self.ws = ws if ws is not None else api.workspace(self.n)

    def launches(self) -> int:
        return self.n if self.path == "plain" else (self.n + 63) // 64

    def __call__(self):
        if self.path == "plain":
            for fn, prm, pl, cam, li, img in self.calls:
                self.F.check(fn(prm, pl, cam, li, img, self.stream))
        else:
            self.F.check(self.F.fr_render_batch(self.arr, self.n, self.ws.data_ptr(), self.ws.numel(),
                                                self.stream))


def time_steps(torch, step, steps, stream, flush, dist=None, clk_index=None):
    """K steps, each bracketed by CUDA events on the launching stream, with the
    L2 flushed (256 MB write) between steps outside the events.  Returns the
    per-step device times (ms), the max over ranks of their sum (s) and clocks."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(clk_index) if clk_index is not None else None
    if clk:
        clk.__enter__()
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    if dist:
        dist.barrier()
    times = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total = max_over_ranks(torch, dist, sum(times) / 1e3, "cuda")
    return times, total, (clk.summary() if clk else None)


def max_over_ranks(torch, dist, seconds: float, device) -> float:
    """The job's time is its slowest rank's (weak scaling: no exchange on the data path)."""
    if not dist:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def count_scenes(api, torch, scenes):
    """Counting-kernel pass (untimed): the FR_STAT_* counters of each scene."""
    from paper_2102_01747_gb300 import _ffi as F

    per = []
    for s in scenes:
        c = api.render(s, rgba8=False, depth=False, stats=True)
        torch.cuda.synchronize()
        per.append([int(v) for v in c["stats"].cpu().tolist()][:F.FR_NSTATS])
    return per


def _sum_counts(per):
    return [sum(c[k] for c in per) for k in range(len(per[0]))]


def rays_of(c):
    return c[0] + c[1] + c[6]  # camera, shadow and mirror rays


def des_of(c):
    return c[2] + c[3] + c[4] + c[7]


def fp32_peak_tflops(clock_mhz: float, sms: int) -> float:
    return sms * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12


def ffma_probe(torch, F, dev, sms: int, seconds: float = 0.05, reps: int = 5) -> dict:
    """The FP32 FFMA rate of this GPU (fr_ffma_probe): 8 blocks of 256 threads per
    SM, each thread 8 independent FFMA chains, launches of about `seconds`;
    the fastest of `reps` timed launches (a burst, like the kernels it is the
    denominator for), with the clocks sampled meanwhile."""
    blocks, threads = sms * 8, 256
    iters = max(1, int(seconds * 80e12 / F.fr_ffma_probe_flops(blocks, threads, 1)))
    sink = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def launch():
        F.check(F.fr_ffma_probe(blocks, threads, iters, sink.data_ptr(), stream.cuda_stream))

    for _ in range(2):
        launch()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(dev.index or 0) as clk:
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            launch()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    c = clk.summary()
    flops = F.fr_ffma_probe_flops(blocks, threads, iters)
    tflops = flops / (min(ms) / 1e3) / 1e12
    mhz = c.get("sm_mhz") or 2070.0
    return {"tflops": tflops, "ms_per_launch": min(ms), "launch": [blocks, threads, iters],
            "flops_per_launch": flops, "clocks": c,
            "ffma_lanes_per_sm": tflops * 1e12 / (sms * 2 * mhz * 1e6)}


def roofline_of(flops_ncu, flops_alg, kernel_ms, launches, peak, peak_derived, traffic, kern):
    achieved = flops_ncu / launches / (kernel_ms / 1e3) / 1e12
    achieved_alg = flops_alg / launches / (kernel_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kern,
            "achieved_algorithmic": achieved_alg, "frac_algorithmic": achieved_alg / peak,
            "frac_of_derived_peak": achieved / peak_derived}


def measure(args, torch, api, F, scenes, path, env, steps, warmup, clk_index=None, tune=True, tune_reps=3,
            compare=True, dist=None, world=1):
    """Counters, an optional untimed autotuner search, then `steps` timed steps of
    the scenes through `path` (and through the other path when `compare`).
    Returns the measurement and the tuning the autotuner left applied."""
    dev, tstream, flush = env["dev"], env["tstream"], env["flush"]
    stream = api.current_stream(dev)
    tuning = None
    if tune and path == "batch":
        from paper_2102_01747_gb300 import autotune

        space = dict(autotune.SPACE)
        if args.batch_kernel is not None:
            del space["batch_kernel"]
        if args.tile_order is not None:
            del space["tile_order"]
        if args.sample_lanes is not None:
            del space["sample_lanes"]
        if args.unroll is not None:
            del space["plain_unroll"]
        r = autotune.tune(scenes, reps=tune_reps, space=space)  # untimed search over the launch shape
        tuning = {"config": r["config"], "search_ms": r["ms"], "trials": len(r["trials"])}
    elif tune and path == "plain" and len(scenes) == 1:
        from paper_2102_01747_gb300 import autotune

        space = dict(autotune.SINGLE_SPACE)
        if args.tile_order is not None:
            del space["tile_order"]
        if args.single_kernel is not None:
            del space["single_kernel"]
        if args.sample_lanes is not None:
            del space["sample_lanes"]
        if args.unroll is not None:
            del space["plain_unroll"]
        r = autotune.tune_single(scenes[0], reps=max(tune_reps, 3), space=space, start_kernel=args.single_kernel)
        tuning = {"config": r["config"], "search_ms": r["ms"], "trials": len(r["trials"]),
                  "trial_ms": [[{k: t[k] for k in space}, round(t["ms"], 4)] for t in r["trials"]]}
    per = count_scenes(api, torch, scenes)
    tot = _sum_counts(per)
    flops_ncu = sum(flops_per_iter(s) * c[5] for s, c in zip(scenes, per))
    flops_alg = sum(alg_flops(s, c) for s, c in zip(scenes, per))
    outs = [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]
    paths = [path] + ([p for p in ("plain", "batch") if p != path] if compare else [])
    results = {}
    for pth in paths:
        step = Renderer(api, F, scenes, outs, pth, stream)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        times, total_s, clk = time_steps(torch, step, steps, tstream, flush, dist,
                                         clk_index=clk_index if pth == path else None)
        results[pth] = {"times": times, "total_s": total_s, "clk": clk, "launches": step.launches()}
    tu = F.fr_get_tuning()
    if path == "plain":  # the kernel fr_render_* launches under the tuned single_kernel
        kern = {0: "plain_kernel", 1: "persist_kernel", 2: "batch_plain_kernel"}[tu.single_kernel]
    else:
        kern = {0: "persist_kernel", 1: "batch_plain_kernel", 2: "batch_refill_kernel"}[tu.batch_kernel]
    main_r = results[path]
    return {"per": per, "counts": tot, "flops_ncu": flops_ncu, "flops_alg": flops_alg, "outs": outs,
            "results": results, "main": main_r, "kernel": kern, "tuning": tuning,
            "value": rays_of(tot) * steps * world / main_r["total_s"] / 1e6,
            "kernel_ms": statistics.mean(main_r["times"]) / main_r["launches"]}


def summary_of(m, steps, peak, peak_derived, traffic=None, world=1):
    """The compact record of a measurement (for the extras)."""
    total_s = m["main"]["total_s"]
    out = {"ms_per_step": total_s / steps * 1e3, "value": m["value"], "unit": "Mrays/s",
           "rays_per_step": rays_of(m["counts"]), "de_calls_per_step": des_of(m["counts"]),
           "orbit_iters_per_step": m["counts"][5],
           "de_evals_per_s": des_of(m["counts"]) * steps * world / total_s,
           "roofline": roofline_of(m["flops_ncu"], m["flops_alg"], m["kernel_ms"], m["main"]["launches"], peak,
                                   peak_derived, traffic, m["kernel"])}
    for pth, r in m["results"].items():
        if r is not m["main"]:
            out["other_path"] = {"path": pth, "ms_per_step": r["total_s"] / steps * 1e3,
                                 "launches_per_step": r["launches"]}
            out["speedup_vs_" + pth] = r["total_s"] / total_s
    if m["tuning"]:
        out["tuning"] = {k: v for k, v in m["tuning"].items() if k != "trial_ms"}
    return out


def measure_gradient(args, torch, api, F, scene, steps, warmup):
    """One step = a differentiable Julia render (colour, depth, saved hit state) plus
    the adjoint (fr_render_backward) of an L2 loss: gradients per second.  The
    finite-difference alternative needs 22 forward renders per gradient (central
    differences over c[4], plane n[3], offset, light[3])."""
    s = scene
    out = api.alloc_image(s, rgba8=False, rgba=True, depth=True, saved=True)
    target = api.render(s, rgba8=False, rgba=True, depth=False)["rgba"].clone()
    grad = torch.zeros(11, dtype=torch.float32, device="cuda")
    d_rgba = torch.empty_like(out["rgba"])
    prm, pl, cam, li = api.julia_params(s), api.plane_struct(s), api.camera_struct(s), api.light_struct(s)
    img = api.image_struct(out)
    stream = api.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def forward():
        F.check(F.fr_render_julia(prm, pl, cam, li, img, stream))

    def step():
        forward()
        torch.sub(out["rgba"], target, out=d_rgba)  # dL/drgba of 0.5 |rgba - target|^2
        F.check(F.fr_render_backward(prm, pl, cam, li, out["saved"].data_ptr(), d_rgba.data_ptr(),
                                     None, grad.data_ptr(), stream))

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tstream = torch.cuda.current_stream()
    times, total_s, clk = time_steps(torch, step, steps, tstream, flush, None, clk_index=0)
    ftimes, ftotal, _ = time_steps(torch, forward, steps, tstream, flush, None)
    grad_per_s = steps / total_s
    fd_per_s = 1.0 / (22 * ftotal / steps)
    e2e_t0 = time.perf_counter()
    for _ in range(steps):
        step()
        grad.cpu()
    e2e = steps / (time.perf_counter() - e2e_t0)
    return {"value": grad_per_s, "unit": "grad/s", "ms_per_step": total_s / steps * 1e3,
            "forward_ms": ftotal / steps * 1e3, "fd_grad_per_s": fd_per_s, "speedup_vs_fd": grad_per_s / fd_per_s,
            "e2e": {"value": e2e, "unit": "grad/s", "h2d_bytes_per_step": ctypes_sizeof_inputs(F, 1),
                    "d2h_bytes_per_step": 44},
            "clocks": clk, "width": s["camera"]["width"], "height": s["camera"]["height"]}


def cpu_gradient_baseline(scene, budget_s: float = 10.0):
    """The oracle's double-precision gradient (forward-mode dual numbers, the
    march included) of the same scene and a fixed random cotangent, on all host
    cores, over every stride-th pixel (the stride grown until the sample takes
    about budget_s / 2); reported as whole-image gradients per second."""
    import numpy as np

    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    n = scene["camera"]["width"] * scene["camera"]["height"]
    rng = np.random.default_rng(W.BASE_SEED)
    d_rgba = rng.standard_normal((n, 4))
    d_depth = 0.3 * rng.standard_normal(n)
    stride = 64
    while True:
        mask = np.zeros(n, np.uint8)
        mask[::stride] = 1
        t0 = time.perf_counter()
        oracle.julia_grad(scene, d_rgba, d_depth, mask=mask, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 4 or stride == 1:
            break
        stride = max(1, int(stride * dt / (budget_s / 2)) if dt > 0 else 1)
    reps = 1
    while dt < budget_s / 2 and reps < 10:
        t0 = time.perf_counter()
        oracle.julia_grad(scene, d_rgba, d_depth, mask=mask, threads=threads)
        dt += time.perf_counter() - t0
        reps += 1
    frac = float(mask.sum()) / n
    return {"value": reps * frac / dt, "unit": "grad/s", "cores": threads, "kind": "oracle",
            "sample": "%s of the image, %d pass%s, %.1f s (double precision, dual numbers)" % (
                _stride_words(stride), reps, "" if reps == 1 else "es", dt)}


def run_gradient(args, torch, api, F, scenes, desc, rank, world):
    g = measure_gradient(args, torch, api, F, scenes[0], args.steps, args.warmup)
    if rank != 0:
        return
    extra = {}
    if world == 1 and not args.no_cpu_baseline:
        extra["cpu_baseline"] = cpu_gradient_baseline(scenes[0])
    print(json.dumps({
        "metric": "grad/s", "value": g["value"], "unit": "grad/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": g["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": desc, "width": g["width"], "height": g["height"],
                                        "l2": "flushed between timed steps (256 MB write)"},
        "forward_ms": g["forward_ms"], "fd_grad_per_s": g["fd_grad_per_s"], "speedup_vs_fd": g["speedup_vs_fd"],
        "e2e": g["e2e"], "gpu_launches": 2 * args.steps, "clocks": g["clocks"], **extra,
    }))


def run_animation(args, torch, api, F, desc, rank, world):
    """The animated stress scene: 120 frames of the Mandelbulb at 3840x2160 with 4
    jittered samples, iteration cap 4 + floor(16k/119) and the camera at azimuth
    3k degrees; per-frame device time (CUDA events), median and p95."""
    frames = [W.stress_bulb_4k(k) for k in range(120)]
    out = api.alloc_image(frames[0], rgba8=True, depth=True)
    stream = api.current_stream()
    tstream = torch.cuda.current_stream()
    tuning = None
    if args.path == "plain" and not args.no_autotune:
        from paper_2102_01747_gb300 import autotune

        # untimed search on the middle frame (cap 12); every frame then runs with it
        space = {k: v for k, v in autotune.SINGLE_SPACE.items() if k != "plain_unroll"}
        tuning = autotune.tune_single(frames[60], reps=3, space=space)["config"]
    steps = [Renderer(api, F, [f], [out], args.path, stream) for f in frames]
    for st in steps[:args.warmup]:
        st()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in frames]
    with ClockSampler(0) as clk:
        for (a, b), st in zip(ev, steps):
            a.record(tstream)
            st()
            b.record(tstream)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    srt = sorted(ms)
    rays = [3840 * 2160 * 4] * len(frames)
    if rank != 0:
        return
    print(json.dumps({
        "metric": "ms/frame", "value": statistics.median(ms), "unit": "ms", "n_gpus": world,
        "steps": len(frames), "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": desc, "path": args.path},
        "p95_ms": srt[int(0.95 * (len(srt) - 1))], "max_ms": srt[-1],
        "per_frame_ms": [round(v, 3) for v in ms],
        "primary_mrays_per_s": sum(rays) / (sum(ms) / 1e3) / 1e6,
        "gpu_launches": len(frames), "clocks": clk.summary(), "tuning": tuning,
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bulb_1080p")
    ap.add_argument("--path", default="auto", choices=["auto", "plain", "batch"],
                    help="plain: one fr_render_julia/fr_render_mandelbulb call per request; batch: "
                         "fr_render_batch over all requests (schedule autotuned); auto: plain for one "
                         "request, batch for several")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other path")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the other configurations and the FFMA probe")
    ap.add_argument("--no-autotune", action="store_true", help="keep the current launch shape")
    ap.add_argument("--single-kernel", type=int, choices=(0, 1, 2), default=None,
                    help="fix the kernel of fr_render_julia / fr_render_mandelbulb (0 single-request "
                         "kernel, 1 lane state machine, 2 batch kernel); the autotuner then keeps it")
    ap.add_argument("--tile-order", type=int, choices=(0, 1, 2), default=None,
                    help="fix the tile order of the one-ray-per-thread kernels (0 rows, 1 columns, "
                         "2 rows upward); the autotuner then keeps it")
    ap.add_argument("--batch-kernel", type=int, choices=[0, 1, 2], default=None,
                    help="fix fr_render_batch's schedule (1 one-ray-per-thread kernel over all "
                         "tiles, 2 persistent warps taking tiles from a queue, 0 persistent lane "
                         "state machine); the autotuner then keeps it")
    ap.add_argument("--unroll", type=int, choices=[1, 2, 4], default=None,
                    help="fix the orbit-loop unroll depth of the one-ray-per-thread kernels "
                         "(the batch kernels take 1 or 2); the autotuner then keeps it")
    ap.add_argument("--sample-lanes", type=int, choices=[0, 1], default=None,
                    help="fix where a pixel's 2, 4 or 8 samples run (1 adjacent lanes, 0 in turn on "
                         "one lane); the autotuner then keeps it")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    scenes, desc = workload(args.workload, rank)

    if args.impl == "reference":
        run_reference(args, scenes, desc, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api, build as B

    B.build()
    F.load()
    if (args.batch_kernel is not None or args.tile_order is not None or args.single_kernel is not None
            or args.sample_lanes is not None or args.unroll is not None):
        t = F.fr_get_tuning()
        if args.unroll is not None:
            t.plain_unroll = args.unroll
        if args.sample_lanes is not None:
            t.sample_lanes = args.sample_lanes
        if args.batch_kernel is not None:
            t.batch_kernel = args.batch_kernel
        if args.single_kernel is not None:
            t.single_kernel = args.single_kernel
        if args.tile_order is not None:
            t.tile_order = args.tile_order
        F.check(F.fr_set_tuning(t))
    tstream = torch.cuda.current_stream(dev)
    if args.path == "auto":
        # the animation renders its frames one call each
        args.path = "plain" if len(scenes) == 1 or args.workload == "stress_anim" else "batch"
    if args.workload == "diff_julia":
        return run_gradient(args, torch, api, F, scenes, desc, rank, world)
    if args.workload == "stress_anim":
        return run_animation(args, torch, api, F, desc, rank, world)

    env = {"dev": dev, "tstream": tstream,
           "flush": torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)}  # > 129 MB L2
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    extras = args.workload == "bulb_1080p" and not args.no_extras and world == 1
    probe = ffma_probe(torch, F, dev, sms) if extras else None

    m = measure(args, torch, api, F, scenes, args.path, env, args.steps, args.warmup, clk_index=local,
                tune=not args.no_autotune, tune_reps=9, compare=not args.no_compare, dist=dist, world=world)
    main_r, outs = m["main"], m["outs"]
    total_s = main_r["total_s"]
    counts = m["counts"]
    rays_per_step = rays_of(counts)

    # end to end through the public API with host buffers: the scene parameters go
    # in with the call, every image (rgba8 + depth) comes back to pinned memory.
    # Serial: render, copy back, wait, every step.  Pipelined (the reported
    # value): two sets of output buffers, the copy of step k on a second stream
    # while step k + 1 renders; a buffer is rendered into again only after its
    # previous copy has finished, and the clock stops when the last copy lands.
    hosts = [(torch.empty(o["rgba8"].shape, dtype=torch.int32, pin_memory=True),
              torch.empty(o["depth"].shape, dtype=torch.float32, pin_memory=True)) for o in outs]

    def e2e_render(os_):
        if args.path == "plain":
            for s, o in zip(scenes, os_):
                api.render(s, out=o)
        else:
            api.render_batch(scenes, os_)

    def e2e_copy(os_):
        for (hr, hd), o in zip(hosts, os_):
            hr.copy_(o["rgba8"], non_blocking=True)
            hd.copy_(o["depth"], non_blocking=True)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_render(outs)
        e2e_copy(outs)
        torch.cuda.synchronize()
    e2e_serial = rays_per_step * args.steps / (time.perf_counter() - t0) / 1e6

    bufs = [outs, [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]]
    cstream = torch.cuda.Stream(dev)
    copied = [None, None]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        b = k & 1
        if copied[b] is not None:
            tstream.wait_event(copied[b])
        e2e_render(bufs[b])
        rendered = torch.cuda.Event()
        rendered.record(tstream)
        cstream.wait_event(rendered)
        with torch.cuda.stream(cstream):
            e2e_copy(bufs[b])
            copied[b] = torch.cuda.Event()
            copied[b].record(cstream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = rays_per_step * args.steps / e2e_s / 1e6
    in_bytes = ctypes_sizeof_inputs(F, len(scenes))
    out_bytes = sum(o["rgba8"].numel() * 4 + o["depth"].numel() * 4 for o in outs)

    c = main_r["clk"] or {}
    max_mhz = c.get("sm_max_mhz") or 2070.0
    peak_derived = fp32_peak_tflops(max_mhz, sms)
    peak = probe["tflops"] if probe else peak_derived
    fresh = kernel_sources_sha() == COUNTED_SHA
    traffic = TRAFFIC.get((args.workload, m["kernel"])) if fresh else None
    roof = roofline_of(m["flops_ncu"], m["flops_alg"], m["kernel_ms"], main_r["launches"], peak, peak_derived,
                       traffic, m["kernel"])
    roof.update({
        "flops_per_step": m["flops_ncu"], "flops_per_step_algorithmic": m["flops_alg"],
        "per_unit_figures_current": fresh,
        "peak_basis": ("measured: FFMA probe (fr_ffma_probe), fastest of 5 launches of %.0f ms" %
                       probe["ms_per_launch"]) if probe else
                      "derived: %d SMs x %d lanes x 2 flops x %.0f MHz (max clock)" % (sms, FP32_LANES_PER_SM, max_mhz),
        "peak_derived": peak_derived,
        "peak_derived_basis": "%d SMs x %d FFMA lanes x 2 flops x %.0f MHz (max clock)" % (
            sms, FP32_LANES_PER_SM, max_mhz),
        "frac_at_observed_clock": (m["flops_ncu"] / main_r["launches"] / (m["kernel_ms"] / 1e3) / 1e12 /
                                   fp32_peak_tflops(c["sm_mhz"], sms)) if c.get("sm_mhz") else None,
    })

    if rank != 0:
        return
    res = {
        "metric": "Mrays/s", "value": m["value"], "unit": "Mrays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "path": args.path, "requests": len(scenes),
                   "pixels_per_step": sum(s["camera"]["width"] * s["camera"]["height"] for s in scenes),
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas (one frame per rank)" if world > 1 else "single GPU"},
        "de_evals_per_s": des_of(counts) * args.steps * world / total_s,
        "orbit_iters_per_s": counts[5] * args.steps * world / total_s,
        "per_step": {"rays": rays_per_step, "primary_rays": counts[0], "shadow_rays": counts[1],
                     "mirror_rays": counts[6], "de_calls": des_of(counts), "orbit_iters": counts[5]},
        "per_request": ([{"rays": rays_of(c), "de_calls": des_of(c), "orbit_iters": c[5]} for c in m["per"]]
                        if 1 < len(scenes) <= 16 else None),
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "Mrays/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes, "serial_value": e2e_serial,
                "note": "inputs are the scene parameter structs passed in each call; value: the copy of "
                        "step k back to pinned host memory overlaps the render of step k+1 (two output "
                        "buffers, a copy stream); serial_value: render, copy, wait every step"},
        "gpu_launches": main_r["launches"] * args.steps,
        "clocks": c,
        "tuning": m["tuning"],
    }
    for path, r in m["results"].items():
        if path != args.path:
            res["other_path"] = {"path": path,
                                 "value": rays_per_step * args.steps * world / r["total_s"] / 1e6,
                                 "ms_per_step": r["total_s"] / args.steps * 1e3}
            res["speedup_vs_" + path] = r["total_s"] / total_s
    if extras:
        res["extras"] = bulb_extras(args, torch, api, F, scenes, env, peak, peak_derived)
        res["extras"]["ffma_probe"] = probe
        res["extras"].update(other_configs(args, torch, api, F, env, peak, peak_derived))
    if world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(scenes)
    print(json.dumps(res))


def bulb_extras(args, torch, api, F, scenes, env, peak, peak_derived):
    """More views of the same frame, each timed like the headline (CUDA events,
    L2 flushed): (1) Eq. 1 evaluated without transcendental calls (de Moivre
    powers; same image within the parity bar); (2) the analytic normal in place
    of the tetrahedral stencil; (3) with the orbit-trap output; (4) eight
    consecutive frames of the camera orbit in one fr_render_batch call, where
    one frame's slowest pixels overlap the other frames' work (the steady state
    of an animation)."""
    out = {}
    n = max(5, args.steps // 2)
    w = 3
    alg = [dict(s, algebraic=True) for s in scenes]
    for name, sc in (("algebraic_power", alg), ("analytic_normal", [dict(s, normal_mode="analytic") for s in scenes])):
        mm = measure(args, torch, api, F, sc, "plain", env, n, w, tune=False, compare=False)
        out[name] = dict(summary_of(mm, n, peak, peak_derived), path="plain")
    # the orbit-trap output (one more DE per hit pixel)
    per = count_scenes(api, torch, scenes)
    oo = [api.alloc_image(s, trap=True) for s in scenes]
    step = Renderer(api, F, scenes, oo, "plain", api.current_stream())
    for _ in range(w):
        step()
    times, total, _ = time_steps(torch, step, n, env["tstream"], env["flush"])
    out["orbit_trap"] = {"path": "plain", "ms_per_step": total / n * 1e3,
                         "value": rays_of(_sum_counts(per)) * n / total / 1e6, "unit": "Mrays/s"}
    frames = [W.bulb_1080p(10 + k) for k in range(8)]
    mm = measure(args, torch, api, F, frames, "batch", env, n, w, tune=False, compare=False)
    out["eight_frames_in_flight"] = dict(summary_of(mm, n, peak, peak_derived), path="batch",
                                         batch_kernel=F.fr_get_tuning().batch_kernel,
                                         workload="Mandelbulb n=8 1920x1080, frames 10..17 of the camera "
                                                  "orbit in one fr_render_batch call",
                                         ms_per_frame=mm["main"]["total_s"] / n * 1e3 / 8)
    return out


def other_configs(args, torch, api, F, env, peak, peak_derived):
    """The other configurations, each measured in the same run as the headline:
    the 64-request mixed batch (autotuned schedule against one plain launch per
    request), the differentiable Julia render (grad/s against finite
    differences) and one 4K frame of the stress animation (4 jittered samples)."""
    out = {}
    keep = F.fr_get_tuning()
    keep = F.fr_tuning(*[getattr(keep, k) for k, _ in F.fr_tuning._fields_])
    try:
        sc, desc = workload("batch_mixed")
        mm = measure(args, torch, api, F, sc, "batch", env, 5, 3, tune=True, tune_reps=3, compare=True)
        out["batch_mixed"] = dict(summary_of(mm, 5, peak, peak_derived), workload=desc, path="batch")
        F.check(F.fr_set_tuning(keep))
        sc, desc = workload("stress_bulb_4k")
        mm = measure(args, torch, api, F, sc, "plain", env, 5, 3, tune=True, tune_reps=3, compare=False)
        out["stress_bulb_4k"] = dict(summary_of(mm, 5, peak, peak_derived), workload=desc, path="plain")
        F.check(F.fr_set_tuning(keep))
        sc, desc = workload("diff_julia")
        g = measure_gradient(args, torch, api, F, sc[0], 20, 5)
        out["diff_julia"] = dict(g, workload=desc)
    finally:
        F.fr_set_tuning(keep)
    return out


def ctypes_sizeof_inputs(F, n):
    import ctypes

    return n * (ctypes.sizeof(F.fr_request) - ctypes.sizeof(F.fr_image))


if __name__ == "__main__":
    main()
