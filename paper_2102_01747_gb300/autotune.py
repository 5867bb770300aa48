"""Autotuner for the launch shapes and schedules of fr_tuning.

For fr_render_batch (tune):
  batch_kernel       1 one-ray-per-thread kernel over all tiles, 2 persistent warps taking the
                     tiles from a queue, 0 persistent lane state machine
  plain_block        threads per CTA of the one-ray-per-thread batch kernel
  plain_unroll       orbit-loop unroll depth of the one-ray-per-thread batch kernels (1 or 2)
  tile_order         order of the tiles in the launch (rows, columns, rows upward)
  sample_lanes       requests with 2, 4 or 8 samples: their samples on adjacent lanes (1) or
                     in turn on one lane (0)
  persist_block      threads per CTA of the persistent kernel (64, 128, 256)
  refill_threshold   idle lanes that trigger a warp refill (the compaction interval)
  persist_unroll     Julia orbit steps per scheduling round (the unroll depth)
For one request through fr_render_julia / fr_render_mandelbulb (tune_single):
  single_kernel      0 the single-request kernel, 2 the batch kernel's code
  plain_block, plain_unroll (orbit-loop unroll depth), tile_order and sample_lanes.
The search is coordinate descent from the current setting: each knob in turn is
swept with the others fixed, each candidate timed with CUDA events (median of a
few calls on the caller's scenes), and a candidate replaces the current
setting only when it is faster by more than `margin` (1 %), so that timing noise
does not move the setting.  A knob of the schedule not in use is skipped.
Every setting renders the same images bit for bit.
Results are cached in a JSON file keyed by GPU name and workload key, so a
later process applies them without searching again.
"""
from __future__ import annotations

import json
import os

import torch

from . import _ffi as F
from . import api

SPACE = {
    "batch_kernel": (1, 2, 0),
    "plain_block": (32, 64, 128, 256),
    "plain_unroll": (1, 2),
    "tile_order": (0, 1, 2),
    "sample_lanes": (1, 0),
    "persist_block": (64, 128, 256),
    "refill_threshold": (1, 2, 4, 8, 16),
    "persist_unroll": (2, 4, 8),
}
SINGLE_SPACE = {
    "single_kernel": (0, 2),
    "plain_block": (32, 64, 128, 256),
    "plain_unroll": (1, 2, 4),
    "tile_order": (0, 1, 2),
    "sample_lanes": (1, 0),
}
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")


def current() -> dict:
    t = F.fr_get_tuning()
    return {n: getattr(t, n) for n, _ in F.fr_tuning._fields_}


def apply(cfg: dict) -> None:
    t = F.fr_get_tuning()
    for k, v in cfg.items():
        setattr(t, k, int(v))
    F.check(F.fr_set_tuning(t))


def _median_ms(run, reps: int) -> float:
    run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def _time_batch(scenes, outs, ws, reps: int) -> float:
    arr = api.request_array(scenes, outs)
    stream = api.current_stream()
    return _median_ms(lambda: F.check(F.fr_render_batch(arr, len(scenes), ws.data_ptr(), ws.numel(), stream)),
                      reps)


def _time_single(scene, out, reps: int) -> float:
    """One fr_render_julia / fr_render_mandelbulb call with prebuilt structs."""
    fn = F.fr_render_julia if scene["kind"] == "julia" else F.fr_render_mandelbulb
    prm = api.julia_params(scene) if scene["kind"] == "julia" else api.bulb_params(scene)
    args = (prm, api.plane_struct(scene), api.camera_struct(scene), api.light_struct(scene),
            api.image_struct(out), api.current_stream())
    return _median_ms(lambda: F.check(fn(*args)), reps)


PERSIST_KNOBS = ("persist_block", "persist_ctas_per_sm", "refill_threshold", "persist_unroll")


def _in_use(knob: str, cfg: dict) -> bool:
    """Whether `knob` changes what fr_render_batch launches under `cfg`."""
    if knob in PERSIST_KNOBS:
        return cfg.get("batch_kernel", 0) == 0
    if knob in ("plain_block", "plain_unroll", "tile_order", "sample_lanes"):
        return cfg.get("batch_kernel", 0) in (1, 2)
    return True


def tune(scenes, reps: int = 5, passes: int = 1, space: dict | None = None, log=None,
         margin: float = 0.01) -> dict:
    """Coordinate descent over `space` for fr_render_batch on `scenes`; returns
    {"config": ..., "ms": ..., "trials": [...]} and leaves the best
    configuration applied."""
    outs = [api.alloc_image(s) for s in scenes]
    ws = api.workspace(len(scenes))
    lanes = _sample_lanes_matter(scenes)
    return _descent(lambda: _time_batch(scenes, outs, ws, reps), space or SPACE,
                    lambda k, c: _in_use(k, c) and (k != "sample_lanes" or lanes), passes, log, margin)


def _sample_lanes_matter(scenes) -> bool:
    """sample_lanes changes the launch only for requests with 2, 4 or 8 samples."""
    return any(s["camera"]["spp"] in (2, 4, 8) for s in scenes)


def tune_single(scene, reps: int = 9, passes: int = 1, space: dict | None = None, log=None,
                margin: float = 0.01, start_kernel: int | None = None) -> dict:
    """The same search for one request through fr_render_julia /
    fr_render_mandelbulb, starting from the single-request kernel
    (single_kernel 0, or start_kernel); the lane state machine (1) is not a
    candidate."""
    out = api.alloc_image(scene)
    apply({"single_kernel": 0 if start_kernel is None else start_kernel})
    lanes = _sample_lanes_matter([scene])
    return _descent(lambda: _time_single(scene, out, reps), space or SINGLE_SPACE,
                    lambda k, c: k != "sample_lanes" or (lanes and c.get("single_kernel", 0) != 1), passes,
                    log, margin)


def _descent(timer, space, in_use, passes, log, margin) -> dict:
    best = current()
    best_ms = timer()
    trials = [dict(best, ms=best_ms)]
    for _ in range(passes):
        for knob, values in space.items():
            if not in_use(knob, best):
                continue
            for v in values:
                if v == best[knob]:
                    continue
                cand = dict(best, **{knob: v})
                apply(cand)
                ms = timer()
                trials.append(dict(cand, ms=ms))
                if log:
                    log("%s=%s: %.3f ms" % (knob, v, ms))
                if ms < best_ms * (1.0 - margin):
                    best, best_ms = cand, ms
            apply(best)
    apply(best)
    return {"config": best, "ms": best_ms, "trials": trials}


def gpu_key() -> str:
    return torch.cuda.get_device_name()


def load_cached(key: str, path: str = DEFAULT_CACHE):
    if not os.path.exists(path):
        return None
    try:
        return json.load(open(path)).get(gpu_key(), {}).get(key)
    except (OSError, ValueError):
        return None


def save_cached(key: str, cfg: dict, ms: float, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    data = {}
    if os.path.exists(path):
        try:
            data = json.load(open(path))
        except (OSError, ValueError):
            data = {}
    data.setdefault(gpu_key(), {})[key] = {"config": cfg, "ms": ms}
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, path)


def tuned(key: str, scenes, reps: int = 5, path: str = DEFAULT_CACHE, retune: bool = False) -> dict:
    """Apply the cached configuration for `key`, or search for it (and cache it)."""
    hit = None if retune else load_cached(key, path)
    if hit:
        apply(hit["config"])
        return {"config": hit["config"], "ms": hit["ms"], "cached": True}
    res = tune(scenes, reps=reps)
    save_cached(key, res["config"], res["ms"], path)
    res["cached"] = False
    return res
