"""Tensor-level entry points: scene dicts (see workloads.py) in, torch CUDA
tensors out.  Each function turns its arguments into the C structs of
include/fr.h and calls libfr.so on the current torch stream; torch supplies
the device memory and the stream, the kernels do all of the work.
"""
from __future__ import annotations

import ctypes

import torch

from . import _ffi as F


def _f(vals, n):
    return (ctypes.c_float * n)(*[float(v) for v in vals])


def _normal_mode(scene: dict) -> int:
    return {"tetra": F.FR_NORMAL_TETRA, "central": F.FR_NORMAL_CENTRAL,
            "analytic": F.FR_NORMAL_ANALYTIC}[scene["normal_mode"]]


def julia_params(scene: dict) -> F.fr_julia_params:
    p = F.fr_julia_params()
    p.c = _f(scene["c"], 4)
    p.p = int(scene["p"])
    p.slice_w = float(scene["slice_w"])
    p.max_iter = int(scene["max_iter"])
    p.escape_r2 = float(scene["escape_r2"])
    p.bound_radius = float(scene["bound_radius"])
    p.max_steps = int(scene["max_steps"])
    p.eps = float(scene["eps"])
    p.max_step = float(scene["max_step"])
    p.normal_mode = _normal_mode(scene)
    p.normal_h = float(scene["normal_h"])
    return p


def bulb_params(scene: dict) -> F.fr_bulb_params:
    p = F.fr_bulb_params()
    p.n = int(scene["n"])
    p.max_iter = int(scene["max_iter"])
    p.bailout = float(scene["bailout"])
    p.bound_radius = float(scene["bound_radius"])
    p.max_steps = int(scene["max_steps"])
    p.eps = float(scene["eps"])
    p.max_step = float(scene["max_step"])
    p.normal_mode = _normal_mode(scene)
    p.normal_h = float(scene["normal_h"])
    p.algebraic = 1 if scene.get("algebraic") else 0
    return p


def plane_struct(scene: dict) -> F.fr_plane:
    pl = F.fr_plane()
    spec = scene.get("plane")
    pl.enabled = 1 if spec else 0
    if spec:
        pl.n = _f(spec["n"], 3)
        pl.offset = float(spec["o"])
    return pl


def camera_struct(scene: dict) -> F.fr_camera:
    cam = scene["camera"]
    c = F.fr_camera()
    c.eye, c.target, c.up = _f(cam["eye"], 3), _f(cam["target"], 3), _f(cam["up"], 3)
    c.fov_y_deg = float(cam["fov_y_deg"])
    c.width, c.height, c.spp = int(cam["width"]), int(cam["height"]), int(cam["spp"])
    c.seed = int(cam["seed"]) & 0xFFFFFFFF
    return c


def light_struct(scene: dict) -> F.fr_light:
    li = scene["light"]
    L = F.fr_light()
    L.dir, L.albedo = _f(li["dir"], 3), _f(li["albedo"], 3)
    L.k_ambient, L.k_diffuse = float(li["k_ambient"]), float(li["k_diffuse"])
    L.shadows = 1 if li["shadows"] else 0
    L.background = _f(li["background"], 4)
    L.shading = {"lambert": F.FR_SHADE_LAMBERT, "phong": F.FR_SHADE_PHONG}[li.get("shading", "lambert")]
    L.k_specular = float(li.get("k_specular", 0.0))
    L.shininess = float(li.get("shininess", 1.0))
    L.reflect_coef = float(li.get("reflect_coef", 0.0))
    return L


def alloc_image(scene: dict, device="cuda", rgba8=True, rgba=False, depth=True, saved=False,
                stats=False, trap=False) -> dict:
    """Output tensors for one scene: rgba8 (H, W) int32 holding the packed
    uint32, rgba (H, W, 4) float32, depth (H, W) float32, saved (H, W, 4)
    float32, stats (FR_NSTATS,) int64 (zeroed), trap (H, W, 4) float32."""
    H, W = scene["camera"]["height"], scene["camera"]["width"]
    out = {}
    if rgba8:
        out["rgba8"] = torch.empty((H, W), dtype=torch.int32, device=device)
    if rgba:
        out["rgba"] = torch.empty((H, W, 4), dtype=torch.float32, device=device)
    if depth:
        out["depth"] = torch.empty((H, W), dtype=torch.float32, device=device)
    if saved:
        out["saved"] = torch.empty((H, W, 4), dtype=torch.float32, device=device)
    if stats:
        out["stats"] = torch.zeros(F.FR_NSTATS, dtype=torch.int64, device=device)
    if trap:
        out["trap"] = torch.empty((H, W, 4), dtype=torch.float32, device=device)
    return out


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "outputs must be contiguous CUDA tensors"
    return t.data_ptr()


def image_struct(tensors: dict) -> F.fr_image:
    img = F.fr_image()
    img.rgba8 = _ptr(tensors.get("rgba8"))
    img.rgba = _ptr(tensors.get("rgba"))
    img.depth = _ptr(tensors.get("depth"))
    img.saved = _ptr(tensors.get("saved"))
    img.stats = _ptr(tensors.get("stats"))
    img.trap = _ptr(tensors.get("trap"))
    return img


def current_stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def render(scene: dict, out: dict | None = None, stream=None, **alloc) -> dict:
    """Render one scene with the one-ray-per-thread kernel; returns the output
    tensors (allocated with alloc_image(**alloc) unless `out` is given)."""
    if out is None:
        out = alloc_image(scene, **alloc)
    img = image_struct(out)
    s = stream if stream is not None else current_stream()
    if scene["kind"] == "julia":
        st = F.fr_render_julia(julia_params(scene), plane_struct(scene), camera_struct(scene),
                               light_struct(scene), img, s)
    else:
        st = F.fr_render_mandelbulb(bulb_params(scene), plane_struct(scene), camera_struct(scene),
                                    light_struct(scene), img, s)
    F.check(st)
    return out


def request_struct(scene: dict, out: dict) -> F.fr_request:
    r = F.fr_request()
    if scene["kind"] == "julia":
        r.kind = F.FR_KIND_JULIA
        r.julia = julia_params(scene)
    else:
        r.kind = F.FR_KIND_BULB
        r.bulb = bulb_params(scene)
    r.plane = plane_struct(scene)
    r.camera = camera_struct(scene)
    r.light = light_struct(scene)
    r.out = image_struct(out)
    return r


def request_array(scenes, outs):
    arr = (F.fr_request * len(scenes))()
    for i, (s, o) in enumerate(zip(scenes, outs)):
        arr[i] = request_struct(s, o)
    return arr


def workspace(n_reqs: int, device="cuda") -> torch.Tensor:
    nbytes = max(int(F.fr_batch_workspace_bytes(n_reqs)), 256)
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def render_batch(scenes, outs=None, ws=None, stream=None, **alloc):
    """Render all scenes with fr_render_batch (one launch per 64 requests, the
    schedule set by fr_tuning.batch_kernel)."""
    if outs is None:
        outs = [alloc_image(s, **alloc) for s in scenes]
    if ws is None:
        ws = workspace(len(scenes))
    arr = request_array(scenes, outs)
    s = stream if stream is not None else current_stream()
    F.check(F.fr_render_batch(arr, len(scenes), ws.data_ptr(), ws.numel(), s))
    return outs


def unpack_rgba8(t: torch.Tensor):
    """(H, W) packed tensor -> (H, W, 4) uint8 numpy array."""
    import numpy as np

    a = t.detach().cpu().numpy().view(np.uint32)
    return np.stack([(a >> (8 * k)) & 0xFF for k in range(4)], -1).astype(np.uint8)
