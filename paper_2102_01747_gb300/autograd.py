"""torch.autograd.Function around the Julia render and its adjoint.

    rgba, depth = julia_render(scene, c, plane_n, plane_o, light_dir)

rgba (H, W, 4) float32 and depth (H, W) float32 (+inf on a miss) come from
fr_render_julia with the float colour and the saved hit state requested; the
backward pass is fr_render_backward_ws (implicit differentiation at the saved
hit points, reverse mode through the recomputed orbit) with a workspace of its
own, so backward passes on different streams may overlap.  The differentiable inputs
are 1-D tensors: c (4), plane_n (3), plane_o (1), light_dir (3).  Every other
parameter is taken from `scene`.  Gradients with respect to the alpha channel
are ignored (alpha is piecewise constant); so are depth cotangents on pixels
that miss.

    rgba, depth = bulb_render(scene, plane_n, plane_o, light_dir)

is the same for a Mandelbulb scene, differentiable with respect to the cut
plane and the light (fr_render_backward_mandelbulb; the fractal has no c).
"""
from __future__ import annotations

import copy

import torch

from . import _ffi as F
from . import api


def _scene_with(scene, c, plane_n, plane_o, light_dir):
    s = copy.deepcopy(scene)
    s["c"] = tuple(float(v) for v in c.detach().cpu().tolist())
    s["plane"] = {"n": tuple(float(v) for v in plane_n.detach().cpu().tolist()),
                  "o": float(plane_o.detach().cpu().reshape(-1)[0])}
    s["light"]["dir"] = tuple(float(v) for v in light_dir.detach().cpu().tolist())
    return s


class JuliaRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, plane_n, plane_o, light_dir, scene):
        s = _scene_with(scene, c, plane_n, plane_o, light_dir)
        if s["kind"] != "julia" or s["camera"]["spp"] != 1:
            raise ValueError("the differentiable render takes a Julia scene with spp = 1")
        out = api.render(s, rgba8=False, rgba=True, depth=True, saved=True)
        ctx.scene = s
        ctx.save_for_backward(out["saved"])
        ctx.dev = out["rgba"].device
        ctx.in_dev = (c.device, plane_n.device, plane_o.device, light_dir.device)
        return out["rgba"], out["depth"]

    @staticmethod
    def backward(ctx, d_rgba, d_depth):
        (saved,) = ctx.saved_tensors
        s = ctx.scene
        grad = torch.zeros(11, dtype=torch.float32, device=ctx.dev)
        d_rgba = (torch.zeros_like(saved) if d_rgba is None else d_rgba).float().contiguous()
        dd = None
        if d_depth is not None:
            dd = torch.nan_to_num(d_depth.float(), nan=0.0, posinf=0.0, neginf=0.0).contiguous()
        ws = backward_workspace(ctx.dev)
        st = F.fr_render_backward_ws(api.julia_params(s), api.plane_struct(s), api.camera_struct(s),
                                     api.light_struct(s), saved.data_ptr(), d_rgba.data_ptr(),
                                     None if dd is None else dd.data_ptr(), grad.data_ptr(),
                                     ws.data_ptr(), ws.numel() * ws.element_size(),
                                     api.current_stream(ctx.dev))
        F.check(st)
        dc, dn, do, dl = ctx.in_dev
        return grad[0:4].to(dc), grad[4:7].to(dn), grad[7:8].to(do), grad[8:11].to(dl), None


def julia_render(scene, c, plane_n, plane_o, light_dir):
    return JuliaRender.apply(c, plane_n, plane_o, light_dir, scene)


class BulbRender(torch.autograd.Function):
    """The Mandelbulb render, differentiable with respect to the cut plane and
    the light (fr_render_backward_mandelbulb; the fractal has no parameter c)."""

    @staticmethod
    def forward(ctx, plane_n, plane_o, light_dir, scene):
        s = copy.deepcopy(scene)
        s["plane"] = {"n": tuple(float(v) for v in plane_n.detach().cpu().tolist()),
                      "o": float(plane_o.detach().cpu().reshape(-1)[0])}
        s["light"]["dir"] = tuple(float(v) for v in light_dir.detach().cpu().tolist())
        if s["kind"] != "bulb" or s["camera"]["spp"] != 1:
            raise ValueError("the differentiable Mandelbulb render takes a Mandelbulb scene with spp = 1")
        out = api.render(s, rgba8=False, rgba=True, depth=True, saved=True)
        ctx.scene = s
        ctx.save_for_backward(out["saved"])
        ctx.in_dev = (plane_n.device, plane_o.device, light_dir.device)
        return out["rgba"], out["depth"]

    @staticmethod
    def backward(ctx, d_rgba, d_depth):
        (saved,) = ctx.saved_tensors
        d_rgba = (torch.zeros_like(saved) if d_rgba is None else d_rgba).float().contiguous()
        dd = None
        if d_depth is not None:
            dd = torch.nan_to_num(d_depth.float(), nan=0.0, posinf=0.0, neginf=0.0).contiguous()
        grad = backward_raw(ctx.scene, saved, d_rgba, dd, workspace=backward_workspace(saved.device))
        dn, do, dl = ctx.in_dev
        return grad[4:7].to(dn), grad[7:8].to(do), grad[8:11].to(dl), None


def bulb_render(scene, plane_n, plane_o, light_dir):
    return BulbRender.apply(plane_n, plane_o, light_dir, scene)


def backward_workspace(device) -> torch.Tensor:
    """Device scratch for one fr_render_backward_ws call (16-byte aligned)."""
    return torch.empty((int(F.fr_backward_workspace_bytes()) + 7) // 8, dtype=torch.float64, device=device)


def backward_raw(scene, saved, d_rgba, d_depth=None, grad=None, workspace=None):
    """Direct call of fr_render_backward (the library's accumulator) or, with a
    workspace tensor, fr_render_backward_ws; returns the 11-vector
    (accumulated into grad)."""
    if grad is None:
        grad = torch.zeros(11, dtype=torch.float32, device=saved.device)
    if scene["kind"] == "bulb":  # plane and light only (the Mandelbulb has no c)
        st = F.fr_render_backward_mandelbulb(
            api.bulb_params(scene), api.plane_struct(scene), api.camera_struct(scene), api.light_struct(scene),
            saved.data_ptr(), d_rgba.data_ptr(), None if d_depth is None else d_depth.data_ptr(), grad.data_ptr(),
            None if workspace is None else workspace.data_ptr(),
            0 if workspace is None else workspace.numel() * workspace.element_size(), api.current_stream(saved.device))
        F.check(st)
        return grad
    args = (api.julia_params(scene), api.plane_struct(scene), api.camera_struct(scene),
            api.light_struct(scene), saved.data_ptr(), d_rgba.data_ptr(),
            None if d_depth is None else d_depth.data_ptr(), grad.data_ptr())
    stream = api.current_stream(saved.device)
    if workspace is None:
        st = F.fr_render_backward(*args, stream)
    else:
        st = F.fr_render_backward_ws(*args, workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                     stream)
    F.check(st)
    return grad
