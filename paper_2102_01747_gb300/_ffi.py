"""ctypes mirror of include/fr.h and the loader of libfr.so.

Argument marshalling only: every step of the render runs in the CUDA kernels
of libfr.so.  The library is loaded on first use; if it has not been built the
call raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_uint32, c_float, c_void_p = ctypes.c_int32, ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p

FR_OK, FR_EINVAL, FR_ECUDA, FR_ETIMEOUT, FR_ENOMEM, FR_ENOTIMPL = range(6)
FR_KIND_JULIA, FR_KIND_BULB = 0, 1
FR_NORMAL_TETRA, FR_NORMAL_CENTRAL, FR_NORMAL_ANALYTIC = 0, 1, 2
FR_SHADE_LAMBERT, FR_SHADE_PHONG = 0, 1
(FR_STAT_PRIMARY_RAYS, FR_STAT_SHADOW_RAYS, FR_STAT_PRIMARY_DE, FR_STAT_NORMAL_DE,
 FR_STAT_SHADOW_DE, FR_STAT_ORBIT_ITERS, FR_STAT_REFLECT_RAYS, FR_STAT_REFLECT_DE,
 FR_NSTATS) = range(9)
STATUS_NAMES = {0: "FR_OK", 1: "FR_EINVAL", 2: "FR_ECUDA", 3: "FR_ETIMEOUT", 4: "FR_ENOMEM",
                5: "FR_ENOTIMPL"}


class fr_camera(ctypes.Structure):
    _fields_ = [("eye", c_float * 3), ("target", c_float * 3), ("up", c_float * 3),
                ("fov_y_deg", c_float), ("width", c_int32), ("height", c_int32), ("spp", c_int32),
                ("seed", c_uint32)]


class fr_light(ctypes.Structure):
    _fields_ = [("dir", c_float * 3), ("albedo", c_float * 3), ("k_ambient", c_float),
                ("k_diffuse", c_float), ("shadows", c_int32), ("background", c_float * 4),
                ("shading", c_int32), ("k_specular", c_float), ("shininess", c_float),
                ("reflect_coef", c_float)]


class fr_plane(ctypes.Structure):
    _fields_ = [("enabled", c_int32), ("n", c_float * 3), ("offset", c_float)]


class fr_julia_params(ctypes.Structure):
    _fields_ = [("c", c_float * 4), ("p", c_int32), ("slice_w", c_float), ("max_iter", c_int32),
                ("escape_r2", c_float), ("bound_radius", c_float), ("max_steps", c_int32),
                ("eps", c_float), ("max_step", c_float), ("normal_mode", c_int32),
                ("normal_h", c_float)]


class fr_bulb_params(ctypes.Structure):
    _fields_ = [("n", c_int32), ("max_iter", c_int32), ("bailout", c_float),
                ("bound_radius", c_float), ("max_steps", c_int32), ("eps", c_float),
                ("max_step", c_float), ("normal_mode", c_int32), ("normal_h", c_float),
                ("algebraic", c_int32)]


class fr_image(ctypes.Structure):
    _fields_ = [("rgba8", c_void_p), ("rgba", c_void_p), ("depth", c_void_p), ("saved", c_void_p),
                ("stats", c_void_p), ("trap", c_void_p)]


class fr_request(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("julia", fr_julia_params), ("bulb", fr_bulb_params),
                ("plane", fr_plane), ("camera", fr_camera), ("light", fr_light), ("out", fr_image)]


class fr_tuning(ctypes.Structure):
    _fields_ = [("plain_block", c_int32), ("plain_unroll", c_int32), ("persist_block", c_int32),
                ("persist_ctas_per_sm", c_int32), ("refill_threshold", c_int32),
                ("persist_unroll", c_int32), ("single_kernel", c_int32), ("batch_kernel", c_int32),
                ("tile_order", c_int32), ("sample_lanes", c_int32)]


# every entry point of include/fr.h with its ctypes signature
SIGNATURES = {
    "fr_render_julia": (c_int32, [ctypes.POINTER(fr_julia_params), ctypes.POINTER(fr_plane),
                                  ctypes.POINTER(fr_camera), ctypes.POINTER(fr_light),
                                  ctypes.POINTER(fr_image), c_void_p]),
    "fr_render_mandelbulb": (c_int32, [ctypes.POINTER(fr_bulb_params), ctypes.POINTER(fr_plane),
                                       ctypes.POINTER(fr_camera), ctypes.POINTER(fr_light),
                                       ctypes.POINTER(fr_image), c_void_p]),
    "fr_batch_workspace_bytes": (ctypes.c_size_t, [c_int32]),
    "fr_render_batch": (c_int32, [ctypes.POINTER(fr_request), c_int32, c_void_p, ctypes.c_size_t,
                                  c_void_p]),
    "fr_render_batch_static": (c_int32, [ctypes.POINTER(fr_request), c_int32, c_void_p]),
    "fr_render_backward": (c_int32, [ctypes.POINTER(fr_julia_params), ctypes.POINTER(fr_plane),
                                     ctypes.POINTER(fr_camera), ctypes.POINTER(fr_light), c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "fr_backward_workspace_bytes": (ctypes.c_size_t, []),
    "fr_render_backward_mandelbulb": (c_int32, [ctypes.POINTER(fr_bulb_params), ctypes.POINTER(fr_plane),
                                                ctypes.POINTER(fr_camera), ctypes.POINTER(fr_light), c_void_p,
                                                c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                                c_void_p]),
    "fr_render_backward_ws": (c_int32, [ctypes.POINTER(fr_julia_params), ctypes.POINTER(fr_plane),
                                        ctypes.POINTER(fr_camera), ctypes.POINTER(fr_light), c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                        c_void_p]),
    "fr_ffma_probe": (c_int32, [c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "fr_ffma_probe_flops": (ctypes.c_double, [c_int32, c_int32, c_int32]),
    "fr_get_tuning": (c_int32, [ctypes.POINTER(fr_tuning)]),
    "fr_set_tuning": (c_int32, [ctypes.POINTER(fr_tuning)]),
    "fr_last_error": (ctypes.c_char_p, []),
    "fr_abi_version": (c_int32, []),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libfr.so (built by paper_2102_01747_gb300.build / __graft_entry__.build()).
    Raises RuntimeError when it is missing: there is no other implementation."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                "libfr.so is not built (%s); run `python -m paper_2102_01747_gb300.build`" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FrError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def check(status: int):
    if status != FR_OK:
        raise FrError(status, load().fr_last_error().decode())
    return status


# thin same-name wrappers around the C entry points ---------------------------

def fr_render_julia(params, plane, camera, light, image, stream=None):
    return load().fr_render_julia(ctypes.byref(params), ctypes.byref(plane) if plane else None,
                                  ctypes.byref(camera), ctypes.byref(light), ctypes.byref(image),
                                  stream)


def fr_render_mandelbulb(params, plane, camera, light, image, stream=None):
    return load().fr_render_mandelbulb(ctypes.byref(params), ctypes.byref(plane) if plane else None,
                                       ctypes.byref(camera), ctypes.byref(light),
                                       ctypes.byref(image), stream)


def fr_batch_workspace_bytes(n_reqs):
    return load().fr_batch_workspace_bytes(int(n_reqs))


def fr_render_batch(reqs, n_reqs, workspace, ws_bytes, stream=None):
    return load().fr_render_batch(reqs, int(n_reqs), workspace, int(ws_bytes), stream)


def fr_render_batch_static(reqs, n_reqs, stream=None):
    return load().fr_render_batch_static(reqs, int(n_reqs), stream)


def fr_render_backward(params, plane, camera, light, saved, d_rgba, d_depth, grad, stream=None):
    return load().fr_render_backward(ctypes.byref(params), ctypes.byref(plane) if plane else None,
                                     ctypes.byref(camera), ctypes.byref(light), saved, d_rgba,
                                     d_depth, grad, stream)


def fr_backward_workspace_bytes():
    return load().fr_backward_workspace_bytes()


def fr_render_backward_ws(params, plane, camera, light, saved, d_rgba, d_depth, grad, workspace, ws_bytes,
                          stream=None):
    return load().fr_render_backward_ws(ctypes.byref(params), ctypes.byref(plane) if plane else None,
                                        ctypes.byref(camera), ctypes.byref(light), saved, d_rgba,
                                        d_depth, grad, workspace, int(ws_bytes), stream)


def fr_render_backward_mandelbulb(params, plane, camera, light, saved, d_rgba, d_depth, grad, workspace=None,
                                  ws_bytes=0, stream=None):
    return load().fr_render_backward_mandelbulb(ctypes.byref(params), ctypes.byref(plane) if plane else None,
                                                ctypes.byref(camera), ctypes.byref(light), saved, d_rgba,
                                                d_depth, grad, workspace, int(ws_bytes), stream)


def fr_ffma_probe(blocks, threads, iters, sink, stream=None):
    return load().fr_ffma_probe(int(blocks), int(threads), int(iters), sink, stream)


def fr_ffma_probe_flops(blocks, threads, iters) -> float:
    return float(load().fr_ffma_probe_flops(int(blocks), int(threads), int(iters)))


def fr_get_tuning():
    t = fr_tuning()
    check(load().fr_get_tuning(ctypes.byref(t)))
    return t


def fr_set_tuning(t):
    return load().fr_set_tuning(ctypes.byref(t))


def fr_last_error() -> str:
    return load().fr_last_error().decode()


def fr_abi_version() -> int:
    return load().fr_abi_version()
