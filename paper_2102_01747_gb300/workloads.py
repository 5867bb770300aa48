"""Seeded synthetic scenes for the renders, the parity tests and the benchmark.

This module only describes inputs: fractal parameters, camera placement,
light and image size, drawn from numpy's PCG64 with a fixed seed.  It holds
none of the rendering arithmetic, so both the CUDA path and the CPU oracle
can be fed from it.  A scene is a plain dict:

    {"kind": "julia" | "bulb",
     "c": (4,), "p": 2, "slice_w": 0.0, "escape_r2": 16.0,   # quaternion Julia
     "n": 8, "bailout": 2.0,                                  # Mandelbulb
     "max_iter": 11, "bound_radius": 2.0, "max_steps": 200, "eps": 1e-3,
     "max_step": 0.2, "normal_mode": "central" | "tetra", "normal_h": 1e-4,
     "plane": None | {"n": (3,), "o": float},     # keep dot(n, x) <= o
     "camera": {"eye", "target", "up", "fov_y_deg", "width", "height", "spp", "seed"},
     "light": {"dir", "albedo", "k_ambient", "k_diffuse", "shadows", "background",
               # optional closest-hit model (default "lambert"):
               "shading": "lambert" | "phong", "k_specular", "shininess", "reflect_coef"}}

The fixed workloads are the ones the renderer is measured on:
  julia_256           quaternion Julia q^2 + c, c = (-0.2, 0.6, 0.2, 0), 256x256
  bulb_1080p          Mandelbulb n = 8, 1920x1080, shadow ray, cut plane z = 0.1
  batch_mixed         64 requests, sides log-uniform in [128, 2048], half Julia
                      (random c in the 4-ball of radius 0.8, random cut plane through
                      the origin), half Mandelbulb (n in 2..10, 8..16 iterations)
  diff_julia          512x512 Julia with a hidden c* for gradient recovery
  stress_bulb_4k      Mandelbulb n = 8, 3840x2160, 4 jittered samples, iteration cap 4..20
  stress_julia_4k     Julia (julia_256 parameters) at 3840x2160 with shadow rays
  phong(scene)        the same scene lit by Phong + one Fresnel-weighted reflection
                      bounce (the paper's closest-hit model) over a sky-blue background
"""
from __future__ import annotations

import copy
import math

import numpy as np

BASE_SEED = 2102

DEFAULT_LIGHT = {
    "dir": (0.577, 0.577, 0.577),
    "albedo": (0.9, 0.75, 0.6),
    "k_ambient": 0.1,
    "k_diffuse": 0.9,
    "shadows": False,
    "background": (0.0, 0.0, 0.0, 0.0),
}


def _camera(eye, width, height, fov=45.0, spp=1, seed=0, target=(0.0, 0.0, 0.0)):
    return {
        "eye": tuple(float(v) for v in eye),
        "target": tuple(float(v) for v in target),
        "up": (0.0, 1.0, 0.0),
        "fov_y_deg": float(fov),
        "width": int(width),
        "height": int(height),
        "spp": int(spp),
        "seed": int(seed),
    }


def orbit_eye(radius: float, frame: float, elevation_deg: float = 20.0, step_deg: float = 3.0):
    """Camera position on a circular orbit: azimuth step_deg * frame, fixed elevation."""
    th = math.radians(step_deg * frame)
    el = math.radians(elevation_deg)
    return (radius * math.sin(th) * math.cos(el), radius * math.sin(el),
            radius * math.cos(th) * math.cos(el))


def julia_256(width: int = 256, height: int = 256) -> dict:
    """Quaternion Julia q^2 + c, c = (-0.2, 0.6, 0.2, 0), slice w = 0, 11 iterations,
    escape |q|^2 > 16, bounding radius 2, 200 steps, eps 1e-3, central-difference
    normals with h = 1e-4, camera at distance 3 on +z, FOV 45 degrees, no cut, no shadow."""
    return {
        "kind": "julia",
        "c": (-0.2, 0.6, 0.2, 0.0), "p": 2, "slice_w": 0.0, "escape_r2": 16.0,
        "n": 8, "bailout": 2.0,
        "max_iter": 11, "bound_radius": 2.0, "max_steps": 200, "eps": 1e-3, "max_step": 0.2,
        "normal_mode": "central", "normal_h": 1e-4,
        "plane": None,
        "camera": _camera((0.0, 0.0, 3.0), width, height),
        "light": dict(DEFAULT_LIGHT),
    }


def bulb_1080p(frame: int = 10, width: int = 1920, height: int = 1080) -> dict:
    """Mandelbulb n = 8, 12 iterations, bailout 2, 256 steps, eps 5e-4, tetrahedral
    normals, one shadow ray per hit, cut plane z = 0.1 (points with z > 0.1 removed),
    camera orbiting at radius 2.5 (frame k: azimuth 3k degrees, elevation 20 degrees)."""
    light = dict(DEFAULT_LIGHT)
    light["shadows"] = True
    return {
        "kind": "bulb",
        "c": (0.0, 0.0, 0.0, 0.0), "p": 2, "slice_w": 0.0, "escape_r2": 16.0,
        "n": 8, "bailout": 2.0,
        "max_iter": 12, "bound_radius": 2.0, "max_steps": 256, "eps": 5e-4, "max_step": 0.2,
        "normal_mode": "tetra", "normal_h": 0.0,
        "plane": {"n": (0.0, 0.0, 1.0), "o": 0.1},
        "camera": _camera(orbit_eye(2.5, frame), width, height),
        "light": light,
    }


def resized(scene: dict, width: int, height: int) -> dict:
    """Copy of `scene` at another image size (same camera and parameters)."""
    s = copy.deepcopy(scene)
    s["camera"]["width"] = int(width)
    s["camera"]["height"] = int(height)
    return s


def _unit(rng) -> np.ndarray:
    g = rng.standard_normal(3)
    return g / np.linalg.norm(g)


def random_julia_c(rng, radius: float = 0.8) -> tuple:
    """Uniform point of the 4-ball of the given radius."""
    g = rng.standard_normal(4)
    r = radius * rng.uniform() ** 0.25
    return tuple(float(v) for v in r * g / np.linalg.norm(g))


def batch_mixed(seed: int = BASE_SEED, n_requests: int = 64, min_log2: float = 7.0,
                max_log2: float = 11.0) -> list:
    """Mixed batch: even indices Julia, odd indices Mandelbulb, square images whose
    side is 2^U(min_log2, max_log2) rounded to a multiple of 8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_requests):
        side = int(round(2.0 ** rng.uniform(min_log2, max_log2) / 8.0)) * 8
        side = max(8, side)
        az = float(rng.uniform(0.0, 360.0))
        if i % 2 == 0:
            s = julia_256(side, side)
            s["c"] = random_julia_c(rng)
            s["plane"] = {"n": tuple(float(v) for v in _unit(rng)), "o": 0.0}
            s["camera"] = _camera(orbit_eye(3.0, az, 20.0, 1.0), side, side)
        else:
            s = bulb_1080p(0, side, side)
            s["n"] = int(rng.integers(2, 11))
            s["max_iter"] = int(rng.integers(8, 17))
            s["camera"] = _camera(orbit_eye(2.5, az, 20.0, 1.0), side, side)
        s["camera"]["seed"] = i
        out.append(s)
    return out


def diff_julia(seed: int = BASE_SEED, width: int = 512, height: int = 512):
    """Differentiable Julia workload.  Returns (target_scene, start_c): the target uses
    a hidden c* with |c*| < 0.8; the optimisation starts from c* + delta, |delta| = 0.1.
    A tilted cut plane gives both fractal-surface and cut-face pixels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = julia_256(width, height)
    base = np.array([-0.2, 0.6, 0.2, 0.0])
    c_star = base + 0.1 * rng.standard_normal(4)
    if np.linalg.norm(c_star) >= 0.8:
        c_star *= 0.79 / np.linalg.norm(c_star)
    delta = rng.standard_normal(4)
    delta *= 0.1 / np.linalg.norm(delta)
    s["c"] = tuple(float(v) for v in c_star)
    s["plane"] = {"n": (0.25, 0.15, 1.0), "o": 0.5}
    s["camera"] = _camera((0.9, 0.7, 2.7), width, height)
    s["light"]["dir"] = (0.5, 0.7, 0.6)
    start = tuple(float(v) for v in c_star + delta)
    return s, start


def stress_bulb_4k(frame: int = 60, width: int = 3840, height: int = 2160, spp: int = 4) -> dict:
    """Mandelbulb n = 8 at 3840x2160 with 4 jittered samples; the iteration cap is
    4 + floor(16 k / 119) for frame k of 120 (4..20), camera at azimuth 3k degrees."""
    s = bulb_1080p(frame, width, height)
    s["max_iter"] = 4 + (16 * frame) // 119
    s["camera"]["spp"] = spp
    s["camera"]["seed"] = frame
    return s


def stress_julia_4k(width: int = 3840, height: int = 2160) -> dict:
    """Quaternion Julia (julia_256 parameters) at 3840x2160 with one shadow ray per hit."""
    s = julia_256(width, height)
    s["light"]["shadows"] = True
    return s


PHONG_LIGHT = {
    "shading": "phong",
    "k_specular": 0.5,
    "shininess": 32.0,
    "reflect_coef": 0.1,  # the closest-hit listing's reflection weight
    "background": (0.25, 0.35, 0.5, 1.0),
}


def phong(scene: dict, **light) -> dict:
    """A copy of `scene` shaded with the Phong + reflection model (white highlight
    k_specular 0.5, exponent 32, reflection weight 0.1, sky-blue background);
    keyword arguments override those light fields."""
    s = copy.deepcopy(scene)
    s["light"].update(PHONG_LIGHT)
    s["light"].update(light)
    return s


def total_pixels(scenes) -> int:
    return sum(s["camera"]["width"] * s["camera"]["height"] for s in scenes)
