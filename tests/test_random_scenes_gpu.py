"""Randomised parity: seeded random scenes across the parameter space the ABI
accepts (degree, power, caps, escape radius, slice, cut plane, stencil,
camera, samples, light, shadows, shading model, trig-free power), rendered by
the single-request kernel and by the batch call (both schedules) and compared
with the float oracle pixel by pixel."""
import math
import os

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 8


def random_scene(rng):
    julia = rng.random() < 0.5
    s = W.julia_256(int(rng.integers(24, 72)), int(rng.integers(20, 60))) if julia else \
        W.bulb_1080p(0, int(rng.integers(24, 72)), int(rng.integers(20, 60)))
    if julia:
        v = rng.standard_normal(4)
        s["c"] = tuple(v / np.linalg.norm(v) * rng.uniform(0.1, 0.85))
        s["p"] = int(rng.choice([2, 3]))
        s["escape_r2"] = float(rng.choice([16.0, 64.0, 256.0]))
        s["slice_w"] = float(rng.uniform(-0.3, 0.3))
        s["normal_mode"] = str(rng.choice(["tetra", "central", "analytic"]))
    else:
        s["n"] = int(rng.integers(2, 17))
        s["bailout"] = float(rng.uniform(1.5, 3.0))
        s["algebraic"] = bool(rng.random() < 0.3)
        s["normal_mode"] = str(rng.choice(["tetra", "central", "analytic"]))
    s["max_iter"] = int(rng.integers(3, 16))
    s["max_steps"] = int(rng.integers(40, 300))
    s["eps"] = float(10 ** rng.uniform(-3.3, -2.3))
    s["max_step"] = float(rng.uniform(0.08, 0.3))
    s["normal_h"] = 0.0 if rng.random() < 0.5 else float(10 ** rng.uniform(-4, -2.5))
    if rng.random() < 0.5:
        nrm = rng.standard_normal(3)
        s["plane"] = {"n": tuple(nrm), "o": float(rng.uniform(-0.3, 0.3))}
    else:
        s["plane"] = None
    theta, phi = rng.uniform(0, 2 * math.pi), rng.uniform(-1.2, 1.2)
    r = rng.uniform(2.6, 3.6)
    s["camera"]["eye"] = (r * math.cos(phi) * math.sin(theta), r * math.sin(phi), r * math.cos(phi) * math.cos(theta))
    s["camera"]["target"] = tuple(rng.uniform(-0.2, 0.2, 3))
    s["camera"]["fov_y_deg"] = float(rng.uniform(25, 70))
    s["camera"]["spp"] = int(rng.choice([1, 1, 2, 3]))
    s["camera"]["seed"] = int(rng.integers(0, 1000))
    li = s["light"]
    d = rng.standard_normal(3)
    li["dir"] = tuple(d)
    li["shadows"] = bool(rng.random() < 0.5)
    li["albedo"] = tuple(rng.uniform(0.3, 1.0, 3))
    li["k_ambient"], li["k_diffuse"] = float(rng.uniform(0.05, 0.3)), float(rng.uniform(0.5, 1.0))
    li["background"] = tuple(rng.uniform(0, 1, 3)) + (float(rng.choice([0.0, 1.0])),)
    if rng.random() < 0.35:
        li.update(shading="phong", k_specular=float(rng.uniform(0, 1)), shininess=float(rng.uniform(2, 64)),
                  reflect_coef=float(rng.uniform(0, 1)))
    return s


SCENES = [random_scene(np.random.default_rng(1000 + i)) for i in range(40)]


@pytest.fixture(scope="module")
def api():
    import torch

    assert torch.cuda.is_available()
    from paper_2102_01747_gb300 import api as A
    from paper_2102_01747_gb300 import build as B

    B.build()
    return A


def _np(t):
    return t.cpu().numpy().reshape(-1)


@pytest.mark.parametrize("i", range(len(SCENES)))
def test_random_scene_matches_oracle(api, orc, i):
    import torch

    s = SCENES[i]
    out = api.render(s, rgba8=True, depth=True)
    torch.cuda.synchronize()
    o = orc.render(s, precision="f32", threads=THREADS)
    res = compare(_np(out["rgba8"]), _np(out["depth"]), o["rgba8"], o["depth"])
    assert res["ok"], (i, res)


@pytest.mark.parametrize("batch_kernel", [1, 2, 0])
def test_random_scenes_as_one_batch(api, batch_kernel):
    """All random scenes in one fr_render_batch call give the single-request
    kernel's images bit for bit, under either schedule."""
    import torch

    from paper_2102_01747_gb300 import _ffi as F

    singles = [api.render(s, rgba8=True, depth=True) for s in SCENES]
    old = F.fr_get_tuning()
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.batch_kernel = batch_kernel
    assert F.fr_set_tuning(t) == F.FR_OK
    try:
        batch = api.render_batch(SCENES, rgba8=True, depth=True)
        torch.cuda.synchronize()
    finally:
        F.fr_set_tuning(old)
    for k, (a, b) in enumerate(zip(singles, batch)):
        assert torch.equal(a["rgba8"], b["rgba8"]) and torch.equal(a["depth"], b["depth"]), k


SWEEP = int(os.environ.get("FR_SWEEP_SCENES", "0"))


@pytest.mark.skipif(SWEEP <= 0, reason="set FR_SWEEP_SCENES=N to render N random scenes (400 in the design notes)")
def test_random_scene_sweep(api, orc):
    """FR_SWEEP_SCENES seeded random scenes (seeds 1000, 1001, ...; the first 40
    are the ones above) against the float oracle.  At least 99 % meet the
    parity bar.  On every other scene hits and depths still meet it, only the
    colour bar is missed, and the float oracle's own colours agree with the
    double oracle's to within half a percent of that bar (the scene is
    ill-conditioned in float, e.g. a sharp Phong highlight)."""
    import torch

    ok, misses = 0, []
    for i in range(SWEEP):
        s = random_scene(np.random.default_rng(1000 + i))
        out = api.render(s, rgba8=True, depth=True)
        torch.cuda.synchronize()
        o = orc.render(s, precision="f32", threads=THREADS)
        res = compare(_np(out["rgba8"]), _np(out["depth"]), o["rgba8"], o["depth"])
        if res["ok"]:
            ok += 1
            continue
        o64 = orc.render(s, precision="f64", threads=THREADS)
        ref = compare(o["rgba8"], o["depth"], o64["rgba8"], o64["depth"])
        misses.append((i, res, ref))
    print("random scenes within the parity bar: %d / %d" % (ok, SWEEP))
    for i, res, ref in misses:
        print("scene", i, "GPU vs float oracle", res, "float vs double oracle", ref)
    assert ok >= 0.99 * SWEEP, misses
    for i, res, ref in misses:
        assert res["hit_agree"] >= 0.995 and res["depth_ok"] >= 0.99, (i, res)
        assert ref["rgb_ok"] < 0.995, (i, res, ref)
