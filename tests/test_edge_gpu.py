"""Edge and degenerate cases of the forward path on the GPU: a scene with a
closed-form answer (c = 0: the unit ball), scenes where nothing or everything
is hit, the camera inside the bounding sphere, rays parallel to the cut plane,
extreme caps, extreme image shapes and the largest image the ABI accepts."""
import math
import os

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def api():
    import torch

    assert torch.cuda.is_available()
    from paper_2102_01747_gb300 import api as A
    from paper_2102_01747_gb300 import build as B

    B.build()
    return A


def gpu(api, scene, **kw):
    import torch

    out = api.render(scene, rgba8=True, depth=True, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().reshape(-1) if k != "stats" else v.cpu().numpy() for k, v in out.items()}


def check(api, orc, scene):
    g = gpu(api, scene)
    o = orc.render(scene, precision="f32", threads=THREADS)
    res = compare(g["rgba8"], g["depth"], o["rgba8"], o["depth"])
    assert res["ok"], res
    return res, g, o


@pytest.mark.parametrize("p", [2, 3])
def test_c_zero_is_the_unit_sphere(api, orc, p):
    """c = 0: the slice of the Julia set is the unit sphere; every depth is the
    ray's entry into it, short by less than about 2 eps / cos (the DE there is half
    the distance), written out here from the ray-sphere quadratic."""
    s = W.julia_256(96, 72)
    s.update(c=(0.0, 0.0, 0.0, 0.0), p=p, max_iter=30, escape_r2=16.0 if p == 2 else 256.0)
    g = gpu(api, s)
    n_hit = 0
    for idx in range(0, 96 * 72, 7):
        ro, rd = orc.camera_ray(s, idx % 96, idx // 96)
        b = ro @ rd
        disc = b * b - (ro @ ro - 1.0)
        if disc < 0.02:
            continue
        t_sphere = -b - math.sqrt(disc)
        assert -1e-5 <= t_sphere - g["depth"][idx] <= 2.5 * s["eps"] / math.sqrt(disc) + 1e-5, idx
        n_hit += 1
    assert n_hit > 200


def test_camera_facing_away_hits_nothing(api, orc):
    s = W.bulb_1080p(10, 120, 80)
    eye = np.array(s["camera"]["eye"])
    s["camera"]["target"] = tuple(2 * eye)  # looking away from the bounding sphere
    g = gpu(api, s, stats=True)
    assert np.all(g["depth"] == np.inf) and np.all(g["rgba8"] == 0)
    assert g["stats"][2] == 0 and g["stats"][5] == 0  # no DE call, no orbit step
    check(api, orc, s)


def test_camera_inside_the_bounding_sphere(api, orc):
    s = W.bulb_1080p(10, 160, 100)
    s["camera"]["eye"] = (0.3, 1.1, 1.2)  # |eye| < 2: the interval starts at eps
    res, _, _ = check(api, orc, s)
    assert res["hits"] > 1000


def test_rays_parallel_to_the_cut_plane(api, orc):
    """Odd width: the centre column's rays have rd.z = 0 (exactly in the oracle's
    camera, within rounding in the kernel's), parallel to the plane z = o.  With
    the eye on the kept side they march; with the eye on the removed side they
    miss, whichever side of zero rd.z falls."""
    for o_plane, expect_hits in ((0.05, True), (-0.05, False)):
        s = W.julia_256(101, 61)
        s["camera"]["eye"] = (3.0, 0.0, 0.0)
        s["plane"] = {"n": (0.0, 0.0, 1.0), "o": o_plane}
        res, g, o = check(api, orc, s)
        col = np.arange(61) * 101 + 50
        assert np.array_equal(np.isfinite(g["depth"][col]), np.isfinite(o["depth"][col]))
        assert np.any(np.isfinite(g["depth"][col])) == expect_hits


@pytest.mark.parametrize("kw", [dict(max_steps=1), dict(max_iter=1), dict(eps=0.1), dict(max_step=0.01),
                                dict(max_steps=2000, eps=1e-5)])
@pytest.mark.parametrize("kind", ["julia", "bulb"])
def test_extreme_caps(api, orc, kind, kw):
    s = W.julia_256(90, 70) if kind == "julia" else W.bulb_1080p(10, 96, 64)
    s.update(kw)
    check(api, orc, s)


@pytest.mark.parametrize("w,h", [(65535, 2), (3, 65535)])
def test_extreme_shapes(api, orc, w, h):
    """The widest and tallest images the ABI takes: every 97th pixel plus the
    corners against the oracle."""
    s = W.julia_256(w, h)
    g = gpu(api, s)
    px = np.unique(np.r_[np.arange(0, w * h, 97), [0, w - 1, w * (h - 1), w * h - 1]])
    o = orc.render(s, pixels=px, precision="f32", threads=THREADS)
    res = compare(g["rgba8"][px], g["depth"][px], o["rgba8"], o["depth"])
    assert res["ok"], res


@pytest.mark.parametrize("path", ["plain", "lanes", "single_via_batch_kernel", "batch_kernel", "batch_refill",
                                  "batch_persistent"])
def test_largest_image(api, orc, path):
    """46340 x 46340 = 2,147,395,600 pixels, just under the 2^31 limit of
    width*height*spp (its padded 4 x 8 tiles hold more than 2^31 pixel slots):
    17 GB of outputs; sampled pixels (random, the last row and column, the
    corners) against the oracle, gathered on the device.  Every kernel that
    renders a single image runs it."""
    import torch

    from paper_2102_01747_gb300 import _ffi as F

    w = h = 46340
    s = W.julia_256(w, h)
    old = F.fr_get_tuning()
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.single_kernel = {"lanes": 1, "single_via_batch_kernel": 2}.get(path, 0)
    t.batch_kernel = {"batch_persistent": 0, "batch_refill": 2}.get(path, 1)
    assert F.fr_set_tuning(t) == F.FR_OK
    try:
        if path.startswith("batch_"):
            out = api.render_batch([s], rgba8=True, depth=True)[0]
        else:
            out = api.render(s, rgba8=True, depth=True)
        torch.cuda.synchronize()
    finally:
        F.fr_set_tuning(old)
    rng = np.random.default_rng(3)
    px = np.unique(np.r_[rng.integers(0, w * h, 4000), (h - 1) * w + np.arange(0, w, 997),
                         np.arange(0, h, 997) * w + (w - 1), [0, w - 1, (h - 1) * w, w * h - 1]])
    idx = torch.from_numpy(px).to("cuda")
    r8 = out["rgba8"].reshape(-1).index_select(0, idx).cpu().numpy()
    dp = out["depth"].reshape(-1).index_select(0, idx).cpu().numpy()
    del out
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    o = orc.render(s, pixels=px, precision="f32", threads=THREADS)
    res = compare(r8, dp, o["rgba8"], o["depth"])
    assert res["ok"], res
    assert res["hits"] > 100
