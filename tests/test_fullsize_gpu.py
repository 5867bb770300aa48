"""Parity at the measured workloads' full sizes, in the launch configuration
bench.py times (default tuning: the one-ray-per-thread kernel for single
requests, the batch kernel for the 64-request batch), on pixels sampled from
every image and traced one by one by the float oracle."""
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


def _sample(scene, k, seed):
    """k random pixels plus the four corners and the centre."""
    w, h = scene["camera"]["width"], scene["camera"]["height"]
    rng = np.random.default_rng(seed)
    fixed = [0, w - 1, (h - 1) * w, w * h - 1, (h // 2) * w + w // 2]
    return np.unique(np.r_[rng.integers(0, w * h, k), fixed]).astype(np.int64)


def _check_sampled(out, scene, px, orc):
    g8 = out["rgba8"].reshape(-1).cpu().numpy()[px]
    gd = out["depth"].reshape(-1).cpu().numpy()[px]
    o = orc.render(scene, pixels=px, precision="f32", threads=THREADS)
    res = compare(g8, gd, o["rgba8"], o["depth"])
    assert res["ok"], res
    return res


def test_batch_mixed_full_size(api, orc):
    """The 64-request mixed batch (44.6 M pixels) in one fr_render_batch call;
    1500 pixels of every request against the oracle."""
    import torch

    scenes = W.batch_mixed(W.BASE_SEED)
    outs = api.render_batch(scenes, rgba8=True, depth=True)
    torch.cuda.synchronize()
    hits = 0
    for i, (s, o) in enumerate(zip(scenes, outs)):
        hits += _check_sampled(o, s, _sample(s, 1500, i), orc)["hits"]
    assert hits > 10000


@pytest.mark.parametrize("name", ["stress_bulb_4k", "stress_julia_4k", "bulb_1080p_phong", "julia_4k_analytic",
                                  "bulb_1080p_analytic"])
def test_single_request_full_size(api, orc, name):
    import torch

    s = {"stress_bulb_4k": lambda: W.stress_bulb_4k(60), "stress_julia_4k": W.stress_julia_4k,
         "bulb_1080p_phong": lambda: W.phong(W.bulb_1080p(10)),
         "julia_4k_analytic": lambda: dict(W.stress_julia_4k(), normal_mode="analytic"),
         "bulb_1080p_analytic": lambda: dict(W.bulb_1080p(10), normal_mode="analytic")}[name]()
    out = api.render(s, rgba8=True, depth=True)
    torch.cuda.synchronize()
    res = _check_sampled(out, s, _sample(s, 20000, 7), orc)
    assert res["hits"] > 2000


def test_stress_animation_frames(api, orc):
    """Frames across the animated iteration-cap sweep (caps 4, 12 and 20), 4K x 4 spp."""
    import torch

    for k in (0, 60, 119):
        s = W.stress_bulb_4k(k)
        out = api.render(s, rgba8=True, depth=True)
        torch.cuda.synchronize()
        _check_sampled(out, s, _sample(s, 6000, k), orc)


@pytest.mark.parametrize("name", ["stress_julia_4k", "stress_bulb_4k"])
def test_tile_orders_bitwise_at_full_size(api, name):
    """The tile order the autotuner picks for the 4K workloads (columns) gives
    the row-order image bit for bit at full size."""
    import torch

    from paper_2102_01747_gb300 import _ffi as F

    s = W.stress_julia_4k() if name == "stress_julia_4k" else W.stress_bulb_4k(60)
    old = F.fr_get_tuning()
    imgs = []
    try:
        for order in (0, 1, 2):
            t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
            t.tile_order, t.single_kernel = order, 0
            assert F.fr_set_tuning(t) == F.FR_OK
            out = api.render(s, rgba8=True, depth=True)
            torch.cuda.synchronize()
            imgs.append(out)
    finally:
        F.fr_set_tuning(old)
    for o in imgs[1:]:
        assert torch.equal(o["rgba8"], imgs[0]["rgba8"]) and torch.equal(o["depth"], imgs[0]["depth"])


@pytest.mark.parametrize("name", ["bulb_1080p", "stress_bulb_4k"])
def test_single_request_kernels_bitwise_at_full_size(api, name):
    """fr_render_mandelbulb on the batch kernel (single_kernel 2, what the
    autotuner keeps for these frames) gives the single-request kernel's image
    bit for bit at full size."""
    import torch

    from paper_2102_01747_gb300 import _ffi as F

    s = W.bulb_1080p(10) if name == "bulb_1080p" else W.stress_bulb_4k(60)
    old = F.fr_get_tuning()
    imgs = []
    try:
        for sk in (0, 2):
            t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
            t.single_kernel = sk
            assert F.fr_set_tuning(t) == F.FR_OK
            out = api.render(s, rgba8=True, depth=True)
            torch.cuda.synchronize()
            imgs.append(out)
    finally:
        F.fr_set_tuning(old)
    assert torch.equal(imgs[0]["rgba8"], imgs[1]["rgba8"]) and torch.equal(imgs[0]["depth"], imgs[1]["depth"])
