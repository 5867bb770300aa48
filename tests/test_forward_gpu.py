"""GPU forward renders (one-ray-per-thread kernel, through the C ABI) against the
CPU oracle on the same seeded scenes, pixel by pixel.

The bar (tests/parity.py): hit/miss agreement >= 99.5%, relative depth <= 1e-3
on >= 99% of common hits, RGB within 3/255 on >= 99% of pixels.  The primary
comparison is with the float oracle (same precision); the double oracle is
held to the same bar on the workload scenes."""
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

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2102_01747_gb300 import api as A
    from paper_2102_01747_gb300 import build as B

    B.build()
    return A


def gpu(api, scene, **kw):
    import torch

    out = api.render(scene, rgba8=True, depth=True, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def check(api, orc, scene, precision="f32", pixels=None):
    g = gpu(api, scene)
    o = orc.render(scene, pixels=pixels, precision=precision, threads=THREADS)
    rg, dg = g["rgba8"].reshape(-1), g["depth"].reshape(-1)
    if pixels is not None:
        rg, dg = rg[pixels], dg[pixels]
    res = compare(rg, dg, o["rgba8"], o["depth"])
    assert res["ok"], res
    return res, g, o


def test_julia_256_parity(api, orc):
    res, _, _ = check(api, orc, W.julia_256())
    assert res["hits"] > 10000
    check(api, orc, W.julia_256(), precision="f64")


def test_bulb_small_parity(api, orc):
    res, _, o = check(api, orc, W.bulb_1080p(10, 240, 135))
    assert res["hits"] > 5000
    assert ((o["flags"] & 4) > 0).sum() > 50  # some shadowed pixels


def test_bulb_1080p_full_parity(api, orc):
    s = W.bulb_1080p(10)
    res, _, _ = check(api, orc, s)
    assert res["n"] == 1920 * 1080


def test_bulb_1080p_f64_sampled(api, orc):
    s = W.bulb_1080p(10)
    rng = np.random.default_rng(0)
    px = np.unique(np.r_[rng.integers(0, 1920 * 1080, 20000), np.arange(1920),
                         1920 * 1079 + np.arange(1920), np.arange(1080) * 1920 + 1919])
    check(api, orc, s, precision="f64", pixels=px)


@pytest.mark.parametrize("w,h", [(1, 1), (37, 23), (1, 64), (64, 1), (13, 100), (250, 3)])
@pytest.mark.parametrize("kind", ["julia", "bulb"])
def test_ragged_sizes(api, orc, kind, w, h):
    s = W.julia_256(w, h) if kind == "julia" else W.bulb_1080p(10, w, h)
    check(api, orc, s)


def test_julia_cube_slice_cut_shadow_tetra(api, orc):
    """The listing's own setting: degree 3, escape |q|^2 > 256, tetrahedral
    normals; plus a nonzero slice, a cut plane and shadow rays."""
    s = W.julia_256(160, 120)
    s.update(p=3, escape_r2=256.0, max_iter=12, normal_mode="tetra", normal_h=0.0, slice_w=0.05,
             c=(-0.1, 0.55, 0.3, 0.1))
    s["plane"] = {"n": (0.2, -0.3, 1.0), "o": 0.1}
    s["light"]["shadows"] = True
    res, _, o = check(api, orc, s)
    assert ((o["flags"] & 2) > 0).sum() > 100 and res["hits"] > 2000


def test_jittered_samples(api, orc):
    s = W.bulb_1080p(20, 96, 64)
    s["camera"]["spp"] = 4
    s["camera"]["seed"] = 7
    check(api, orc, s)


@pytest.mark.parametrize("block,unroll,single,order", [(32, 1, 0, 0), (64, 2, 0, 0), (256, 4, 0, 0), (128, 1, 0, 0),
                                                      (128, 1, 0, 1), (64, 2, 0, 2), (32, 4, 0, 1), (256, 1, 0, 2),
                                                      (128, 1, 1, 0), (64, 2, 1, 0), (256, 8, 1, 0),
                                                      (128, 1, 2, 0), (64, 2, 2, 1), (256, 1, 2, 2)])
def test_launch_shapes_give_identical_images(api, block, unroll, single, order):
    from paper_2102_01747_gb300 import _ffi as F

    old = F.fr_get_tuning()
    keep = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    s = W.bulb_1080p(10, 200, 120)
    j = W.julia_256(130, 70)
    ref = (gpu(api, s), gpu(api, j))
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.plain_block, t.single_kernel, t.tile_order = block, single, order
    if single == 1:
        t.persist_unroll = unroll  # the lane state machine's Julia steps per round
    else:
        t.plain_unroll = unroll
    assert F.fr_set_tuning(t) == F.FR_OK
    try:
        for scene, r in zip((s, j), ref):
            g = gpu(api, scene)
            # every rounding step is explicit, so neither the block shape, the
            # unroll depth, the tile order nor the kernel (nested loops or lane
            # state machine) can change a single bit
            assert np.array_equal(g["rgba8"], r["rgba8"])
            assert np.array_equal(g["depth"], r["depth"])
    finally:
        F.fr_set_tuning(keep)


@pytest.mark.parametrize("order", [1, 2])
def test_tile_orders_in_batch(api, order):
    """The batch kernel under every tile order gives the single-request images
    bit for bit, on requests whose sides are not multiples of the tile."""
    import torch

    from paper_2102_01747_gb300 import _ffi as F

    scenes = [W.julia_256(130, 70), W.bulb_1080p(3, 61, 93), W.julia_256(8, 8), W.bulb_1080p(7, 257, 31)]
    singles = [gpu(api, sc) for sc in scenes]
    old = F.fr_get_tuning()
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.tile_order, t.batch_kernel = order, 1
    assert F.fr_set_tuning(t) == F.FR_OK
    try:
        outs = api.render_batch(scenes, rgba8=True, depth=True)
        torch.cuda.synchronize()
    finally:
        F.fr_set_tuning(old)
    for r, o in zip(singles, outs):
        assert np.array_equal(r["rgba8"], o["rgba8"].cpu().numpy())
        assert np.array_equal(r["depth"], o["depth"].cpu().numpy())


def test_saved_state_and_outputs(api, orc):
    import torch

    s, _ = W.diff_julia(W.BASE_SEED, 96, 80)
    out = api.render(s, rgba8=True, rgba=True, depth=True, saved=True)
    torch.cuda.synchronize()
    o = orc.render(s, precision="f32", threads=THREADS)
    saved = out["saved"].cpu().numpy().reshape(-1, 4)
    flags = saved[:, 3].view(np.uint32)
    assert np.mean(flags == o["flags"].astype(np.uint32)) >= 0.995
    hit = (flags & 1) > 0
    depth = out["depth"].cpu().numpy().reshape(-1)
    # saved hit point lies on the camera ray at the reported depth
    eye = np.array(s["camera"]["eye"])
    dist = np.linalg.norm(saved[hit, :3] - eye, axis=1)
    assert np.allclose(dist, depth[hit], rtol=1e-5, atol=1e-5)
    rgba = out["rgba"].cpu().numpy().reshape(-1, 4)
    from parity import unpack

    q = unpack(out["rgba8"].cpu().numpy().reshape(-1))
    assert np.all(np.abs(np.floor(np.clip(rgba, 0, 1) * 255 + 0.5) - q) <= 1)


@pytest.mark.parametrize("normal", ["tetra", "analytic"])
def test_stats_counters_match_oracle(api, orc, normal):
    """Work counters against the oracle's (the analytic normal counts one
    normal evaluation and one orbit per hit)."""
    s = dict(W.bulb_1080p(10, 160, 90), normal_mode=normal)
    out = api.render(s, stats=True)
    import torch

    torch.cuda.synchronize()
    st = out["stats"].cpu().numpy()
    o = orc.render(s, precision="f32", threads=THREADS)
    os_ = o["stats"].sum(0)  # primary DE, normal DE, shadow DE, orbit, shadow rays
    assert st[0] == 160 * 90
    assert abs(st[1] - os_[4]) <= 0.01 * os_[4] + 2
    for g_i, o_i in ((2, 0), (3, 1), (4, 2), (5, 3)):
        assert abs(int(st[g_i]) - int(os_[o_i])) <= 0.02 * os_[o_i] + 10, (g_i, st, os_)


def test_nondefault_stream(api, orc):
    import torch

    s = W.julia_256(64, 64)
    ref = gpu(api, s)
    strm = torch.cuda.Stream()
    with torch.cuda.stream(strm):
        out = api.render(s, rgba8=True, depth=True)
    strm.synchronize()
    assert np.array_equal(out["rgba8"].cpu().numpy(), ref["rgba8"])


@pytest.mark.parametrize("n", [8, 2, 3, 5, 9])
def test_algebraic_power_matches_oracle(api, orc, n):
    """The de Moivre evaluation of Eq. 1 (no transcendental calls) against the
    oracle's acos / atan2 / sin / cos evaluation of the same formula."""
    s = W.bulb_1080p(25, 200, 112)
    s["n"] = n
    s["algebraic"] = True
    res, _, _ = check(api, orc, s)
    assert res["hits"] > 1000


@pytest.mark.parametrize("kind", ["julia", "bulb"])
def test_orbit_trap_output(api, orc, kind):
    """The orbit-trap colour parameters at the nearest hit point against the oracle's.
    The trap is a sensitive function of the hit point (the final |w|^2 above all),
    so the bar is calibrated on the oracle itself: per component, the GPU agrees
    with the float oracle (within 1e-3 relative) about as often as the float
    oracle agrees with the double oracle."""
    import torch

    s = W.julia_256(120, 90) if kind == "julia" else W.bulb_1080p(14, 160, 90)
    out = api.render(s, rgba8=True, depth=True, trap=True)
    torch.cuda.synchronize()
    g = out["trap"].cpu().numpy().reshape(-1, 4)
    o = orc.render(s, precision="f32", threads=THREADS)
    o64 = orc.render(s, precision="f64", threads=THREADS)
    gd = out["depth"].cpu().numpy().reshape(-1)
    assert np.all(g[~np.isfinite(gd)] == 0)
    both = np.isfinite(gd) & np.isfinite(o["depth"]) & np.isfinite(o64["depth"])
    assert both.sum() > 500

    def agree(a, b):
        return np.mean(np.abs(a[both] - b[both]) <= 1e-3 * np.abs(b[both]) + 1e-6, 0)

    got, calib = agree(g, o["trap"]), agree(o["trap"], o64["trap"])
    assert np.all(got >= calib - 0.05), (got, calib)
    assert np.all(np.median(np.abs(g[both] - o["trap"][both]) / (np.abs(o["trap"][both]) + 1e-6), 0) < 1e-3)
    # both batch schedules write the same values
    from paper_2102_01747_gb300 import _ffi as F

    old = F.fr_get_tuning()
    try:
        for bk in (1, 0):
            t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
            t.batch_kernel = bk
            assert F.fr_set_tuning(t) == F.FR_OK
            b = api.render_batch([s], rgba8=True, depth=True, trap=True)[0]
            torch.cuda.synchronize()
            assert np.array_equal(b["trap"].cpu().numpy(), out["trap"].cpu().numpy()), bk
    finally:
        F.fr_set_tuning(old)


@pytest.mark.parametrize("p", [2, 3])
def test_analytic_normal_render(api, orc, p):
    """Julia renders shaded with the analytic normal (Sec. 2) against the oracle."""
    s = W.julia_256(160, 120)
    s.update(p=p, escape_r2=256.0 if p == 3 else 16.0, max_iter=11, normal_mode="analytic")
    s["light"]["shadows"] = True
    res, _, _ = check(api, orc, s)
    assert res["hits"] > 3000
    import torch

    b = api.render_batch([s], rgba8=True, depth=True)[0]
    torch.cuda.synchronize()
    g = gpu(api, s)
    assert np.array_equal(b["rgba8"].cpu().numpy(), g["rgba8"])


@pytest.mark.parametrize("n,alg", [(8, False), (8, True), (3, False), (5, False)])
def test_bulb_analytic_normal_render(api, orc, n, alg):
    """Mandelbulbs shaded with the analytic normal (J = dw/dc carried through
    Eq. 1) against the oracle, and the batch call's image bit for bit."""
    s = W.bulb_1080p(5, 200, 120)
    s.update(n=n, algebraic=alg, normal_mode="analytic")
    s["light"]["shadows"] = True
    res, _, _ = check(api, orc, s)
    assert res["hits"] > 3000
    import torch

    b = api.render_batch([s], rgba8=True, depth=True)[0]
    torch.cuda.synchronize()
    g = gpu(api, s)
    assert np.array_equal(b["rgba8"].cpu().numpy(), g["rgba8"])


@pytest.mark.parametrize("case", ["bulb", "julia_cut", "julia_analytic", "bulb_analytic", "bulb_jitter"])
def test_phong_reflection_render(api, orc, case):
    """The Phong + Fresnel-weighted mirror-ray model against the oracle's."""
    if case == "bulb":
        s = W.phong(W.bulb_1080p(12, 200, 120))
    elif case == "julia_cut":
        s = W.phong(dict(W.julia_256(160, 120), plane={"n": (0.2, 0.1, 1.0), "o": 0.1}), reflect_coef=0.6)
        s["light"]["shadows"] = True
    elif case == "julia_analytic":
        s = W.phong(dict(W.julia_256(128, 128), normal_mode="analytic"), k_specular=0.8, shininess=8.0)
    elif case == "bulb_analytic":
        s = W.phong(dict(W.bulb_1080p(8, 160, 96), normal_mode="analytic"), reflect_coef=0.7)
    else:
        s = W.phong(W.bulb_1080p(3, 96, 64), reflect_coef=1.0)
        s["camera"]["spp"], s["camera"]["seed"] = 3, 5
    res, g, o = check(api, orc, s)
    assert res["hits"] > 1000
    # the mirror rays do reach the surface somewhere (reflection DE calls and orbit work)
    assert o["stats"][:, 5].sum() > 1000


def test_phong_counters_match_oracle(api, orc):
    import torch

    s = W.phong(W.bulb_1080p(10, 160, 90))
    out = api.render(s, rgba8=False, depth=False, stats=True)
    torch.cuda.synchronize()
    st = out["stats"].cpu().numpy()
    os_ = orc.render(s, precision="f32", threads=THREADS)["stats"].sum(0)
    assert abs(int(st[6]) - int(os_[6])) <= 0.01 * os_[6] + 2  # reflection rays
    for g_i, o_i in ((2, 0), (3, 1), (4, 2), (5, 3), (7, 5)):
        assert abs(int(st[g_i]) - int(os_[o_i])) <= 0.02 * os_[o_i] + 10, (g_i, st, os_)


def test_phong_on_the_lane_kernel(api):
    """The lane state machine (single_kernel 1) runs the mirror stage and the
    Mandelbulb's analytic normal too and gives the one-ray-per-thread kernel's
    images bit for bit."""
    from paper_2102_01747_gb300 import _ffi as F

    scenes = [W.phong(W.bulb_1080p(12, 120, 72)),
              W.phong(dict(W.julia_256(96, 64), plane={"n": (0.2, 0.1, 1.0), "o": 0.1}), reflect_coef=0.6),
              dict(W.bulb_1080p(6, 120, 72), n=5, normal_mode="analytic"),
              W.phong(dict(W.bulb_1080p(9, 120, 72), normal_mode="analytic"))]
    scenes[1]["light"]["shadows"] = True
    scenes[2]["light"]["shadows"] = True
    refs = [gpu(api, s) for s in scenes]
    old = F.fr_get_tuning()
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.single_kernel = 1
    assert F.fr_set_tuning(t) == F.FR_OK
    try:
        got = [gpu(api, s) for s in scenes]
    finally:
        F.fr_set_tuning(old)
    for r, g in zip(refs, got):
        assert np.array_equal(r["rgba8"], g["rgba8"]) and np.array_equal(r["depth"], g["depth"])
