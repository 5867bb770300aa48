"""The two layouts of a pixel's samples in the one-ray-per-thread kernels
(fr_tuning.sample_lanes): every sample of a pixel in turn on one lane, or the
spp samples on spp adjacent lanes, folded into the pixel's first lane in sample
order.  They must give the same bits for every output (packed and float
colour, depth, saved state, orbit trap, counters), for both fractals, the
Phong model and the analytic normal, through the single-request kernel, the
batch kernel with one request (single_kernel 2) and fr_render_batch, on
ragged image sizes; and the sample-lane renders must match the oracle."""
import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    assert torch.cuda.is_available()
    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api
    from paper_2102_01747_gb300 import build as B

    B.build()
    F.load()
    return torch, F, api


def _tuned(F, **kw):
    old = F.fr_get_tuning()
    keep = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    for k, v in kw.items():
        setattr(t, k, v)
    assert F.fr_set_tuning(t) == F.FR_OK
    return keep


# the counters switch the launch to the counting instantiation, so they are taken
# in a render of their own
OUTS = dict(rgba8=True, rgba=True, depth=True, saved=True, trap=True)
COUNTS = dict(rgba8=False, depth=False, stats=True)


def _scene(case, spp):
    if case == "bulb":
        s = W.bulb_1080p(12, 37, 29)
    elif case == "julia_shadow":
        s = W.stress_julia_4k(41, 27)
    elif case == "bulb_phong":
        s = W.phong(W.bulb_1080p(14, 33, 26))
    elif case == "bulb_analytic":
        s = dict(W.bulb_1080p(16, 35, 22), normal_mode="analytic")
    else:  # julia_analytic_cut
        s, _ = W.diff_julia(W.BASE_SEED, 39, 30)
        s["normal_mode"] = "analytic"
    s["camera"]["spp"], s["camera"]["seed"] = spp, 11
    return s


def _render(torch, api, scene, single_kernel, F):
    keep = _tuned(F, single_kernel=single_kernel)
    try:
        out = dict(api.render(scene, **OUTS))
        out.update(api.render(scene, **COUNTS))
        torch.cuda.synchronize()
    finally:
        F.fr_set_tuning(keep)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("spp", [2, 4, 8, 3])
@pytest.mark.parametrize("case", ["bulb", "julia_shadow", "bulb_phong", "bulb_analytic", "julia_analytic_cut"])
def test_sample_layouts_same_bits(mods, case, spp):
    torch, F, api = mods
    s = _scene(case, spp)
    results = {}
    for lanes in (0, 1):
        keep = _tuned(F, sample_lanes=lanes)
        try:
            for single in (0, 2):
                results[(lanes, single)] = _render(torch, api, s, single, F)
        finally:
            F.fr_set_tuning(keep)
    ref = results[(0, 0)]
    for key, r in results.items():
        for k in list(OUTS) + ["stats"]:
            assert np.array_equal(r[k].view(np.uint8), ref[k].view(np.uint8)), (key, k)


@pytest.mark.parametrize("batch_kernel", [1, 2, 0])
def test_sample_layouts_in_a_batch(mods, batch_kernel):
    """A batch mixing spp 1, 2, 4, 8 and 3 on ragged sizes: with sample lanes
    on, fr_render_batch gives the bits of single requests rendered with them off."""
    torch, F, api = mods
    scenes = W.batch_mixed(seed=29, n_requests=10, min_log2=4.3, max_log2=6.2)
    for i, s in enumerate(scenes):
        s["camera"]["spp"] = (1, 2, 4, 8, 3)[i % 5]
        s["camera"]["width"] += i % 3  # ragged widths (quad stores off for some)
    keep = _tuned(F, sample_lanes=0)
    try:
        refs = []
        for s in scenes:
            o = api.render(s, rgba8=True, depth=True, rgba=True)
            torch.cuda.synchronize()
            refs.append({k: v.cpu().numpy() for k, v in o.items()})
    finally:
        F.fr_set_tuning(keep)
    keep = _tuned(F, sample_lanes=1, batch_kernel=batch_kernel)
    try:
        outs = api.render_batch(scenes, rgba8=True, depth=True, rgba=True)
        torch.cuda.synchronize()
    finally:
        F.fr_set_tuning(keep)
    for i, (o, r) in enumerate(zip(outs, refs)):
        for k in r:
            assert np.array_equal(o[k].cpu().numpy().view(np.uint8), r[k].view(np.uint8)), (i, k)


@pytest.mark.parametrize("spp", [2, 4, 8])
def test_sample_lanes_match_oracle(mods, orc, spp):
    torch, F, api = mods
    s = W.bulb_1080p(20, 72, 40)
    s["camera"]["spp"], s["camera"]["seed"] = spp, 7
    keep = _tuned(F, sample_lanes=1, single_kernel=0)
    try:
        g = api.render(s, rgba8=True, depth=True)
        torch.cuda.synchronize()
    finally:
        F.fr_set_tuning(keep)
    o = orc.render(s, precision="f32", threads=8)
    res = compare(g["rgba8"].cpu().numpy().reshape(-1), g["depth"].cpu().numpy().reshape(-1), o["rgba8"],
                  o["depth"])
    assert res["ok"], res
