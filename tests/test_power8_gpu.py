"""The Mandelbulb of the paper's power n = 8 has single-request kernels of its
own, compiled with n a constant: Lambert and Phong shading, with a stencil
normal or the analytic normal, and the kernel with a pixel's samples on
adjacent lanes.  The batch kernels run every power through orbit loops with n
at run time, carry the analytic normal out of line, and hold both fractals.
All of them make the same products in the same order, so a power-8 request
renders to the same bits through every one of them: packed and float colour,
depth, saved state, orbit trap and counters, for both forms of Eq. 1."""
import itertools

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W

pytestmark = pytest.mark.gpu

OUTS = dict(rgba8=True, rgba=True, depth=True, saved=True, trap=True)
COUNTS = dict(rgba8=False, depth=False, stats=True)


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


def _scene(shading, normal, spp, alg):
    s = W.bulb_1080p(17, 70, 44)  # ragged: 70 is not a multiple of the 4-pixel tile width
    s["camera"]["eye"] = (0.35, 0.8, 2.3)
    if shading == "phong":
        s = W.phong(s)
    s["normal_mode"] = normal
    if normal == "central":
        s["normal_h"] = 1e-4
    s["camera"]["spp"], s["camera"]["seed"] = spp, 5
    s["algebraic"] = bool(alg)
    return s


def _host(torch, outs):
    torch.cuda.synchronize()
    return [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]


CASES = list(itertools.product(["lambert", "phong"], ["tetra", "central", "analytic"], [1, 4], [0, 1]))


@pytest.mark.parametrize("shading,normal,spp,alg", CASES)
def test_power8_kernels_equal_the_generic_batch_kernels(mods, shading, normal, spp, alg):
    torch, F, api = mods
    s = _scene(shading, normal, spp, alg)
    other = dict(s, n=5)  # a second power in the batch launch
    single = _host(torch, [dict(api.render(s, **OUTS), **api.render(s, **COUNTS))])[0]
    assert (single["rgba8"].view(np.uint32) >> 24).sum() > 0  # something was hit
    for schedule in (2, 1):
        keep = _tuned(F, batch_kernel=schedule)
        try:
            got = _host(torch, api.render_batch([other, s], **OUTS))[1]
            counted = _host(torch, api.render_batch([other, s], **COUNTS))[1]
        finally:
            F.fr_set_tuning(keep)
        for k in OUTS:
            assert np.array_equal(got[k].view(np.uint8), single[k].view(np.uint8)), (schedule, k)
        assert np.array_equal(counted["stats"], single["stats"]), schedule
