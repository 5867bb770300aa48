"""Host-side checks of the C ABI: the library loads without a GPU, exports every
entry point include/fr.h declares, its ctypes mirror has the C layout, and bad
arguments are refused on the host (FR_EINVAL) before anything is launched.

Every refused call below leaves all output pointers NULL, so even a missing
check could not reach a kernel: the "no output buffer" check would still
refuse it.  The tests look at the message to see which check fired."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2102_01747_gb300 import build as B
from paper_2102_01747_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fr.h")


@pytest.fixture(scope="module")
def F():
    B.build()
    from paper_2102_01747_gb300 import _ffi

    _ffi.load()
    return _ffi


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"FR_API\s+[\w\s\*]+?\b(fr_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(F):
    names = declared_functions()
    assert len(names) >= 9
    lib = ctypes.CDLL(B.LIB)
    for n in names:
        assert hasattr(lib, n), n
        assert n in F.SIGNATURES, "binding lacks " + n
    assert F.fr_abi_version() == 3


def test_struct_layout_matches_header(F):
    """Compile a probe against fr.h with gcc and compare sizes and offsets."""
    structs = ["fr_camera", "fr_light", "fr_plane", "fr_julia_params", "fr_bulb_params",
               "fr_image", "fr_request", "fr_tuning"]
    fields = {"fr_request": ["julia", "bulb", "plane", "camera", "light", "out"],
              "fr_camera": ["fov_y_deg", "seed"], "fr_light": ["shadows", "background"],
              "fr_image": ["stats"]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fr.h"', "int main(void){"]
    for s in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fields.get(s, []):
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write("\n".join(lines))
        exe = os.path.join(d, "probe")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.split() for l in out.strip().splitlines())
    for s in structs:
        assert int(got[s]) == ctypes.sizeof(getattr(F, s)), s
        for f in fields.get(s, []):
            assert int(got[s + "." + f]) == getattr(getattr(F, s), f).offset, s + "." + f


def _structs(scene):
    from paper_2102_01747_gb300 import api

    return (api.julia_params(scene) if scene["kind"] == "julia" else api.bulb_params(scene),
            api.plane_struct(scene), api.camera_struct(scene), api.light_struct(scene))


def _call(F, scene, img=None):
    p, pl, cam, li = _structs(scene)
    img = img if img is not None else F.fr_image()
    fn = F.fr_render_julia if scene["kind"] == "julia" else F.fr_render_mandelbulb
    return fn(p, pl, cam, li, img, None), F.fr_last_error()


@pytest.mark.parametrize("mutate, needle", [
    (lambda s: s.update(p=5), "degree"),
    (lambda s: s.update(max_iter=0), "max_iter"),
    (lambda s: s.update(eps=-1.0), "eps"),
    (lambda s: s.update(max_step=0.0), "max_step"),
    (lambda s: s.update(max_steps=0), "max_steps"),
    (lambda s: s.update(escape_r2=0.0), "escape_r2"),
    (lambda s: s.update(bound_radius=float("nan")), "bound_radius"),
    (lambda s: s.update(normal_mode="bogus"), None),
    (lambda s: s["camera"].update(width=0), "empty"),
    (lambda s: s["camera"].update(spp=65), "spp"),
    (lambda s: s["camera"].update(fov_y_deg=180.0), "fov"),
    (lambda s: s["camera"].update(target=s["camera"]["eye"]), "eye equals target"),
    (lambda s: s["camera"].update(up=(0.0, 0.0, -1.0)), "parallel"),
    (lambda s: s["light"].update(dir=(0.0, 0.0, 0.0)), "light direction"),
    (lambda s: s.update(plane={"n": (0.0, 0.0, 0.0), "o": 0.0}), "plane normal"),
    (lambda s: s.update(c=(float("inf"), 0.0, 0.0, 0.0)), "not finite"),
    (lambda s: s["light"].update(shading="bogus"), None),
    (lambda s: s["light"].update(shading="phong", shininess=0.5), "shininess"),
    (lambda s: s["light"].update(shading="phong", reflect_coef=1.5), "reflect_coef"),
    (lambda s: s["light"].update(shading="phong", k_specular=-1.0), "k_specular"),
    (lambda s: s["camera"].update(width=40000, height=40000, spp=2), "2^31"),
])
def test_bad_julia_arguments_refused(F, mutate, needle):
    s = W.julia_256(16, 16)
    mutate(s)
    if s["normal_mode"] == "bogus":
        p, pl, cam, li = _structs(dict(s, normal_mode="tetra"))
        p.normal_mode = 7
        st = F.fr_render_julia(p, pl, cam, li, F.fr_image(), None)
        assert st == F.FR_EINVAL and "normal_mode" in F.fr_last_error()
        return
    if s["light"].get("shading") == "bogus":
        s["light"]["shading"] = "lambert"
        p, pl, cam, li = _structs(s)
        li.shading = 7
        st = F.fr_render_julia(p, pl, cam, li, F.fr_image(), None)
        assert st == F.FR_EINVAL and "shading" in F.fr_last_error()
        return
    st, msg = _call(F, s)
    assert st == F.FR_EINVAL
    assert needle in msg, msg


@pytest.mark.parametrize("mutate, needle", [
    (lambda s: s.update(n=1), "power"),
    (lambda s: s.update(n=17), "power"),
    (lambda s: s.update(bailout=0.0), "bailout"),
    (lambda s: s.update(max_iter=2000), "max_iter"),
])
def test_bad_bulb_arguments_refused(F, mutate, needle):
    s = W.bulb_1080p(0, 16, 16)
    mutate(s)
    st, msg = _call(F, s)
    assert st == F.FR_EINVAL and needle in msg, msg


@pytest.mark.parametrize("mode", ["tetra", "central", "analytic"])
def test_scene_normal_mode_reaches_both_param_structs(F, mode):
    """The binding carries every normal mode into both fractals' parameter
    blocks, and an unknown mode is an error rather than a silent default."""
    from paper_2102_01747_gb300 import api

    code = {"tetra": F.FR_NORMAL_TETRA, "central": F.FR_NORMAL_CENTRAL, "analytic": F.FR_NORMAL_ANALYTIC}[mode]
    assert api.julia_params(dict(W.julia_256(8, 8), normal_mode=mode)).normal_mode == code
    assert api.bulb_params(dict(W.bulb_1080p(0, 8, 8), normal_mode=mode)).normal_mode == code
    with pytest.raises(KeyError):
        api.bulb_params(dict(W.bulb_1080p(0, 8, 8), normal_mode="sobel"))


def test_no_output_refused(F):
    st, msg = _call(F, W.julia_256(16, 16))
    assert st == F.FR_EINVAL and "no output" in msg


def test_null_structs_refused(F):
    p, pl, cam, li = _structs(W.julia_256(16, 16))
    lib = F.load()
    img = F.fr_image()
    assert lib.fr_render_julia(None, None, ctypes.byref(cam), ctypes.byref(li), ctypes.byref(img), None) == F.FR_EINVAL
    assert lib.fr_render_julia(ctypes.byref(p), None, None, ctypes.byref(li), ctypes.byref(img), None) == F.FR_EINVAL
    assert lib.fr_render_julia(ctypes.byref(p), None, ctypes.byref(cam), None, ctypes.byref(img), None) == F.FR_EINVAL
    assert lib.fr_render_julia(ctypes.byref(p), None, ctypes.byref(cam), ctypes.byref(li), None, None) == F.FR_EINVAL


def test_tuning_roundtrip_and_checks(F):
    t = F.fr_get_tuning()
    old = tuple(getattr(t, n) for n, _ in F.fr_tuning._fields_)
    bad = F.fr_tuning(*old)
    bad.plain_block = 48
    assert F.fr_set_tuning(bad) == F.FR_EINVAL
    bad = F.fr_tuning(*old)
    bad.persist_unroll = 3
    assert F.fr_set_tuning(bad) == F.FR_EINVAL
    bad = F.fr_tuning(*old)
    bad.refill_threshold = 0
    assert F.fr_set_tuning(bad) == F.FR_EINVAL
    bad = F.fr_tuning(*old)
    bad.batch_kernel = 3
    assert F.fr_set_tuning(bad) == F.FR_EINVAL and "batch_kernel" in F.fr_last_error()
    for v in (-1, 3):
        bad = F.fr_tuning(*old)
        bad.tile_order = v
        assert F.fr_set_tuning(bad) == F.FR_EINVAL and "tile_order" in F.fr_last_error()
        bad = F.fr_tuning(*old)
        bad.single_kernel = v
        assert F.fr_set_tuning(bad) == F.FR_EINVAL and "single_kernel" in F.fr_last_error()
    good = F.fr_tuning(*old)
    good.plain_block = 64
    good.tile_order = 2
    good.single_kernel = 2
    assert F.fr_set_tuning(good) == F.FR_OK
    assert F.fr_get_tuning().plain_block == 64 and F.fr_get_tuning().tile_order == 2
    assert F.fr_set_tuning(F.fr_tuning(*old)) == F.FR_OK


def test_batch_grid_limit_refused_before_launch(F):
    """64 requests of 46000 x 46000 pixels with 32-thread CTAs need 4.3e9 CTAs in
    one launch of the one-ray-per-thread batch kernel: refused on the host.  The
    outputs are placeholder addresses that must never reach a kernel, so this
    runs only where there is no GPU at all."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("placeholder output addresses: host-only check")
    s = W.julia_256(46000, 46000)
    req = F.fr_request()
    req.kind = F.FR_KIND_JULIA
    req.julia, req.plane, req.camera, req.light = _structs(s)
    req.out.rgba8 = 1 << 20  # placeholder, 256-byte aligned, never dereferenced
    arr = (F.fr_request * 64)(*([req] * 64))
    old = F.fr_get_tuning()
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.batch_kernel, t.plain_block = 1, 32
    assert F.fr_set_tuning(t) == F.FR_OK
    try:
        st = F.fr_render_batch(arr, 64, 1 << 21, F.fr_batch_workspace_bytes(64), None)
        msg = F.fr_last_error()
    finally:
        F.fr_set_tuning(F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_]))
    assert st == F.FR_EINVAL and "CTAs" in msg, msg


def test_autotune_skips_knobs_of_the_other_schedule():
    from paper_2102_01747_gb300 import autotune

    assert autotune._in_use("batch_kernel", {"batch_kernel": 1})
    assert autotune._in_use("plain_block", {"batch_kernel": 1})
    assert autotune._in_use("plain_block", {"batch_kernel": 2})
    assert not autotune._in_use("refill_threshold", {"batch_kernel": 2})
    assert not autotune._in_use("refill_threshold", {"batch_kernel": 1})
    assert autotune._in_use("persist_unroll", {"batch_kernel": 0})
    assert not autotune._in_use("plain_block", {"batch_kernel": 0})


def test_autotune_descent_switches_only_beyond_the_margin(F):
    """Coordinate descent on a synthetic cost table (no GPU): a candidate
    replaces the setting only when it is more than 1 % faster, and the search
    leaves its choice applied through fr_set_tuning."""
    from paper_2102_01747_gb300 import autotune

    old = F.fr_get_tuning()
    keep = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    cost = {("plain_block", 64): 0.995, ("plain_block", 256): 0.90, ("tile_order", 1): 0.985,
            ("tile_order", 2): 1.2}
    try:
        autotune.apply({"plain_block": 128, "tile_order": 0})

        def timer():
            cur = autotune.current()
            ms = 1.0
            for (k, v), f in cost.items():
                if cur[k] == v:
                    ms *= f
            return ms

        res = autotune._descent(timer, {"plain_block": (64, 128, 256), "tile_order": (0, 1, 2)},
                                lambda k, c: True, 1, None, 0.01)
        # 64 (0.5 % faster) is not taken, 256 (10 %) is; then column order (1.5 %) is
        assert res["config"]["plain_block"] == 256 and res["config"]["tile_order"] == 1
        assert abs(res["ms"] - 0.90 * 0.985) < 1e-12
        t = F.fr_get_tuning()
        assert t.plain_block == 256 and t.tile_order == 1
    finally:
        F.fr_set_tuning(keep)


def test_backward_refuses_phong(F):
    """The adjoint covers Lambert shading; every buffer is NULL, so nothing could launch."""
    s = W.phong(W.julia_256(16, 16))
    p, pl, cam, li = _structs(s)
    st = F.fr_render_backward(p, pl, cam, li, None, None, None, None, None)
    assert st == F.FR_EINVAL and "Lambert" in F.fr_last_error(), F.fr_last_error()


def test_backward_workspace_checked_first(F):
    """fr_render_backward_ws checks its workspace before anything else; the
    pointers below are never dereferenced because every call is refused on
    the host."""
    s = W.julia_256(16, 16)
    p, pl, cam, li = _structs(s)
    n = F.fr_backward_workspace_bytes()
    assert n >= 11 * 8 + 4 and n % 16 == 0
    st = F.fr_render_backward_ws(p, pl, cam, li, None, None, None, None, None, n, None)
    assert st == F.FR_EINVAL and "workspace is NULL" in F.fr_last_error()
    st = F.fr_render_backward_ws(p, pl, cam, li, None, None, None, None, 8, n, None)
    assert st == F.FR_EINVAL and "aligned" in F.fr_last_error()
    st = F.fr_render_backward_ws(p, pl, cam, li, None, None, None, None, 256, n - 16, None)
    assert st == F.FR_ENOMEM
    # a well-formed workspace, then the ordinary argument checks
    ph = _structs(W.phong(s))
    st = F.fr_render_backward_ws(*ph, None, None, None, None, 256, n, None)
    assert st == F.FR_EINVAL and "Lambert" in F.fr_last_error(), F.fr_last_error()
    st = F.fr_render_backward_ws(p, pl, cam, li, None, None, None, None, 256, n, None)
    assert st == F.FR_EINVAL and "must be given" in F.fr_last_error(), F.fr_last_error()


def test_mandelbulb_backward_host_checks(F):
    """fr_render_backward_mandelbulb refuses on the host; no pointer below is
    ever dereferenced."""
    s = W.bulb_1080p(0, 16, 16)
    p, pl, cam, li = _structs(s)
    st = F.fr_render_backward_mandelbulb(p, pl, cam, li, None, None, None, None)
    assert st == F.FR_EINVAL and "must be given" in F.fr_last_error(), F.fr_last_error()
    st = F.fr_render_backward_mandelbulb(p, pl, cam, li, None, None, None, None, 8, 128)
    assert st == F.FR_EINVAL and "aligned" in F.fr_last_error()
    st = F.fr_render_backward_mandelbulb(p, pl, cam, li, None, None, None, None, 256, 64)
    assert st == F.FR_ENOMEM
    ph = _structs(W.phong(s))
    st = F.fr_render_backward_mandelbulb(*ph, None, None, None, None)
    assert st == F.FR_EINVAL and "Lambert" in F.fr_last_error()


def test_c_client_compiles_against_the_header():
    """A plain C99 program (tests/c_client/render_request.c) compiles with
    -Wall -Wextra -Werror against include/fr.h and links against libfr.so."""
    import c_client_build

    with tempfile.TemporaryDirectory() as d:
        exe = c_client_build.build(d)
        assert os.path.exists(exe)


def test_static_batch_checks_requests_before_any_cuda_call(F):
    """fr_render_batch_static refuses a NULL request array, a count outside
    1..4096 and a bad request on the host, before it asks CUDA for the device
    or the array's address (here there is no GPU, so any CUDA call would fail
    with FR_ECUDA instead)."""
    lib = F.load()
    assert lib.fr_render_batch_static(None, 3, None) == F.FR_EINVAL
    assert "NULL" in F.fr_last_error()
    s = W.julia_256(16, 16)
    req = F.fr_request()
    req.kind = F.FR_KIND_JULIA
    req.julia, req.plane, req.camera, req.light = _structs(s)
    arr = (F.fr_request * 2)(req, req)  # no output buffer in either request
    assert F.fr_render_batch_static(arr, 2, None) == F.FR_EINVAL
    assert "request 0" in F.fr_last_error() and "no output" in F.fr_last_error()
    arr[0].julia.p = 5
    assert F.fr_render_batch_static(arr, 2, None) == F.FR_EINVAL
    assert "request 0" in F.fr_last_error() and "degree" in F.fr_last_error()


def test_ffma_probe_host_checks_and_flop_count(F):
    """fr_ffma_probe refuses bad launch shapes and a NULL sink on the host;
    fr_ffma_probe_flops counts 2 flops per FFMA of 8 chains x 16 links per trip."""
    lib = F.load()
    assert F.fr_ffma_probe_flops(2, 64, 3) == 2 * 2 * 64 * 3 * 16 * 8
    assert F.fr_ffma_probe_flops(0, 64, 3) == 0.0
    assert lib.fr_ffma_probe(0, 256, 10, None, None) == F.FR_EINVAL
    assert lib.fr_ffma_probe(8, 48, 10, None, None) == F.FR_EINVAL and "threads" in F.fr_last_error()
    assert lib.fr_ffma_probe(8, 256, 0, None, None) == F.FR_EINVAL
    assert lib.fr_ffma_probe(8, 256, 10, None, None) == F.FR_EINVAL and "sink" in F.fr_last_error()


def test_sample_lanes_tuning_checked(F):
    t = F.fr_get_tuning()
    old = tuple(getattr(t, n) for n, _ in F.fr_tuning._fields_)
    assert t.sample_lanes == 1  # default: a pixel's 2, 4 or 8 samples on adjacent lanes
    bad = F.fr_tuning(*old)
    bad.sample_lanes = 2
    assert F.fr_set_tuning(bad) == F.FR_EINVAL and "sample_lanes" in F.fr_last_error()
    assert F.fr_set_tuning(F.fr_tuning(*old)) == F.FR_OK
