"""The C ABI used from plain C (tests/c_client/render_request.c: its own
cudaMalloc, stream and copies; no Python or PyTorch in the process): the
images equal the ones rendered through the Python binding, bit for bit."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scene", ["bulb", "julia_cut", "phong"])
def test_c_client_matches_binding(scene):
    import torch

    import c_client_build
    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api

    s = {"bulb": W.bulb_1080p(10, 123, 77),
         "julia_cut": dict(W.julia_256(96, 64), plane={"n": (0.1, 0.2, 1.0), "o": 0.05}),
         "phong": W.phong(W.bulb_1080p(5, 64, 48))}[scene]
    ref = api.render(s, rgba8=True, depth=True)
    torch.cuda.synchronize()
    kind = F.FR_KIND_JULIA if s["kind"] == "julia" else F.FR_KIND_BULB
    prm = api.julia_params(s) if s["kind"] == "julia" else api.bulb_params(s)
    blob = (ctypes.c_int32(kind), prm, api.plane_struct(s), api.camera_struct(s), api.light_struct(s))
    with tempfile.TemporaryDirectory() as d:
        exe = c_client_build.build(d)
        pin, pout = os.path.join(d, "params.bin"), os.path.join(d, "out.bin")
        with open(pin, "wb") as f:
            for part in blob:
                f.write(bytes(part))
        r = subprocess.run([exe, pin, pout], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stderr
        raw = np.fromfile(pout, dtype=np.uint8)
    n = s["camera"]["width"] * s["camera"]["height"]
    assert raw.size == 8 * n
    rgba8 = raw[:4 * n].view(np.uint32)
    depth = raw[4 * n:].view(np.float32)
    assert np.array_equal(rgba8, ref["rgba8"].cpu().numpy().reshape(-1).view(np.uint32))
    assert np.array_equal(depth, ref["depth"].cpu().numpy().reshape(-1))


@pytest.mark.parametrize("normal", ["central", "analytic"])
def test_c_client_adjoint_matches_binding(normal):
    """The plain-C client's adjoint (fr_render_backward_ws with its own
    workspace, cotangent = the float colour) equals the binding's bit for bit."""
    import torch

    import c_client_build
    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api, autograd

    s, _ = W.diff_julia(W.BASE_SEED, 96, 80)
    s["normal_mode"] = normal
    out = api.render(s, rgba8=False, rgba=True, depth=False, saved=True)
    ref = autograd.backward_raw(s, out["saved"], out["rgba"], workspace=autograd.backward_workspace("cuda"))
    torch.cuda.synchronize()
    blob = (ctypes.c_int32(F.FR_KIND_JULIA), api.julia_params(s), api.plane_struct(s), api.camera_struct(s),
            api.light_struct(s))
    with tempfile.TemporaryDirectory() as d:
        exe = c_client_build.build(d)
        pin, pout, pgrad = (os.path.join(d, n) for n in ("params.bin", "out.bin", "grad.bin"))
        with open(pin, "wb") as f:
            for part in blob:
                f.write(bytes(part))
        r = subprocess.run([exe, pin, pout, pgrad], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stderr
        g = np.fromfile(pgrad, dtype=np.float32)
    assert g.size == 11 and np.any(g != 0)
    assert np.array_equal(g, ref.cpu().numpy())
