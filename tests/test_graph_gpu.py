"""CUDA-graph capture of the render calls: every entry point launches only
stream-ordered work (kernels, and for the persistent schedule a memset of its
queue head) with its parameters passed by value, so a captured call replays to
the same images as the eager call."""
import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
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
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    for k, v in kw.items():
        setattr(t, k, v)
    assert F.fr_set_tuning(t) == F.FR_OK
    return F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])


def _replay_matches_eager(torch, outs, call):
    """Eager call -> reference; clear the outputs; capture the call; replay twice;
    the outputs must equal the reference bit for bit after each replay."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        call(s)
    s.synchronize()
    ref = [{k: v.clone() for k, v in o.items()} for o in outs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call(s)
    for _ in range(2):
        for o in outs:
            for v in o.values():
                v.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            for k in o:
                assert torch.equal(o[k], r[k]), k


def test_single_request_graph(env):
    torch, F, api = env
    scene = W.bulb_1080p(10, 160, 96)
    out = api.alloc_image(scene, rgba8=True, depth=True)
    args = (api.bulb_params(scene), api.plane_struct(scene), api.camera_struct(scene),
            api.light_struct(scene), api.image_struct(out))

    def call(s):
        F.check(F.fr_render_mandelbulb(*args, s.cuda_stream))

    _replay_matches_eager(torch, [out], call)


@pytest.mark.parametrize("batch_kernel", [1, 2, 0])
def test_batch_graph(env, batch_kernel):
    torch, F, api = env
    scenes = W.batch_mixed(seed=7, n_requests=70, min_log2=4.0, max_log2=6.5)  # two launches
    outs = [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]
    arr = api.request_array(scenes, outs)
    ws = api.workspace(len(scenes))
    old = _tuned(F, batch_kernel=batch_kernel)
    try:
        def call(s):
            F.check(F.fr_render_batch(arr, len(scenes), ws.data_ptr(), ws.numel(), s.cuda_stream))

        _replay_matches_eager(torch, outs, call)
    finally:
        F.fr_set_tuning(old)


@pytest.mark.parametrize("batch_kernel, n_requests", [(1, 5), (0, 70), (2, 70)])
def test_static_batch_graph(env, batch_kernel, n_requests):
    """The allocation-free batch call: its eager call looks up the device array's
    address; captured afterwards, it replays like the others.  Under the
    persistent schedules (which read the queue heads in the array) 70 requests
    make two launches, using two slots of the array."""
    torch, F, api = env
    scenes = W.batch_mixed(seed=8, n_requests=n_requests, min_log2=4.0, max_log2=6.0)
    outs = [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]
    arr = api.request_array(scenes, outs)
    old = _tuned(F, batch_kernel=batch_kernel)
    try:
        def call(s):
            F.check(F.fr_render_batch_static(arr, len(scenes), s.cuda_stream))

        _replay_matches_eager(torch, outs, call)
    finally:
        F.fr_set_tuning(old)
    # and the images are the per-request kernel's
    for sc, o in zip(scenes, outs):
        ref = api.render(sc, rgba8=True, depth=True)
        torch.cuda.synchronize()
        assert torch.equal(ref["rgba8"], o["rgba8"]) and torch.equal(ref["depth"], o["depth"])


def test_backward_graph(env):
    """Forward (with saved state) and adjoint captured together: every replay
    adds the same gradient bits to the accumulator (the adjoint's device-side
    double accumulator is cleared by each launch)."""
    torch, F, api = env
    s, _ = W.diff_julia(W.BASE_SEED, 128, 96)
    out = api.alloc_image(s, rgba8=False, rgba=True, depth=True, saved=True)
    n = 128 * 96
    rng = np.random.default_rng(2)
    d_rgba = torch.tensor(rng.standard_normal((n, 4)).astype(np.float32), device="cuda")
    d_depth = torch.tensor(rng.standard_normal(n).astype(np.float32), device="cuda")
    grad = torch.zeros(11, dtype=torch.float32, device="cuda")
    img = api.image_struct(out)
    args = (api.julia_params(s), api.plane_struct(s), api.camera_struct(s), api.light_struct(s), img)

    def call(st):
        F.check(F.fr_render_julia(*args, st.cuda_stream))
        F.check(F.fr_render_backward(args[0], args[1], args[2], args[3], out["saved"].data_ptr(),
                                     d_rgba.data_ptr(), d_depth.data_ptr(), grad.data_ptr(), st.cuda_stream))

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        call(st)
    st.synchronize()
    once = grad.clone()
    grad.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        call(st)
    grad.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(grad, once)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(grad, once + once)
