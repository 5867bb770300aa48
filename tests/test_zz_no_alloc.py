"""fr_render_batch_static: the batched render for callers that cannot allocate
device memory, such as a plugin whose host application owns every device
allocation, or a frame loop that may not call cudaMalloc once it runs (an
allocation can synchronise the device).  Its scratch memory, one queue head
per launch of up to 64 requests, lives in a fixed array inside the library.

Called through the C ABI twice in a row, it must give the same images, bit
for bit, as fr_render_batch given a caller workspace.  The persistent
schedules (batch_kernel 2, the default, and 0) read the queue heads, so they
run here with 130 small requests: three launches, which use three different
slots of the array.  The grid schedule (batch_kernel 1), which reads no queue
head, is checked too.
This file sorts last, so a stop-at-first-failure run has already run every
other test."""
import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _set_batch_kernel(F, batch_kernel):
    """Set fr_tuning.batch_kernel; returns the previous tuning."""
    old = F.fr_get_tuning()
    keep = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t = F.fr_tuning(*[getattr(old, n) for n, _ in F.fr_tuning._fields_])
    t.batch_kernel = batch_kernel
    assert F.fr_set_tuning(t) == F.FR_OK
    return keep


@pytest.mark.parametrize("batch_kernel, n_requests", [(0, 130), (2, 130), (1, 9)])
def test_static_workspace_batch_matches_workspace_batch(batch_kernel, n_requests):
    import torch

    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api
    from paper_2102_01747_gb300 import build as B

    assert torch.cuda.is_available()
    B.build()
    F.load()
    scenes = W.batch_mixed(seed=17, n_requests=n_requests, min_log2=4.0, max_log2=5.5)
    old = _set_batch_kernel(F, batch_kernel)
    try:
        ref_outs = [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]
        ws = api.workspace(len(scenes))
        assert ws.numel() >= 256 * ((len(scenes) + 63) // 64)
        st = F.fr_render_batch(api.request_array(scenes, ref_outs), len(scenes), ws.data_ptr(), ws.numel(),
                               api.current_stream())
        assert st == F.FR_OK, F.fr_last_error()
        torch.cuda.synchronize()
        ref = [(o["rgba8"].cpu().numpy(), o["depth"].cpu().numpy()) for o in ref_outs]
        assert sum(int((r8 != 0).sum()) for r8, _ in ref) > 0  # something was drawn
        for call in range(2):
            outs = [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]
            for o in outs:  # poison: every pixel must be written by the call
                o["rgba8"].fill_(-1)
                o["depth"].fill_(-1.0)
            arr = api.request_array(scenes, outs)
            st = F.fr_render_batch_static(arr, len(scenes), api.current_stream())
            assert st == F.FR_OK, F.fr_last_error()
            torch.cuda.synchronize()
            for k, ((r8, rd), o) in enumerate(zip(ref, outs)):
                assert np.array_equal(o["rgba8"].cpu().numpy(), r8), (call, k)
                assert np.array_equal(o["depth"].cpu().numpy(), rd), (call, k)
    finally:
        F.fr_set_tuning(old)


def test_static_workspace_rejects_oversized_batch():
    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api

    scenes = [W.julia_256(8, 8)]
    outs = [api.alloc_image(scenes[0])]
    arr = api.request_array(scenes, outs)
    assert F.fr_render_batch_static(arr, 5000, None) == F.FR_EINVAL
    assert "4096" in F.fr_last_error()
    assert F.fr_render_batch_static(arr, 0, None) == F.FR_EINVAL
