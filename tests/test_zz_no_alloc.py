"""fr_render_batch_static: the batched render for callers that cannot allocate
device memory (the scratch queue heads live in a fixed array inside the
library).  Called through the C ABI twice in a row, it must give the same
images as fr_render_batch with a caller workspace.  This file sorts last so a
stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_workspace_batch_matches_workspace_batch():
    import torch

    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api
    from paper_2102_01747_gb300 import build as B

    assert torch.cuda.is_available()
    B.build()
    scenes = W.batch_mixed(seed=17, n_requests=9, min_log2=4.6, max_log2=7.0)
    ref_outs = api.render_batch(scenes, rgba8=True, depth=True)
    torch.cuda.synchronize()
    ref = [(o["rgba8"].cpu().numpy(), o["depth"].cpu().numpy()) for o in ref_outs]
    for call in range(2):
        outs = [api.alloc_image(s, rgba8=True, depth=True) for s in scenes]
        for o in outs:  # poison: every pixel must be written by the call
            o["rgba8"].fill_(-1)
            o["depth"].fill_(-1.0)
        arr = api.request_array(scenes, outs)
        st = F.fr_render_batch_static(arr, len(scenes), api.current_stream())
        assert st == F.FR_OK, F.fr_last_error()
        torch.cuda.synchronize()
        for (r8, rd), o in zip(ref, outs):
            assert np.array_equal(o["rgba8"].cpu().numpy(), r8), call
            assert np.array_equal(o["depth"].cpu().numpy(), rd), call


def test_static_workspace_rejects_oversized_batch():
    from paper_2102_01747_gb300 import _ffi as F
    from paper_2102_01747_gb300 import api

    scenes = [W.julia_256(8, 8)]
    outs = [api.alloc_image(scenes[0])]
    arr = api.request_array(scenes, outs)
    assert F.fr_render_batch_static(arr, 5000, None) == F.FR_EINVAL
    assert "4096" in F.fr_last_error()
    assert F.fr_render_batch_static(arr, 0, None) == F.FR_EINVAL
