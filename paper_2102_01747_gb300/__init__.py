"""GB300 (sm_103a) renderer for distance-estimated sphere tracing of the
quaternion Julia set and the Mandelbulb (da Silva, Novello, Lopes, Velho,
"Real-time rendering of complex fractals").

Layers:
  include/fr.h            C ABI (fr_render_julia, fr_render_mandelbulb,
                          fr_render_batch, fr_render_backward, ...)
  csrc/*.cu               CUDA kernels and the ABI implementation -> _build/libfr.so
  _ffi.py                 ctypes mirror of fr.h, same-name thin wrappers
  api.py                  scene dicts + torch tensors -> C structs -> kernels
  workloads.py            seeded synthetic scenes
"""
from . import workloads  # noqa: F401  (inputs only; no compute)

__all__ = ["workloads", "api", "_ffi", "build"]


def __getattr__(name):
    # the tensor API pulls in torch; import it on first use
    if name in ("api", "_ffi", "build", "autograd", "autotune"):
        import importlib

        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
