"""Image comparison used by the GPU-vs-oracle parity tests.

Tolerances (float32 renders of a chaotic iteration; both sides compute in
float, the GPU with fused multiply-adds and the CUDA math library, the oracle
with the host libm and no fusion):
  - hit / miss agreement on >= 99.5% of pixels (alpha > 0 counts as a hit);
  - relative depth error <= 1e-3 on >= 99% of the pixels both sides hit;
  - every RGB channel within 3/255 on >= 99% of pixels;
  - no depth is NaN or -inf (a hit has a finite depth, a miss +inf), and the
    GPU's and the oracle's depths are finite on the same pixels on >= 99.5%
    of them, so no NaN slips past the depth comparison.  (The alpha channel is
    the hit flag only where the background is transparent.)
"""
import numpy as np

HIT_AGREE = 0.995
DEPTH_REL = 1e-3
DEPTH_FRAC = 0.99
RGB_TOL = 3
RGB_FRAC = 0.99


def unpack(rgba8):
    a = np.asarray(rgba8).astype(np.int64) & 0xFFFFFFFF
    return np.stack([(a >> (8 * k)) & 0xFF for k in range(4)], -1).astype(np.int64)


def compare(gpu_rgba8, gpu_depth, orc_rgba8, orc_depth):
    """Return a dict of agreement fractions; `ok` tells whether all bars are met."""
    g, o = unpack(gpu_rgba8).reshape(-1, 4), unpack(orc_rgba8).reshape(-1, 4)
    gd, od = np.asarray(gpu_depth, np.float64).ravel(), np.asarray(orc_depth, np.float64).ravel()
    gh, oh = g[:, 3] > 0, o[:, 3] > 0
    hit_agree = float(np.mean(gh == oh)) if len(gh) else 1.0
    both = gh & oh & np.isfinite(gd) & np.isfinite(od)
    rel = np.abs(gd[both] - od[both]) / np.maximum(np.abs(od[both]), 1e-30)
    depth_ok = float(np.mean(rel <= DEPTH_REL)) if both.any() else 1.0
    rgb_ok = float(np.mean(np.all(np.abs(g[:, :3] - o[:, :3]) <= RGB_TOL, 1))) if len(g) else 1.0
    res = {
        "n": int(len(g)),
        "hits": int(oh.sum()),
        "hit_agree": hit_agree,
        "depth_ok": depth_ok,
        "rgb_ok": rgb_ok,
        "depth_rel_p50": float(np.median(rel)) if both.any() else 0.0,
        "bad_depths": int(np.sum(np.isnan(gd)) + np.sum(np.isneginf(gd))),
        "finite_agree": float(np.mean(np.isfinite(gd) == np.isfinite(od))) if len(gd) else 1.0,
    }
    res["ok"] = (hit_agree >= HIT_AGREE and depth_ok >= DEPTH_FRAC and rgb_ok >= RGB_FRAC
                 and res["bad_depths"] == 0 and res["finite_agree"] >= HIT_AGREE)
    return res
