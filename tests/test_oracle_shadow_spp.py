"""Pins of the oracle's shadow ray and of its combination of samples.

Neither step is printed in the paper (it reflects instead of casting shadow
rays, and it renders one sample per pixel), so both follow stated readings:
the shadow ray starts at x + 4 eps n and marches toward the light, any hit
shadows; a pixel's colour is the mean over its samples and its depth the
nearest hit.  The pins below check those readings against geometry and
against single-sample renders, never against a re-typed copy of the oracle's
arithmetic:

* With c = 0 the quaternion Julia set of z^2 + c is the closed unit ball (the
  orbit z^(2^k) stays bounded exactly when |z| <= 1), so its slice is the unit
  ball of R^3.  For a convex solid a boundary point is in shadow exactly when
  the ray toward the light enters the solid, i.e. when the outward normal n
  satisfies n . L < 0.  The same holds on the face a cutting plane leaves
  (ball intersected with a half-space is still convex), whose outward normal
  is the plane's.  Flipping the offset of the shadow ray's start, or marching
  toward -L, contradicts the rule on every pixel away from the terminator.
* A pixel with spp samples is the mean of the colours, and the minimum of the
  depths, of the single rays through its sample positions; each such ray is
  rendered on its own as the one pixel of a 1 x 1 image whose camera looks
  along it.
"""
import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W


def _unit_ball_scene(width, height, light_dir, plane=None, max_iter=30):
    s = W.julia_256(width, height)
    s.update(c=(0.0, 0.0, 0.0, 0.0), p=2, max_iter=max_iter, escape_r2=16.0, normal_mode="central",
             normal_h=1e-4, plane=plane)
    s["light"] = dict(s["light"], dir=tuple(light_dir), shadows=True)
    return s


def _hits(orc, s, r):
    """(pixel, hit point, view ray) of every pixel the render marks as hit."""
    W_, H_ = s["camera"]["width"], s["camera"]["height"]
    out = []
    for idx in np.flatnonzero((r["flags"] & 1) > 0):
        ro, rd = orc.camera_ray(s, idx % W_, idx // W_)
        out.append((idx, ro + r["depth64"][idx] * rd, rd))
    return out


@pytest.mark.parametrize("light", [(1.0, 0.3, -0.2), (-0.6, -0.7, 0.4)])
def test_shadow_on_unit_ball_is_the_terminator(orc, light):
    """c = 0: a hit on the unit sphere is shadowed iff (x/|x|) . L < 0.  Points
    with |n . L| below 0.25 are skipped: the ray from x + 4 eps n grazes the
    sphere there and the finite eps decides."""
    s = _unit_ball_scene(48, 48, light)
    r = orc.render(s, precision="f64", threads=4)
    L = np.asarray(light) / np.linalg.norm(light)
    lit = shadowed = 0
    for idx, x, _ in _hits(orc, s, r):
        n = x / np.linalg.norm(x)
        assert abs(np.linalg.norm(x) - 1.0) < 4 * s["eps"], idx  # on the sphere
        ndl = float(n @ L)
        if abs(ndl) < 0.25:
            continue
        flagged = bool(r["flags"][idx] & 4)
        assert flagged == (ndl < 0.0), (idx, ndl)
        lit += not flagged
        shadowed += flagged
    assert lit > 100 and shadowed > 100, (lit, shadowed)


@pytest.mark.parametrize("light, want_shadow", [((0.3, 0.2, 1.0), False), ((0.4, 0.5, -1.0), True)])
def test_shadow_on_cut_face_follows_the_plane_normal(orc, light, want_shadow):
    """The plane z = 0.3 cuts the unit ball; the camera on +z sees the cut face
    (a disk of radius sqrt(1 - 0.09)), whose outward normal is +z.  The face is
    in shadow exactly when L.z < 0: then the shadow ray, started 4 eps above
    the face, re-enters the kept half-space at once and is inside the ball.
    Eight orbit steps: with more, |z|^(2^k) of the disk's centre underflows to
    0 and the listing's 0.25 log(m2) sqrt(m2 / dz2) becomes 0 * inf = NaN."""
    s = _unit_ball_scene(40, 40, light, plane={"n": (0.0, 0.0, 1.0), "o": 0.3}, max_iter=8)
    r = orc.render(s, precision="f64", threads=4)
    faces = np.flatnonzero((r["flags"] & 2) > 0)
    assert len(faces) > 400
    for idx in faces:
        ro, rd = orc.camera_ray(s, idx % 40, idx // 40)
        x = ro + r["depth64"][idx] * rd
        assert abs(x[2] - 0.3) < 1e-9 and x[0] ** 2 + x[1] ** 2 < 1.0  # on the disk
        assert bool(r["flags"][idx] & 4) == want_shadow, idx
    # the colour says the same: Lambert with vis = 0 leaves the ambient term only
    L = np.asarray(light) / np.linalg.norm(light)
    li = s["light"]
    k = li["k_ambient"] + (0.0 if want_shadow else li["k_diffuse"] * max(0.0, L[2]))
    want = np.array(li["albedo"]) * k
    assert np.allclose(r["rgba64"][faces, :3], want, rtol=0, atol=1e-12)


def _single_ray_scene(s, ro, rd):
    """A 1 x 1 image whose only (centre) ray starts at ro along rd."""
    one = W.resized(s, 1, 1)
    cam = dict(one["camera"], eye=tuple(float(v) for v in ro),
               target=tuple(float(a + b) for a, b in zip(ro, rd)), spp=1)
    # keep `up` off the view direction
    cam["up"] = (0.0, 1.0, 0.0) if abs(rd[1]) < 0.9 else (1.0, 0.0, 0.0)
    one["camera"] = cam
    return one


@pytest.mark.parametrize("which", ["julia", "bulb"])
def test_spp_is_mean_colour_and_nearest_depth(orc, which):
    """spp = 4 with jitter: the pixel's float colour is the mean of the four
    single-ray renders through its sample positions and its depth the
    smallest of their depths (+inf when all miss)."""
    if which == "julia":
        s = W.julia_256(16, 16)
        s["light"] = dict(s["light"], shadows=True)
    else:
        s = W.bulb_1080p(10, 16, 12)
    s["camera"] = dict(s["camera"], spp=4, seed=5)
    Wd, H = s["camera"]["width"], s["camera"]["height"]
    r = orc.render(s, precision="f64", threads=4)
    col_err, dep_err, spread, mixed = [], [], 0, 0
    for idx in range(Wd * H):
        cols, deps = [], []
        for k in range(4):
            ro, rd = orc.camera_ray(s, idx % Wd, idx // Wd, k)
            o = orc.render(_single_ray_scene(s, ro, rd), precision="f64")
            cols.append(o["rgba64"][0])
            deps.append(o["depth64"][0])
        want_c = np.mean(cols, axis=0)
        want_d = min(deps)
        col_err.append(np.max(np.abs(r["rgba64"][idx] - want_c)))
        got_d = r["depth64"][idx]
        if np.isfinite(want_d):
            dep_err.append(abs(got_d - want_d) / want_d)
        else:
            dep_err.append(0.0 if not np.isfinite(got_d) else 1.0)
        fin = [d for d in deps if np.isfinite(d)]
        spread += len(fin) > 1 and max(fin) - min(fin) > 1e-4 * min(fin)
        mixed += 0 < len(fin) < 4
    col_err, dep_err = np.array(col_err), np.array(dep_err)
    # the 1 x 1 camera re-normalises the ray once more (a rounding in the last
    # bit of the direction), which can move a chaotic grazing ray: allow 1 %
    assert np.mean(col_err < 1e-9) >= 0.99, np.sort(col_err)[-5:]
    assert np.mean(dep_err < 1e-9) >= 0.99, np.sort(dep_err)[-5:]
    # the cases that tell mean from another combination and min from max exist
    assert spread > 20 and mixed > 3, (spread, mixed)
