"""Pins of the oracle's Phong + reflection closest-hit model (the paper's
closest-hit listing for the Julia set: Phong lighting plus a reflection ray
weighted by the Fresnel-Schlick reflectance).

Each check compares the oracle with a closed form written out here from the
definitions (Phong's mirror-direction highlight, Schlick's approximation), or
with a configuration whose answer is fixed by geometry: a ray mirrored off the
cut face heads back into the half-space the cut removed, so it must see the
background.
"""
import math

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W


def _scene(**light):
    s = W.phong(W.julia_256(8, 8), **light)
    s["light"]["albedo"] = (0.9, 0.6, 0.3)
    s["light"]["k_ambient"], s["light"]["k_diffuse"] = 0.15, 0.7
    return s


def _schlick(f0, cos):
    return np.asarray(f0) + (1.0 - np.asarray(f0)) * (1.0 - cos) ** 5


def test_phong_reduces_to_lambert(orc):
    """k_specular = 0 and reflect_coef = 0 leave exactly the Lambert image."""
    for base in (W.bulb_1080p(10, 96, 54), dict(W.julia_256(64, 64), plane={"n": (0.0, 0.0, 1.0), "o": 0.0})):
        base["light"]["shadows"] = True
        ph = W.phong(base, k_specular=0.0, reflect_coef=0.0, background=base["light"]["background"])
        for prec in ("f64", "f32"):
            a = orc.render(base, precision=prec, threads=4)
            b = orc.render(ph, precision=prec, threads=4)
            assert np.array_equal(a["rgba"], b["rgba"]) and np.array_equal(a["depth"], b["depth"])
            assert np.array_equal(a["flags"], b["flags"])
            # the reflection ray is still traced and counted, once per hit
            hits = (b["flags"] & 1) == 1
            assert np.array_equal(b["stats"][:, 6], hits.astype(np.int64))
            assert np.all(a["stats"][:, 5:] == 0)


def test_highlight_peak_and_fresnel_at_normal_incidence(orc):
    """Light, normal and view on one axis: the highlight is k_s, the Schlick
    reflectance equals F0 (the albedo)."""
    s = _scene(k_specular=0.4, shininess=16.0, reflect_coef=0.2)
    s["light"]["dir"] = (0.0, 0.0, 2.0)  # normalised by the oracle
    refl = np.array([0.3, 0.2, 0.1])
    albedo = np.array(s["light"]["albedo"])
    got = orc.shade_phong(s, (0.0, 0.0, 1.0), (0.0, 0.0, -1.0), 1.0, refl)
    want = albedo * (0.15 + 0.7) + 0.4 + 0.2 * albedo * refl
    assert np.allclose(got[:3], want, rtol=0, atol=1e-15) and got[3] == 1.0
    # in shadow: ambient plus reflection only
    got = orc.shade_phong(s, (0.0, 0.0, 1.0), (0.0, 0.0, -1.0), 0.0, refl)
    assert np.allclose(got[:3], albedo * 0.15 + 0.2 * albedo * refl, rtol=0, atol=1e-15)


@pytest.mark.parametrize("alpha, delta, shin", [(0.3, 0.2, 8.0), (0.6, -0.4, 32.0), (0.1, 0.05, 64.0),
                                                (0.5, 1.3, 4.0)])
def test_highlight_falls_off_as_cos_power(orc, alpha, delta, shin):
    """Light at angle alpha from the normal, viewer at alpha + delta on the mirror
    side: the mirrored light direction and the view direction are delta apart, so
    the highlight is k_s cos(delta)^shininess (zero once delta passes 90 degrees);
    the Schlick weight uses the viewer's angle."""
    s = _scene(k_specular=0.7, shininess=shin, reflect_coef=0.3)
    s["light"]["dir"] = (math.sin(alpha), 0.0, math.cos(alpha))
    view = np.array([-math.sin(alpha + delta), 0.0, math.cos(alpha + delta)])  # toward the eye
    rd = -view
    refl = np.array([0.2, 0.5, 0.8])
    albedo = np.array(s["light"]["albedo"])
    got = orc.shade_phong(s, (0.0, 0.0, 1.0), rd, 1.0, refl)
    spec = max(0.0, math.cos(delta)) ** shin
    cos_v = max(0.0, math.cos(alpha + delta))
    want = albedo * (0.15 + 0.7 * math.cos(alpha)) + 0.7 * spec + 0.3 * _schlick(albedo, cos_v) * refl
    assert np.allclose(got[:3], want, rtol=1e-13, atol=1e-15)


def test_light_behind_surface_and_grazing_view(orc):
    s = _scene(k_specular=0.9, shininess=2.0, reflect_coef=0.25)
    s["light"]["dir"] = (0.0, 0.3, -1.0)  # below the surface z = 0
    albedo = np.array(s["light"]["albedo"])
    refl = np.array([0.4, 0.4, 0.4])
    # no diffuse and no highlight; a view along the surface sees F = 1
    got = orc.shade_phong(s, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), 1.0, refl)
    assert np.allclose(got[:3], albedo * 0.15 + 0.25 * refl, rtol=0, atol=1e-15)
    # Schlick at cos = 1/2: F0 + (1 - F0) / 32
    rd = np.array([math.sqrt(3) / 2, 0.0, -0.5])
    got = orc.shade_phong(s, (0.0, 0.0, 1.0), rd, 1.0, refl)
    assert np.allclose(got[:3], albedo * 0.15 + 0.25 * (albedo + (1 - albedo) / 32) * refl, rtol=1e-14)


def test_mirror_off_the_cut_face_sees_the_background(orc):
    """Julia set cut by z <= 0, camera on +z.  A cut-face pixel's mirror ray goes
    back toward +z, where the cut removed the set: it finds an empty interval
    (no DE call) and the colour is Phong on the plane normal plus
    reflect_coef * Schlick * background, written out here per pixel."""
    s = W.phong(dict(W.julia_256(48, 48), plane={"n": (0.0, 0.0, 2.0), "o": 0.05}),
                k_specular=0.3, shininess=8.0, reflect_coef=1.0)
    s["light"]["shadows"] = True
    s["light"]["dir"] = (0.3, 0.5, 0.8)
    o = orc.render(s, precision="f64", threads=4)
    face = (o["flags"] & 2) == 2
    assert face.sum() > 200
    assert np.all(o["stats"][face, 5] == 0) and np.all(o["stats"][face, 6] == 1)
    L = np.array(s["light"]["dir"]) / np.linalg.norm(s["light"]["dir"])
    albedo = np.array(s["light"]["albedo"])
    bg = np.array(s["light"]["background"][:3])
    n = np.array([0.0, 0.0, 1.0])
    for idx in np.flatnonzero(face):
        _, rd = orc.camera_ray(s, idx % 48, idx // 48)
        vis = 0.0 if o["flags"][idx] & 4 else 1.0
        ndl = n @ L
        r = 2 * ndl * n - L
        spec = max(0.0, -(r @ rd)) ** 8.0 if ndl > 0 else 0.0
        want = albedo * (0.1 + 0.9 * max(ndl, 0.0) * vis) + 0.3 * spec * vis + \
            _schlick(albedo, max(0.0, -(n @ rd))) * bg
        assert np.allclose(o["rgba64"][idx, :3], want, rtol=1e-12, atol=1e-14), idx


def test_reflected_colour_is_background_or_a_lit_surface(orc):
    """Without highlights, (image at reflect_coef 1) - (image at 0) = Schlick(n, rd) *
    (colour along the mirror ray), per channel.  Dividing out Schlick (from the
    pixel's own hit point and normal) leaves either the background or
    albedo * (k_a + k_d * cos) with one cos for all channels in [0, 1]."""
    base = W.bulb_1080p(10, 64, 36)
    a = orc.render(W.phong(base, k_specular=0.0, reflect_coef=0.0), precision="f64", threads=4)
    b = orc.render(W.phong(base, k_specular=0.0, reflect_coef=1.0), precision="f64", threads=4)
    s = W.phong(base, k_specular=0.0, reflect_coef=1.0)
    albedo = np.array(s["light"]["albedo"])
    bg = np.array(s["light"]["background"][:3])
    hits = np.flatnonzero((b["flags"] & 1) == 1)
    assert len(hits) > 300
    n_bg = n_lit = 0
    for idx in hits:
        ro, rd = orc.camera_ray(s, idx % 64, idx // 64)
        if b["flags"][idx] & 2:
            nrm = np.array([0.0, 0.0, 1.0])
        else:
            nrm = orc.normal_scene(s, ro + b["depth64"][idx] * rd, rd)
        F = _schlick(albedo, max(0.0, -(nrm @ rd)))
        c = (b["rgba64"][idx, :3] - a["rgba64"][idx, :3]) / F
        if np.allclose(c, bg, rtol=1e-9, atol=1e-12):
            n_bg += 1
            continue
        k = c / albedo
        assert np.allclose(k, k[0], rtol=1e-9, atol=1e-12), (idx, c)
        assert 0.1 - 1e-12 <= k[0] <= 1.0 + 1e-12, (idx, k)
        n_lit += 1
    assert n_bg > 20 and n_lit > 20, (n_bg, n_lit)
