"""Pins of the oracle's implicit-differentiation gradient against central finite
differences of the oracle's own forward render (a different computation: the
forward march re-run at theta +- h, with no derivative code involved).

Implicit differentiation gives the derivative of the level set of the DE
through the hit point; the marched depth follows it as far as the march has
converged.  With a very tight hit threshold (eps = 1e-9, a converged march)
and a small step (h = 1e-6) the two must agree pixel by pixel.  At the
workload's eps = 1e-3 the marched depth still carries the march's own
convergence error, whose derivative implicit differentiation leaves out by
design, so there only the light gradient (which moves no hit) is compared.
Pixels whose discrete state (hit, cut face,
shadow, march and normal DE counts) changes between theta - h and theta + h
are masked out of both sides.
"""
import copy

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W


def perturb(scene, k, h):
    """scene with parameter k of (c[4], plane n[3], plane o, light dir[3]) moved by h"""
    s = copy.deepcopy(scene)
    if k < 4:
        c = list(s["c"]); c[k] += h; s["c"] = tuple(c)
    elif k < 7:
        n = list(s["plane"]["n"]); n[k - 4] += h; s["plane"]["n"] = tuple(n)
    elif k == 7:
        s["plane"]["o"] += h
    else:
        d = list(s["light"]["dir"]); d[k - 8] += h; s["light"]["dir"] = tuple(d)
    return s


def cotangents(n, seed=0):
    rng = np.random.default_rng(seed)
    d_rgba = rng.standard_normal((n, 4))
    d_rgba[:, 3] = 0.0
    return d_rgba, 0.3 * rng.standard_normal(n)


def fd_per_pixel(orc, scene, d_rgba, d_depth, h, threads=8):
    """Per-pixel central differences of l_i = d_rgba_i . rgba_i + d_depth_i * depth_i
    for the 11 parameters, and the mask of pixels with unchanged discrete state."""
    base = orc.render(scene, precision="f64", threads=threads)
    n = len(base["flags"])
    mask = np.ones(n, bool)
    fd = np.zeros((n, 11))
    discrete = [0, 1, 2, 4]  # primary, normal and shadow DE counts, shadow rays

    def lp(r):
        dep = np.where(np.isfinite(r["depth64"]), r["depth64"], 0.0)
        return np.sum(d_rgba * r["rgba64"], 1) + d_depth * dep

    for k in range(11):
        rp = orc.render(perturb(scene, k, h), precision="f64", threads=threads)
        rm = orc.render(perturb(scene, k, -h), precision="f64", threads=threads)
        for r in (rp, rm):
            mask &= (r["flags"] == base["flags"]) & np.all(
                r["stats"][:, discrete] == base["stats"][:, discrete], 1)
        fd[:, k] = (lp(rp) - lp(rm)) / (2 * h)
    return fd, mask, base


def implicit_per_pixel(orc, scene, d_rgba, d_depth, idx):
    n = scene["camera"]["width"] * scene["camera"]["height"]
    out = np.zeros((len(idx), 11))
    for j, i in enumerate(idx):
        m = np.zeros(n, np.uint8)
        m[i] = 1
        out[j] = orc.julia_grad(scene, d_rgba, d_depth, m)
    return out


@pytest.mark.parametrize("normal", ["central", "analytic"])
def test_implicit_gradient_matches_fd_per_pixel(orc, normal):
    """Per pixel at a converged march; the analytic normal (Sec. 2) moves
    through c and the hit point inside its own orbit, differentiated on dual
    numbers, against the finite differences of the rendered colour."""
    size = 40
    s, _ = W.diff_julia(W.BASE_SEED, size, size)
    s["eps"], s["max_steps"], s["normal_mode"] = 1e-9, 5000, normal
    d_rgba, d_depth = cotangents(size * size)
    fd, mask, base = fd_per_pixel(orc, s, d_rgba, d_depth, 1e-6)
    for kind, sel in (("surface", base["flags"] == 1), ("face", (base["flags"] & 2) > 0)):
        idx = np.flatnonzero(mask & sel)
        assert len(idx) > 100, kind
        g = implicit_per_pixel(orc, s, d_rgba, d_depth, idx)
        err = np.linalg.norm(fd[idx] - g, axis=1) / np.maximum(np.linalg.norm(fd[idx], axis=1), 1e-12)
        assert np.mean(err < 0.01) >= 0.99, kind
        if kind == "face":  # the face depends only on the plane and the light
            assert np.all(g[:, :4] == 0)


def test_shadowed_gradient_matches_fd_per_pixel(orc):
    """With shadow rays the lit surface pixels carry the diffuse term and the
    shadowed ones only the ambient: per pixel at a converged march, both kinds
    against the finite differences of the render (the pixel's state, shadow
    included, unchanged at theta +- h)."""
    size = 40
    s, _ = W.diff_julia(W.BASE_SEED, size, size)
    s["eps"], s["max_steps"] = 1e-9, 5000
    s["light"] = dict(s["light"], shadows=True)
    d_rgba, d_depth = cotangents(size * size, seed=3)
    fd, mask, base = fd_per_pixel(orc, s, d_rgba, d_depth, 1e-6)
    for kind, sel in (("lit", base["flags"] == 1), ("shadowed", base["flags"] == 5)):
        idx = np.flatnonzero(mask & sel)
        assert len(idx) > 30, (kind, len(idx))
        g = implicit_per_pixel(orc, s, d_rgba, d_depth, idx)
        err = np.linalg.norm(fd[idx] - g, axis=1) / np.maximum(np.linalg.norm(fd[idx], axis=1), 1e-12)
        assert np.mean(err < 0.01) >= 0.99, (kind, np.quantile(err, [0.5, 0.99]))


def test_implicit_gradient_fd_moderate_eps(orc):
    """eps = 1e-5, h = 1e-4: the march is converged well enough for 95% of the
    surface pixels to agree within 5%."""
    size = 40
    s, _ = W.diff_julia(W.BASE_SEED, size, size)
    s["eps"], s["max_steps"] = 1e-5, 2000
    d_rgba, d_depth = cotangents(size * size, seed=2)
    fd, mask, base = fd_per_pixel(orc, s, d_rgba, d_depth, 1e-4)
    idx = np.flatnonzero(mask & (base["flags"] == 1))
    assert len(idx) > 100
    g = implicit_per_pixel(orc, s, d_rgba, d_depth, idx)
    err = np.linalg.norm(fd[idx] - g, axis=1) / np.maximum(np.linalg.norm(fd[idx], axis=1), 1e-12)
    assert np.mean(err < 0.05) >= 0.95


def test_light_gradient_matches_fd_at_workload_eps(orc):
    """The light direction does not move the hit, so even at the workload's
    eps = 1e-3 its gradient equals the finite difference of the render."""
    size = 48
    s, _ = W.diff_julia(W.BASE_SEED, size, size)
    d_rgba, d_depth = cotangents(size * size, seed=1)
    fd, mask, _ = fd_per_pixel(orc, s, d_rgba, d_depth, 1e-3)
    fds = (fd * mask[:, None]).sum(0)
    g = orc.julia_grad(s, d_rgba, d_depth, mask.astype(np.uint8), threads=8)
    assert np.allclose(fds[8:], g[8:], rtol=1e-5, atol=1e-6 * np.linalg.norm(fds[8:]))


def test_cut_plane_depth_gradient_is_ray_plane_formula(orc):
    """On cut-face pixels the depth is the ray-plane crossing; its derivative with
    respect to the offset is 1 / (n . rd) (with a depth-only cotangent)."""
    s, _ = W.diff_julia(W.BASE_SEED, 32, 32)
    r = orc.render(s, precision="f64")
    face = (r["flags"] & 2) > 0
    assert face.sum() > 20
    n = np.array(s["plane"]["n"])
    want = 0.0
    for idx in np.flatnonzero(face):
        _, rd = orc.camera_ray(s, idx % 32, idx // 32)
        want += 1.0 / (n @ rd)
    g = orc.julia_grad(s, np.zeros((32 * 32, 4)), np.ones(32 * 32), face.astype(np.uint8))
    assert abs(g[7] - want) <= 1e-12 * abs(want)
    assert np.all(g[:4] == 0) and np.all(g[8:] == 0)


def test_gradient_rejects_bad_scenes(orc):
    s = W.bulb_1080p(0, 8, 8)
    s["camera"]["spp"] = 2
    with pytest.raises(ValueError):
        orc.julia_grad(s, np.zeros((64, 4)))
    s = W.julia_256(8, 8)
    s["camera"]["spp"] = 2
    with pytest.raises(ValueError):
        orc.julia_grad(s, np.zeros((64, 4)))


def test_mandelbulb_gradient_matches_fd_per_pixel(orc):
    """Mandelbulb renders move with the cut plane (cut-face pixels: depth and
    normal) and with the light (every lit pixel); per pixel against central
    differences of the rendered colour and depth.  The fractal has no
    parameter c, so dc is 0, and a surface hit does not move with the plane:
    there the implicit gradient's plane part is 0 by construction, and only
    the light part is compared (the 12-iteration DE is discontinuous where an
    orbit's escape count changes, so the marched depth of a surface hit can
    still wander with the march's start point on the plane -- a dependence
    implicit differentiation, which follows the level set, leaves out)."""
    size = 40
    s = W.bulb_1080p(10, size, size)
    s["eps"], s["max_steps"], s["light"]["shadows"] = 1e-9, 5000, False
    s["camera"]["eye"] = (0.3, 0.9, 2.4)
    d_rgba, d_depth = cotangents(size * size, seed=5)
    base = orc.render(s, precision="f64", threads=8)
    h = 1e-6
    mask = np.ones(size * size, bool)
    fd = np.zeros((size * size, 11))

    def lp(r):
        dep = np.where(np.isfinite(r["depth64"]), r["depth64"], 0.0)
        return np.sum(d_rgba * r["rgba64"], 1) + d_depth * dep

    for k in range(4, 11):
        rp = orc.render(perturb(s, k, h), precision="f64", threads=8)
        rm = orc.render(perturb(s, k, -h), precision="f64", threads=8)
        for r in (rp, rm):
            mask &= (r["flags"] == base["flags"]) & np.all(
                r["stats"][:, [0, 1, 2, 4]] == base["stats"][:, [0, 1, 2, 4]], 1)
        fd[:, k] = (lp(rp) - lp(rm)) / (2 * h)
    for kind, sel, cols in (("surface", base["flags"] == 1, slice(8, 11)),
                            ("face", (base["flags"] & 2) > 0, slice(4, 11))):
        idx = np.flatnonzero(mask & sel)
        assert len(idx) > 100, kind
        g = implicit_per_pixel(orc, s, d_rgba, d_depth, idx)
        assert np.all(g[:, :4] == 0)
        err = np.linalg.norm(fd[idx, cols] - g[:, cols], axis=1) / np.maximum(
            np.linalg.norm(fd[idx, cols], axis=1), 1e-12)
        assert np.mean(err < 0.01) >= 0.99, (kind, np.mean(err < 0.01))
        if kind == "surface":
            assert np.all(g[:, 4:8] == 0)
