"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each compares the
oracle with an identity, a closed form, a special case that reduces to a
textbook routine (Python's complex arithmetic), a brute-force computation,
or a published value.  A plausible slip in the oracle (a dropped factor, a
wrong sign or index, a transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2102_01747_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- splitmix64
def test_splitmix64_published_value(orc):
    """First output of the public splitmix64 reference from state 0."""
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        state, want = (int(v, 16) for v in line.split())
        assert orc.splitmix64(state) == want


def test_jitter_is_exact_24bit_grid(orc):
    for pix in range(50):
        sx, sy = orc.jitter(7, pix, 4, pix % 4)
        for v in (sx, sy):
            assert 0.0 <= v < 1.0
            assert float(v * 2**24).is_integer()
    # different samples of one pixel differ
    assert orc.jitter(7, 3, 4, 0) != orc.jitter(7, 3, 4, 1)


# --------------------------------------------------------------- quaternions
def _rand_q(rng, k):
    return rng.standard_normal((k, 4)) * rng.uniform(0.1, 3.0, (k, 1))


def test_quaternion_units(orc):
    """Hamilton's relations i^2 = j^2 = k^2 = ijk = -1, ij = k, jk = i, ki = j."""
    one, i, j, k = np.eye(4)
    assert np.array_equal(orc.qmul(i, i), -one)
    assert np.array_equal(orc.qmul(j, j), -one)
    assert np.array_equal(orc.qmul(k, k), -one)
    assert np.array_equal(orc.qmul(i, j), k)
    assert np.array_equal(orc.qmul(j, k), i)
    assert np.array_equal(orc.qmul(k, i), j)
    assert np.array_equal(orc.qmul(j, i), -k)
    assert np.array_equal(orc.qmul(orc.qmul(i, j), k), -one)


def test_quaternion_norm_multiplicative(orc):
    """|pq| = |p||q| (the quaternions are a normed division algebra)."""
    rng = np.random.default_rng(1)
    P, Q = _rand_q(rng, 20000), _rand_q(rng, 20000)
    worst64 = worst32 = 0.0
    for a, b in zip(P, Q):
        pq = orc.qmul(a, b)
        want = np.linalg.norm(a) * np.linalg.norm(b)
        worst64 = max(worst64, abs(np.linalg.norm(pq) - want) / want)
        if len(P) and worst32 < 1.0:
            pq32 = orc.qmul(a, b, "f32").astype(np.float64)
            w32 = np.linalg.norm(a.astype(np.float32)) * np.linalg.norm(b.astype(np.float32))
            worst32 = max(worst32, abs(np.linalg.norm(pq32) - w32) / w32)
    assert worst64 < 1e-14
    assert worst32 < 1e-6


def test_quaternion_associative_and_conjugate(orc):
    rng = np.random.default_rng(2)
    for a, b, c in zip(_rand_q(rng, 500), _rand_q(rng, 500), _rand_q(rng, 500)):
        l = orc.qmul(orc.qmul(a, b), c)
        r = orc.qmul(a, orc.qmul(b, c))
        assert np.allclose(l, r, rtol=0, atol=1e-13 * np.linalg.norm(l) + 1e-300)
        conj = a * np.array([1, -1, -1, -1])
        qq = orc.qmul(a, conj)
        assert abs(qq[0] - np.dot(a, a)) <= 1e-14 * np.dot(a, a)
        assert np.all(np.abs(qq[1:]) <= 1e-14 * np.dot(a, a))


def test_quaternion_complex_copy_bitwise(orc):
    """span{1, i} is a copy of C: the product equals Python's complex product."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a = complex(*rng.standard_normal(2))
        b = complex(*rng.standard_normal(2))
        q = orc.qmul([a.real, a.imag, 0, 0], [b.real, b.imag, 0, 0])
        ab = a * b
        assert q[0] == ab.real and q[1] == ab.imag and q[2] == 0 and q[3] == 0


def test_quaternion_power_is_repeated_product(orc):
    rng = np.random.default_rng(4)
    for q in _rand_q(rng, 200):
        q3 = orc.qpow(q, 3)
        assert np.allclose(q3, orc.qmul(orc.qmul(q, q), q), rtol=1e-15, atol=0)
        # q commutes with its powers
        assert np.allclose(orc.qmul(q, orc.qpow(q, 2)), orc.qmul(orc.qpow(q, 2), q),
                           rtol=0, atol=1e-13 * np.linalg.norm(q) ** 3)


# ---------------------------------------------------- White-Nylander power (Eq. 1)
def test_bulb_power_modulus(orc):
    """|p^n| = |p|^n for the spherical power formula."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        v = rng.standard_normal(3) * rng.uniform(0.2, 1.5)
        n = int(rng.integers(2, 17))
        r = np.linalg.norm(v)
        got = np.linalg.norm(orc.bulb_pow(v, n))
        assert abs(got - r**n) <= 1e-13 * r**n


def test_bulb_power_axis_points(orc):
    """On the polar axis p^n stays on the axis; (0, 0, r)^8 has polar angle
    8 * pi/2 = 4 pi, i.e. it lands on +y with modulus r^8."""
    for n in range(2, 12):
        assert np.allclose(orc.bulb_pow([0.0, 1.3, 0.0], n), [0.0, 1.3**n, 0.0], rtol=1e-14, atol=0)
    got = orc.bulb_pow([0.0, 0.0, 0.9], 8)
    assert np.allclose(got, [0.0, 0.9**8, 0.0], rtol=0, atol=1e-14)


def test_bulb_power_reduces_to_complex_power(orc):
    """In the half-plane x = 0, z > 0 the azimuth is 0 and Eq. 1 is the complex
    power: (0, y, z)^n = (0, Re zeta^n, Im zeta^n) with zeta = y + i z."""
    rng = np.random.default_rng(6)
    for _ in range(2000):
        y = rng.uniform(-1.5, 1.5)
        z = rng.uniform(1e-3, 1.5)
        n = int(rng.integers(2, 11))
        zeta = complex(y, z) ** n
        got = orc.bulb_pow([0.0, y, z], n)
        r = abs(complex(y, z))
        # acos near the pole magnifies the rounding of y/r by 1/sin(polar angle) = r/z
        tol = 1e-14 * n * r**n * (1.0 + r / z)
        assert got[0] == 0.0
        assert abs(got[1] - zeta.real) <= tol
        assert abs(got[2] - zeta.imag) <= tol


def test_bulb_power_composes(orc):
    """Eq. 1 multiplies both angles by n, so powers compose while no angle wraps:
    for points near the +y axis with a small azimuth (polar angle b < pi/12,
    |a| < pi/12), (p^2)^3 = (p^3)^2 = p^6.  Checked in general position, off
    the half-plane where the complex reduction above applies."""
    rng = np.random.default_rng(13)
    for _ in range(2000):
        b = rng.uniform(1e-3, np.pi / 12)
        a = rng.uniform(-np.pi / 12, np.pi / 12)
        r = rng.uniform(0.5, 1.3)
        # the listing's axes: polar angle from +y, azimuth atan2(x, z)
        p = r * np.array([np.sin(b) * np.sin(a), np.cos(b), np.sin(b) * np.cos(a)])
        p6 = orc.bulb_pow(p, 6)
        p23 = orc.bulb_pow(orc.bulb_pow(p, 2), 3)
        p32 = orc.bulb_pow(orc.bulb_pow(p, 3), 2)
        tol = 1e-12 * r**6
        assert np.allclose(p23, p6, rtol=0, atol=tol) and np.allclose(p32, p6, rtol=0, atol=tol)


def test_bulb_power_f32_close_to_f64(orc):
    rng = np.random.default_rng(7)
    for _ in range(500):
        v = rng.standard_normal(3)
        v32 = v.astype(np.float32).astype(np.float64)
        a = orc.bulb_pow(v32, 8)
        b = orc.bulb_pow(v32, 8, "f32")
        assert np.allclose(a, b, rtol=0, atol=5e-6 * np.linalg.norm(v32) ** 8)


# ------------------------------------------- Julia set restricted to span{1, i}
def _complex_de(z, c, max_iter, esc2):
    """The 2D escape-time orbit with its derivative, |f'|^2 carried as in the
    quaternion DE: returns (d, n_nonescaping, trips, m2)."""
    dz2, m2, n, trips = 1.0, 0.0, 0, 0
    for _ in range(max_iter):
        trips += 1
        dz2 *= 4.0 * (z.real * z.real + z.imag * z.imag)
        z = z * z + c
        m2 = z.real * z.real + z.imag * z.imag
        if m2 > esc2:
            break
        n += 1
    return 0.25 * math.log(m2) * math.sqrt(m2 / dz2), n, trips, m2


def test_julia_complex_subspace_bitwise(orc):
    """With c and the point in span{1, i}, the quaternion orbit is the complex
    orbit of z^2 + c (Sec. 1.1): counts, |z|^2 and the DE agree bit for bit."""
    rng = np.random.default_rng(8)
    s = W.julia_256(8, 8)
    for trial in range(5):
        c = complex(*rng.uniform(-0.8, 0.8, 2))
        s["c"] = (c.real, c.imag, 0.0, 0.0)
        pts = np.c_[rng.uniform(-1.6, 1.6, (300, 2)), np.zeros(300)]
        d, n, tr, m2 = orc.de(s, pts)
        for j, (x, y, _) in enumerate(pts):
            want = _complex_de(complex(x, y), c, s["max_iter"], s["escape_r2"])
            assert (d[j], n[j], tr[j], m2[j]) == want or (math.isnan(d[j]) and math.isnan(want[0]))


def _complex_de_cube(z, c, max_iter, esc2):
    """The listing's degree-3 orbit on C: |f'|^2 picks up 9 |z^2|^2 per step."""
    dz2, m2, n, trips = 1.0, 0.0, 0, 0
    for _ in range(max_iter):
        trips += 1
        z2 = z * z
        dz2 *= 9.0 * (z2.real * z2.real + z2.imag * z2.imag)
        z = z2 * z + c
        m2 = z.real * z.real + z.imag * z.imag
        if m2 > esc2:
            break
        n += 1
    return 0.25 * math.log(m2) * math.sqrt(m2 / dz2), n, trips, m2


def test_julia_cube_complex_subspace_bitwise(orc):
    """The listing's own degree (qCube, escape |z|^2 > 256): on span{1, i} the
    quaternion orbit of z^3 + c is the complex one, bit for bit."""
    rng = np.random.default_rng(12)
    s = W.julia_256(8, 8)
    s.update(p=3, escape_r2=256.0, max_iter=12)
    for trial in range(4):
        c = complex(*rng.uniform(-0.7, 0.7, 2))
        s["c"] = (c.real, c.imag, 0.0, 0.0)
        pts = np.c_[rng.uniform(-1.4, 1.4, (300, 2)), np.zeros(300)]
        d, n, tr, m2 = orc.de(s, pts)
        for j, (x, y, _) in enumerate(pts):
            want = _complex_de_cube(complex(x, y), c, s["max_iter"], s["escape_r2"])
            assert (d[j], n[j], tr[j], m2[j]) == want or (math.isnan(d[j]) and math.isnan(want[0]))


def test_julia_complex_subspace_float32(orc):
    """Same reduction at float precision, against numpy float32 complex steps."""
    rng = np.random.default_rng(9)
    s = W.julia_256(8, 8)
    f = np.float32
    c = complex(-0.2, 0.6)
    s["c"] = (c.real, c.imag, 0.0, 0.0)
    cr, ci = f(c.real), f(c.imag)
    pts = np.c_[rng.uniform(-1.6, 1.6, (300, 2)), np.zeros(300)].astype(np.float32)
    d, n, tr, m2 = orc.de(s, pts, "f32")
    for j, (x, y, _) in enumerate(pts):
        zr, zi, dz2, mm, cnt = f(x), f(y), f(1), f(0), 0
        for _ in range(s["max_iter"]):
            dz2 = f(dz2 * f(f(4) * f(f(zr * zr) + f(zi * zi))))
            zr, zi = f(f(f(zr * zr) - f(zi * zi)) + cr), f(f(f(zr * zi) + f(zi * zr)) + ci)
            mm = f(f(zr * zr) + f(zi * zi))
            if mm > f(16):
                break
            cnt += 1
        assert n[j] == cnt and m2[j] == mm


def test_julia_rotated_complex_plane(orc):
    """For general c = (c0, c1, c2, 0), points x + s*u with u = Im c / |Im c| stay in
    span{1, u}, a copy of C with c -> c0 + i |Im c|: same escape counts and DE."""
    rng = np.random.default_rng(10)
    s = W.julia_256(8, 8)
    agree, total = 0, 0
    for trial in range(4):
        cv = np.r_[rng.uniform(-0.6, 0.6, 3), 0.0]
        s["c"] = tuple(cv)
        u = cv[1:3] / np.linalg.norm(cv[1:3])
        cc = complex(cv[0], np.linalg.norm(cv[1:3]))
        xs = rng.uniform(-1.5, 1.5, 400)
        ss = rng.uniform(-1.5, 1.5, 400)
        pts = np.c_[xs, ss * u[0], ss * u[1]]
        d, n, tr, m2 = orc.de(s, pts)
        for j in range(len(xs)):
            want = _complex_de(complex(xs[j], ss[j]), cc, s["max_iter"], s["escape_r2"])
            total += 1
            if n[j] == want[1]:
                agree += 1
                assert abs(d[j] - want[0]) <= 1e-10 * max(1.0, abs(want[0]))
    assert agree / total >= 0.995


def test_escape_time_2d_matches_complex(orc):
    rng = np.random.default_rng(11)
    for _ in range(2000):
        z = complex(*rng.uniform(-1.6, 1.6, 2))
        c = complex(-0.2, 0.6)
        k, w = 0, z
        for i in range(50):
            w = w * w + c
            if w.real * w.real + w.imag * w.imag > 16.0:
                k = i + 1
                break
        else:
            k = 50
        assert orc.julia2d_escape(z, c, 50, 16.0) == k


def test_cut_face_is_2d_julia_set(orc):
    """Render-level form of the slice claim (Fig. 1): with c in span{1, i} and the
    plane z = 0 cutting away the half-space the camera sits in, a pixel shows the
    cut face exactly where the 2D complex DE at its plane point is below eps."""
    s = W.julia_256(48, 48)
    c = complex(-0.2, 0.6)
    s["c"] = (c.real, c.imag, 0.0, 0.0)
    s["camera"]["eye"] = (0.0, 0.0, -3.0)
    s["plane"] = {"n": (0.0, 0.0, -1.0), "o": 0.0}  # keep z >= 0
    r = orc.render(s, precision="f64")
    face = (r["flags"] & 2) > 0
    bad = 0
    for idx in range(48 * 48):
        ro, rd = orc.camera_ray(s, idx % 48, idx // 48)
        t = -ro[2] / rd[2]
        x, y = ro[0] + t * rd[0], ro[1] + t * rd[1]
        d2 = _complex_de(complex(x, y), c, s["max_iter"], s["escape_r2"])[0]
        if (d2 < s["eps"]) != face[idx] and abs(d2 - s["eps"]) > 1e-9:
            bad += 1
    assert face.sum() > 100
    assert bad == 0


# ------------------------------------------ DE bracket against brute force (Eq. 2)
def _grid(N, L):
    xs = (np.arange(N) + 0.5) / N * 2 * L - L
    return xs, 2 * L / N


def test_de_bracket_2d_julia(orc):
    """Against the distance to the escape-time set on a 64^2 grid: the DE is a
    lower bound (Sec. 2 derives |eps| >= G/|grad G|, a safe step) and, for the
    connected set of z^2 - 0.2 + 0.6i, within the Koebe factor 4 of it."""
    from scipy.spatial import cKDTree

    c = complex(-0.2, 0.6)
    z0, k = 0j, 0
    for k in range(200):
        z0 = z0 * z0 + c
    assert abs(z0) < 2  # orbit of 0 bounded: the Julia set is connected
    xs, delta = _grid(64, 1.6)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    z = X + 1j * Y
    inside = np.ones(z.shape, bool)
    for _ in range(64):
        z = np.where(inside, z * z + c, z)
        inside &= np.abs(z) ** 2 <= 16
    tree = cKDTree(np.c_[X[inside], Y[inside]])
    rng = np.random.default_rng(12)
    pts = rng.uniform(-1.6, 1.6, (3000, 2))
    dbf, _ = tree.query(pts)
    keep = dbf >= 3 * delta
    pts, dbf = pts[keep], dbf[keep]
    s = W.julia_256(8, 8)
    s["c"] = (c.real, c.imag, 0.0, 0.0)
    d, *_ = orc.de(s, np.c_[pts, np.zeros(len(pts))])
    ratio = dbf / d
    assert np.mean(d <= dbf + math.sqrt(2) * delta) >= 0.99
    assert np.mean(d <= dbf) >= 0.99
    assert np.mean(dbf <= 4 * d + math.sqrt(2) * delta) >= 0.99
    assert 1.2 <= np.median(ratio) <= 2.5


def _quat_julia_inside(X, Y, Z, c, iters=64):
    q = np.stack([X, Y, Z, np.zeros_like(X)], 0)
    inside = np.ones(X.shape, bool)
    cv = np.array(c)[:, None, None, None]
    for _ in range(iters):
        a, b, cc, dd = q
        q2 = np.stack([a * a - b * b - cc * cc - dd * dd, 2 * a * b, 2 * a * cc, 2 * a * dd], 0) + cv
        q = np.where(inside[None], q2, q)
        inside &= (q**2).sum(0) <= 16
    return inside


def _bulb_inside(X, Y, Z, n, iters=64):
    """Membership by the escape-time definition of Sec. 1.2 with Eq. 1 written in
    numpy spherical coordinates (polar from +y, azimuth atan2(x, z))."""
    C = np.stack([X, Y, Z], 0)
    w = C.copy()
    inside = np.ones(X.shape, bool)
    with np.errstate(all="ignore"):
        for _ in range(iters):
            r = np.sqrt((w**2).sum(0))
            th = np.arccos(np.clip(w[1] / np.where(r > 0, r, 1), -1, 1))
            ph = np.arctan2(w[0], w[2])
            rn = r**n
            w2 = np.stack([rn * np.sin(n * th) * np.sin(n * ph), rn * np.cos(n * th),
                           rn * np.sin(n * th) * np.cos(n * ph)], 0) + C
            w = np.where(inside[None], w2, w)
            inside &= (w**2).sum(0) <= 4
    return inside


@pytest.mark.parametrize("kind", ["julia", "bulb"])
def test_de_lower_bound_3d(orc, kind):
    """3D bracket on a 48^3 grid: the DE never exceeds the brute-force distance
    (+ one voxel diagonal).  No theorem gives an upper factor in 3D, so only the
    lower bound is asserted; the median ratio is kept in a sane range."""
    from scipy.spatial import cKDTree

    xs, delta = _grid(48, 1.6)
    X, Y, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    if kind == "julia":
        s = W.julia_256(8, 8)
        inside = _quat_julia_inside(X, Y, Z, s["c"])
    else:
        s = W.bulb_1080p(0, 8, 8)
        inside = _bulb_inside(X, Y, Z, 8)
    tree = cKDTree(np.c_[X[inside], Y[inside], Z[inside]])
    rng = np.random.default_rng(13)
    pts = rng.uniform(-1.6, 1.6, (2500, 3))
    dbf, _ = tree.query(pts)
    keep = dbf >= 3 * delta
    pts, dbf = pts[keep], dbf[keep]
    d, *_ = orc.de(s, pts)
    assert np.mean(d <= dbf + math.sqrt(3) * delta) >= 0.99
    assert 1.1 <= np.median(dbf / d) <= 3.0


@pytest.mark.parametrize("p", [2, 3])
def test_julia_slice_is_a_rotation(orc, p):
    """With c in span{1, i}, z -> z^p + c commutes with every rotation of the
    (j, k) plane (z^p keeps the direction of z's imaginary part; c has no j or
    k part), so |z_n| and |z_n'| are invariant: the DE at (x, y, z) on the
    slice w = s equals the DE at (x, y, sqrt(z^2 + s^2)) on the slice w = 0."""
    rng = np.random.default_rng(32 + p)
    base = W.julia_256(8, 8)
    base["p"], base["c"] = p, ((-0.2, 0.6, 0.0, 0.0) if p == 2 else (-0.1, 0.55, 0.0, 0.0))
    same = close = 0
    for _ in range(40):
        sw = float(rng.uniform(-0.7, 0.7))
        pts = rng.uniform(-1.2, 1.2, (20, 3))
        rot = np.c_[pts[:, :2], np.sqrt(pts[:, 2] ** 2 + sw * sw)]
        d1, n1, t1, _ = orc.de(dict(base, slice_w=sw), pts)
        d0, n0, t0, _ = orc.de(dict(base, slice_w=0.0), rot)
        ok = (n1 == n0) & (t1 == t0)
        same += int(ok.sum())
        close += int(np.sum(ok & (np.abs(d1 - d0) <= 1e-9 * np.maximum(np.abs(d0), 1e-12))))
    assert same >= 0.98 * 800 and close == same


# ------------------------------------------------ gradient schemes (Eq. 5)
def test_tetra_gradient_exact_on_affine(orc):
    """Sum nu_i = 0 and sum (nu_i)_x nu_i = (4, 0, 0) make Eq. 5 exact on affine
    fields for every h."""
    rng = np.random.default_rng(14)
    for _ in range(200):
        a = rng.standard_normal(3)
        b = rng.standard_normal()
        p = rng.standard_normal(3)
        h = 10 ** rng.uniform(-4, 0)
        n = orc.normal_field(1, np.r_[a, b], p, orc.NORMAL_TETRA, h)
        assert np.allclose(n, a / np.linalg.norm(a), rtol=0, atol=1e-9)


def test_central_gradient_exact_on_quadratic(orc):
    rng = np.random.default_rng(15)
    for _ in range(200):
        A = rng.standard_normal((3, 3))
        g = rng.standard_normal(3)
        p = rng.standard_normal(3)
        h = 10 ** rng.uniform(-3, 0)
        n = orc.normal_field(2, np.r_[A.ravel(), g], p, orc.NORMAL_CENTRAL, h)
        grad = (A + A.T) @ p + g
        assert np.allclose(n, grad / np.linalg.norm(grad), rtol=0, atol=1e-8)


def test_tetra_default_step_follows_eps(orc):
    """With normal_h = 0 the tetrahedral stencil takes the listing's step
    h = 0.5773 eps.  The c = 0 Julia set's DE is d = r log(r) / 2 whatever the
    escape count (z_n = r^(2^n), |z_n'| = 2^n r^(2^n - 1)), so the exact normal
    is x / |x|.  On a radial field Eq. 5 errs by a tangential term of order h
    (the tetrahedron's third moment, sum nu (nu . u)^2, is nonzero off its
    axes), so the normal's error is small and falls tenfold with eps."""
    rng = np.random.default_rng(31)
    dirs = rng.standard_normal((60, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    errs = {}
    for eps in (1e-3, 1e-4):
        s = W.julia_256(8, 8)
        s["c"] = (0.0, 0.0, 0.0, 0.0)
        s["normal_mode"], s["normal_h"], s["eps"] = "tetra", 0.0, eps
        errs[eps] = np.array([np.linalg.norm(orc.normal_scene(s, 1.5 * u) - u) for u in dirs])
    assert np.max(errs[1e-3]) < 2e-3
    ratio = np.median(errs[1e-3] / np.maximum(errs[1e-4], 1e-300))
    assert 7.0 < ratio < 14.0, ratio


def test_zero_gradient_falls_back_to_view(orc):
    n = orc.normal_field(1, [0.0, 0.0, 0.0, 1.0], [0.1, 0.2, 0.3], orc.NORMAL_TETRA, 1e-3,
                         rd=[0.0, 0.6, 0.8])
    assert np.allclose(n, [0.0, -0.6, -0.8])


# ------------------------------------------------------ sphere tracing
def test_march_exact_sphere(orc):
    """With an exact SDF the march stops within eps in front of the analytic root."""
    rng = np.random.default_rng(16)
    hits = 0
    for _ in range(500):
        q = rng.uniform(-1, 1, 3)
        r = rng.uniform(0.2, 1.0)
        ro = rng.uniform(-1, 1, 3) + np.array([0, 0, 4.0])
        rd = q + rng.normal(0, 0.3, 3) - ro
        rd /= np.linalg.norm(rd)
        eps = 1e-4
        hit, t, steps = orc.march_field(0, np.r_[q, r], ro, rd, eps, 50.0, 1000, eps, 0.2)
        oc = ro - q
        b = oc @ rd
        disc = b * b - (oc @ oc - r * r)
        if disc >= 0 and -b - math.sqrt(disc) > 0:
            root = -b - math.sqrt(disc)
            assert hit
            # stopped in front of the root, at a point closer than eps to the surface
            assert t <= root + 1e-12
            assert np.linalg.norm(ro + t * rd - q) - r < eps
            # the distance along the ray is at most eps / cos(incidence)
            cosi = -((ro + root * rd - q) / r) @ rd
            assert root - t <= eps / cosi + 1e-12
            assert steps >= math.floor((root - 1.0) / 0.2)  # the step clamp bounds progress
            hits += 1
        else:
            assert not hit
    assert hits > 100


def test_march_step_cap_counts_as_hit(orc):
    """Out of steps inside the interval: the final test of the ray-cast listing
    (t < tmax) reports a hit at the current t."""
    hit, t, steps = orc.march_field(0, [0, 0, 0, 0.5], [0, 0, 10.0], [0, 0, -1.0], 0.0, 100.0,
                                    5, 1e-4, 0.2)
    assert hit and steps == 5 and abs(t - 1.0) < 1e-12


def test_march_miss_past_interval(orc):
    hit, t, steps = orc.march_field(0, [0, 0, 0, 0.5], [0, 0, 10.0], [0, 0, -1.0], 0.0, 5.0,
                                    1000, 1e-4, 0.2)
    assert not hit and t > 5.0 and steps == 25


# ------------------------------------------------------ interval (bounds + cut)
def test_bounds_brute_force(orc):
    rng = np.random.default_rng(17)
    s = W.julia_256(8, 8)
    for trial in range(300):
        nrm = rng.standard_normal(3)
        s["plane"] = {"n": tuple(nrm), "o": float(rng.uniform(-0.5, 0.5))} if trial % 3 else None
        ro = rng.uniform(-3, 3, 3)
        rd = rng.standard_normal(3)
        rd /= np.linalg.norm(rd)
        ok, t0, t1, fp = orc.bounds(s, ro, rd)
        ts = np.linspace(0, 8, 80001)
        P = ro[None] + ts[:, None] * rd[None]
        inside = (np.sum(P * P, 1) <= 4.0) & (ts >= s["eps"])
        if s["plane"]:
            inside &= P @ nrm <= s["plane"]["o"]
        if inside.sum() < 3:
            if inside.sum() == 0:
                assert not ok
            continue
        assert ok
        assert abs(ts[inside].min() - t0) <= 2e-4
        assert abs(ts[inside].max() - t1) <= 2e-4
        if fp:
            assert abs((ro + t0 * rd) @ nrm - s["plane"]["o"]) <= 1e-9 * np.linalg.norm(nrm) * 10


# ------------------------------------------------------ shading and quantiser
def test_lambert_special_cases(orc):
    s = W.julia_256(8, 8)
    L = np.array(s["light"]["dir"]) / np.linalg.norm(s["light"]["dir"])
    alb = np.array(s["light"]["albedo"])
    ka, kd = s["light"]["k_ambient"], s["light"]["k_diffuse"]
    assert np.allclose(orc.shade(s, L)[:3], alb * (ka + kd), rtol=1e-15)
    assert np.allclose(orc.shade(s, -L)[:3], alb * ka, rtol=1e-15)
    perp = np.cross(L, [0, 0, 1.0])
    perp /= np.linalg.norm(perp)
    assert np.allclose(orc.shade(s, perp)[:3], alb * ka, atol=1e-15)
    assert np.allclose(orc.shade(s, L, 0.0)[:3], alb * ka, rtol=1e-15)
    assert orc.shade(s, L)[3] == 1.0


def test_quantizer_round_half_up(orc):
    for prec in ("f64", "f32"):
        assert orc.quantize(0.0, prec) == 0
        assert orc.quantize(-0.3, prec) == 0
        assert orc.quantize(1.0, prec) == 255
        assert orc.quantize(7.0, prec) == 255
        assert orc.quantize(0.5, prec) == 128  # 127.5 rounds up
        assert orc.quantize(float("nan"), prec) == 0
        assert orc.quantize(100.0 / 255.0, prec) == 100


# ------------------------------------------------------ camera
def test_camera_geometry(orc):
    s = W.julia_256(65, 33)
    ro, rd = orc.camera_ray(s, 32, 16)
    f = -np.array(s["camera"]["eye"]) / np.linalg.norm(s["camera"]["eye"])
    assert np.allclose(ro, s["camera"]["eye"]) and np.allclose(rd, f, atol=1e-15)
    _, a = orc.camera_ray(s, 0, 0)
    _, b = orc.camera_ray(s, 64, 32)
    assert np.allclose(a[:2], -b[:2]) and a[1] > 0 and a[0] < 0  # top-left looks up-left
    # the image plane spans the vertical field of view
    half = math.radians(s["camera"]["fov_y_deg"]) / 2
    _, top = orc.camera_ray(s, 32, 0)
    ang = math.atan2(top[1], -top[2])
    assert abs(ang - math.atan((1 - 1 / 33) * math.tan(half))) < 1e-12


# ------------------------------------------------------ float oracle vs double oracle
@pytest.mark.parametrize("which", ["julia", "bulb"])
def test_f32_oracle_close_to_f64(orc, which):
    """The float twin agrees with the double reference within the render tolerances
    (hit/miss on >= 99.5% of pixels, depth and colour on >= 99%)."""
    s = W.julia_256(64, 64) if which == "julia" else W.bulb_1080p(10, 96, 54)
    a = orc.render(s, precision="f64", threads=4)
    b = orc.render(s, precision="f32", threads=4)
    ha, hb = (a["flags"] & 1) > 0, (b["flags"] & 1) > 0
    assert np.mean(ha == hb) >= 0.995
    both = ha & hb
    rel = np.abs(a["depth"][both] - b["depth"][both]) / a["depth"][both]
    assert np.mean(rel <= 1e-3) >= 0.99
    ca = np.stack([(a["rgba8"] >> (8 * k)) & 255 for k in range(4)], -1).astype(int)
    cb = np.stack([(b["rgba8"] >> (8 * k)) & 255 for k in range(4)], -1).astype(int)
    assert np.mean(np.all(np.abs(ca - cb) <= 3, -1)) >= 0.99


# ------------------------------------------------------ orbit traps (listing colour outputs)
def test_julia_trap_is_escape_count(orc):
    """Julia: the listing's second output is the number of non-escaping steps; on
    span{1, i} it equals the complex orbit's count and final |z|^2 bit for bit."""
    rng = np.random.default_rng(31)
    s = W.julia_256(8, 8)
    c = complex(-0.2, 0.6)
    s["c"] = (c.real, c.imag, 0.0, 0.0)
    for x, y in rng.uniform(-1.5, 1.5, (300, 2)):
        t = orc.trap(s, [x, y, 0.0])
        _, n, _, m2 = _complex_de(complex(x, y), c, s["max_iter"], s["escape_r2"])
        assert t[0] == n and t[1] == m2 and t[2] == 0 and t[3] == 0


def test_bulb_trap_on_polar_axis(orc):
    """On the +y axis Eq. 1 maps (0, y, 0) to (0, y^n, 0), so the orbit is the scalar
    recursion y <- y^n + y0 and the trap is (final y^2, y0, 0, y0^2)."""
    s = W.bulb_1080p(0, 8, 8)
    for y0 in (0.3, 0.6, 0.9, 1.05):
        for n in (2, 3, 8):
            s["n"] = n
            y, m = y0, y0 * y0
            for _ in range(s["max_iter"]):
                y = y**n + y0
                m = y * y
                if m > s["bailout"] ** 2:
                    break
            t = orc.trap(s, [0.0, y0, 0.0])
            assert abs(t[0] - m) <= 1e-12 * max(1.0, m)
            assert t[1] == y0 and t[2] == 0.0 and abs(t[3] - y0 * y0) <= 1e-15


def _axis_orbit(y0, n, trips):
    """The orbit of Eq. 1 on the polar axis: y <- y^n + y0 from y = y0."""
    y = y0
    for _ in range(trips):
        y = y**n + y0
    return y


def test_bulb_trap_takes_the_previous_m(orc):
    """The listing folds the new w into the running minimum beside the m of the
    step before, so 'min m' leaves out the final iterate's |w|^2 while 'min |w.y|'
    includes it.  On the -y axis, orbits of y <- y^n + y0 shrink and grow again;
    wherever the last iterate is the smallest, the two orders of the update give
    different minima, and the oracle must give the listing's."""
    s = W.bulb_1080p(0, 8, 8)
    checked = 0
    for n in (2, 3, 8):
        for y0 in np.linspace(-1.2, -0.05, 24):
            for trips in range(1, 13):
                ys = [float(y0)]
                for _ in range(trips):
                    ys.append(ys[-1] ** n + float(y0))
                    if abs(ys[-1]) > s["bailout"]:
                        break
                if abs(ys[-1]) > s["bailout"]:
                    continue  # escaped: then the final m is the largest and the orders agree
                m = [y * y for y in ys]
                old_m, new_m = min(m[:-1]), min(m)
                if abs(old_m - new_m) <= 1e-3 * new_m:
                    continue
                s.update(n=n, max_iter=trips)
                t = orc.trap(s, [0.0, y0, 0.0])
                assert abs(t[3] - old_m) <= 1e-12 * old_m, (n, y0, trips, t, old_m, new_m)
                assert abs(t[1] - min(abs(y) for y in ys)) <= 1e-12, (n, y0, trips, t)
                assert abs(t[0] - m[-1]) <= 1e-12 * max(1.0, m[-1])
                checked += 1
    assert checked > 30


@pytest.mark.parametrize("n", [2, 3, 5, 8, 9])
def test_bulb_de_derivative_on_polar_axis(orc, n):
    """On the +y axis Eq. 1 is the real map y <- y^n + y0 (polar angle 0), every
    iterate stays positive, and the listing's running derivative
    dz <- n |w|^(n-1) dz + 1 from dz = 1 is exactly d y_N / d y0 (the '+1' because
    c = y0 enters every step, |w| taken before the step).  So the DE must equal
    0.25 log(m) sqrt(m) / (d y_N / d y0), the derivative of the real map over the
    oracle's own trip count taken by the complex step (Squire and Trapp, 1998:
    f'(x) = Im f(x + i h) / h up to h^2, with no cancellation), in Python's
    complex arithmetic; dropping the '+1', or taking |w| after the step, changes
    the DE by 10 % or more."""
    s = W.bulb_1080p(0, 8, 8)
    s["n"] = n
    ys = np.concatenate([np.linspace(0.05, 0.6, 12), np.linspace(0.62, 1.6, 24)])
    d, _, trips, m2 = orc.de(s, np.stack([0 * ys, ys, 0 * ys], 1))
    for y0, dd, N, mm in zip(ys, d, trips, m2):
        h = 1e-30
        deriv = _axis_orbit(complex(float(y0), h), n, int(N)).imag / h
        m = _axis_orbit(float(y0), n, int(N)) ** 2
        assert abs(mm - m) <= 1e-12 * m
        want = 0.25 * math.log(m) * math.sqrt(m) / deriv
        assert abs(dd - want) <= 1e-9 * abs(want), (n, y0, N, dd, want)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 9])
def test_bulb_de_brackets_axis_distance(orc, n):
    """The set meets the +y axis in [0, y*], y* the largest y0 whose orbit of 0
    under y <- y^n + y0 stays bounded (found here by bisection on the real map).
    The distance from (0, y0, 0) to the set is therefore at most y0 - y*, and the
    DE, a lower bound on that distance (Sec. 2), may not exceed it.  There is no
    theorem for a lower bracket in 3D; over this sweep (y0 - y*) / DE stays in
    [1.6, 32] for every power, and the test holds it inside [1, 40]."""
    s = W.bulb_1080p(0, 8, 8)
    s["n"] = n

    def bounded(c):
        y = 0.0
        for _ in range(20000):
            y = y**n + c
            if y > 2.0:
                return False
        return True

    lo, hi = 0.0, 2.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if bounded(mid) else (lo, mid)
    y_star = hi
    ys = np.linspace(y_star + 1e-3, 2.0, 200)
    d, _, _, _ = orc.de(s, np.stack([0 * ys, ys, 0 * ys], 1))
    gap = ys - y_star
    assert np.all(d <= gap)
    pos = d > 0  # just outside y*, 12 steps do not tell the orbit from a bounded one
    assert pos.mean() > 0.9
    ratio = gap[pos] / d[pos]
    assert ratio.min() >= 1.0 and ratio.max() <= 40.0, (ratio.min(), ratio.max())


# ------------------------------------------------------ analytic normal (Sec. 2)
@pytest.mark.parametrize("p", [2, 3])
def test_analytic_normal_reduces_to_complex_derivative(orc, p):
    """On span{1, i} with c there too, grad log|z_N| is conj(dz_N/dz_0) z_N in the
    (x, y) plane (the chain rule D <- p z^(p-1) D in complex arithmetic) and 0
    along z; degree 3 with the listing's escape |z|^2 > 256."""
    rng = np.random.default_rng(41)
    s = W.julia_256(8, 8)
    s["normal_mode"] = "analytic"
    s["p"] = p
    if p == 3:
        s["escape_r2"] = 256.0
    c = complex(-0.2, 0.6) if p == 2 else complex(0.1, 0.55)
    s["c"] = (c.real, c.imag, 0.0, 0.0)
    for x, y in rng.uniform(-1.2, 1.2, (300, 2)):
        z, D = complex(x, y), 1.0 + 0j
        for _ in range(s["max_iter"]):
            D = p * z ** (p - 1) * D
            z = z ** p + c
            if abs(z) ** 2 > s["escape_r2"]:
                break
        g = D.conjugate() * z
        want = np.array([g.real, g.imag, 0.0]) / abs(g)
        got = orc.normal_scene(s, [x, y, 0.0])
        assert np.allclose(got, want, rtol=0, atol=1e-9)


@pytest.mark.parametrize("p", [2, 3])
def test_analytic_normal_matches_fine_central_differences(orc, p):
    """grad d = (grad G |grad G| - G grad|grad G|) / |grad G|^2 (Sec. 2) tends to
    grad G / |grad G| as G -> 0: at the hit points (d < eps) the analytic normal
    mostly agrees with a fine central-difference gradient of the DE; where the
    orbit has not escaped within the cap the two part ways, so the bar is on the
    median and on the majority, not on every point."""
    s = W.julia_256(8, 8)
    s.update(p=p, escape_r2=256.0 if p == 3 else 16.0, max_iter=12)
    r = orc.render(W.resized(dict(s, normal_mode="central", normal_h=1e-6), 24, 24), precision="f64")
    hits = np.flatnonzero((r["flags"] & 1) > 0)
    assert len(hits) > 50
    cos = []
    for idx in hits:
        ro, rd = orc.camera_ray(W.resized(s, 24, 24), idx % 24, idx // 24)
        x = ro + r["depth64"][idx] * rd
        a = orc.normal_scene(dict(s, normal_mode="analytic"), x, rd)
        b = orc.normal_scene(dict(s, normal_mode="central", normal_h=1e-7), x, rd)
        cos.append(a @ b)
    cos = np.array(cos)
    assert np.median(cos) > 0.99 and np.mean(cos > 0.99) >= 0.6


# ------------------------------------------- c = 0: the Julia set is the unit ball
@pytest.mark.parametrize("p, mode", [(2, "central"), (3, "tetra"), (2, "analytic")])
def test_c_zero_julia_set_is_unit_ball(orc, p, mode):
    """With c = 0 the orbit is z^(p^k), bounded exactly for |z| <= 1: the Julia set
    is the unit ball and the slice w = 0 the unit sphere.  Its DE near the sphere is
    (1/2)|z| log|z| (half the distance, Eq. 2 with the listings' 1/2), so the march
    stops within about 2 eps of the sphere: depth = the ray's entry into the unit
    sphere, and the normal is radial."""
    s = W.julia_256(40, 30)
    s.update(c=(0.0, 0.0, 0.0, 0.0), p=p, normal_mode=mode, max_iter=30,
             escape_r2=16.0 if p == 2 else 256.0)
    o = orc.render(s, precision="f64", threads=4)
    n_hit = 0
    for idx in range(40 * 30):
        ro, rd = orc.camera_ray(s, idx % 40, idx // 40)
        b = ro @ rd
        disc = b * b - (ro @ ro - 1.0)
        if disc < 0.02:  # misses, and grazing rays whose entry is ill-conditioned
            assert disc >= 0.0 or not np.isfinite(o["depth64"][idx])
            continue
        t_sphere = -b - math.sqrt(disc)
        cos_in = math.sqrt(disc)  # |rd . n| at the entry point of a unit sphere
        assert o["flags"][idx] & 1
        assert 0.0 <= t_sphere - o["depth64"][idx] <= 2.5 * s["eps"] / cos_in, idx
        x = ro + o["depth64"][idx] * rd
        nrm = orc.normal_scene(s, x, rd)
        assert nrm @ (x / np.linalg.norm(x)) > 0.999, (idx, nrm)
        n_hit += 1
    assert n_hit > 300


# ------------------------------------------- Mandelbulb: symmetry and analytic normal
def _rot_y(theta):
    c, s = math.cos(theta), math.sin(theta)
    # the listing's azimuth a = atan2(x, z): a rotation about +y adds theta to a
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


@pytest.mark.parametrize("n", [8, 3, 5])
def test_bulb_rotation_symmetry(orc, n):
    """Eq. 1 multiplies the azimuth by n, so w -> w^n + c commutes with rotations
    about the polar axis by 2 pi / (n - 1): the Mandelbulb, its DE and its analytic
    normal are symmetric under them (the normal rotates with the point)."""
    s = W.bulb_1080p(0, 8, 8)
    s.update(n=n, normal_mode="analytic", max_iter=10)
    rot = _rot_y(2 * math.pi / (n - 1))
    rng = np.random.default_rng(14)
    pts = rng.uniform(-1.2, 1.2, (300, 3))
    d0, n0, _, _ = orc.de(s, pts)
    d1, n1, _, _ = orc.de(s, pts @ rot.T)
    same = n0 == n1
    assert np.mean(same) > 0.98
    assert np.allclose(d0[same], d1[same], rtol=1e-9, atol=1e-12)
    for p in pts[same][:80]:
        a = orc.normal_scene(s, p)
        b = orc.normal_scene(s, rot @ p)
        assert np.allclose(rot @ a, b, rtol=0, atol=1e-8), (p, rot @ a, b)


@pytest.mark.parametrize("n", [8, 3])
def test_bulb_analytic_normal_is_the_potential_gradient(orc, n):
    """The analytic normal is the direction of grad log|w_N| (w_N the orbit's last
    iterate): checked against central differences of log|w_N|^2 from the DE's own
    orbit at points whose iteration count is the same at every tap.  (It is not
    the direction of the DE's gradient: the Mandelbulb listing's DE carries a
    scalar derivative, so its level sets tilt by a few degrees against the
    potential's.)"""
    s = W.bulb_1080p(0, 8, 8)
    s.update(n=n, normal_mode="analytic", max_iter=12)
    rng = np.random.default_rng(15)
    dirs = rng.standard_normal((400, 3))
    pts = dirs / np.linalg.norm(dirs, axis=1)[:, None] * rng.uniform(0.8, 1.4, (400, 1))
    h = 1e-6
    good = agree = 0
    for p in pts:
        d0, n0, tr0, m0 = orc.de(s, [p])
        g = np.zeros(3)
        ok = True
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            _, _, trp, mp = orc.de(s, [p + e])
            _, _, trm, mm = orc.de(s, [p - e])
            ok &= trp[0] == tr0[0] and trm[0] == tr0[0]
            g[j] = (math.log(mp[0]) - math.log(mm[0])) / (2 * h)
        if not ok or not np.all(np.isfinite(g)):
            continue
        good += 1
        a = orc.normal_scene(s, p)
        agree += (a @ g / np.linalg.norm(g)) > 1 - 1e-7
    assert good > 200 and agree / good >= 0.99, (good, agree)
