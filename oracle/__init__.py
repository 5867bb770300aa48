"""CPU oracle for distance-estimated sphere tracing of quaternion Julia sets and
the Mandelbulb -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, the package's smoke() check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
path: the C sources here (fr_oracle.c and the two .inc bodies) are compiled
with gcc into their own shared library, loaded with ctypes.

Scenes are the plain dicts produced by the seeded input generators
(paper_2102_01747_gb300.workloads); this wrapper turns them into the
oracle's own parameter struct.  Every routine exists at two precisions:
"f64" (the reference) and "f32" (the same steps in float, for tolerance
studies and for the closest comparison with the float GPU path).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = ["fr_oracle.c", "fr_oracle_body.inc", "fr_oracle_grad.inc", "fr_oracle.h"]

JULIA, BULB = 0, 1
NORMAL_TETRA, NORMAL_CENTRAL, NORMAL_ANALYTIC = 0, 1, 2
SHADE_LAMBERT, SHADE_PHONG = 0, 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fused multiply-add, no fast math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(os.path.join(HERE, s)) for s in SOURCES)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, os.path.join(HERE, "fr_oracle.c"), "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrcScene(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("c", ctypes.c_double * 4),
        ("p", ctypes.c_int),
        ("slice_w", ctypes.c_double),
        ("escape_r2", ctypes.c_double),
        ("n", ctypes.c_int),
        ("bailout", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("bound_radius", ctypes.c_double),
        ("max_steps", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("max_step", ctypes.c_double),
        ("normal_mode", ctypes.c_int),
        ("normal_h", ctypes.c_double),
        ("plane_enabled", ctypes.c_int),
        ("plane_n", ctypes.c_double * 3),
        ("plane_o", ctypes.c_double),
        ("eye", ctypes.c_double * 3),
        ("target", ctypes.c_double * 3),
        ("up", ctypes.c_double * 3),
        ("fov_y_deg", ctypes.c_double),
        ("width", ctypes.c_int),
        ("height", ctypes.c_int),
        ("spp", ctypes.c_int),
        ("seed", ctypes.c_uint32),
        ("light_dir", ctypes.c_double * 3),
        ("albedo", ctypes.c_double * 3),
        ("k_ambient", ctypes.c_double),
        ("k_diffuse", ctypes.c_double),
        ("shadows", ctypes.c_int),
        ("background", ctypes.c_double * 4),
        ("shading", ctypes.c_int),
        ("k_specular", ctypes.c_double),
        ("shininess", ctypes.c_double),
        ("reflect_coef", ctypes.c_double),
    ]


class OrcOutputs(ctypes.Structure):
    _fields_ = [
        ("rgba", ctypes.c_void_p),
        ("rgba8", ctypes.c_void_p),
        ("depth", ctypes.c_void_p),
        ("flags", ctypes.c_void_p),
        ("stats", ctypes.c_void_p),
        ("rgba64", ctypes.c_void_p),
        ("depth64", ctypes.c_void_p),
        ("trap", ctypes.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        d, f, i, i64 = ctypes.c_double, ctypes.c_float, ctypes.c_int, ctypes.c_int64
        pd, pf, pi = P(d), P(f), P(i)
        for sfx, pr, r in (("d", pd, d), ("f", pf, f)):
            getattr(L, "orc_render_" + sfx).argtypes = [P(OrcScene), P(i64), i64, P(OrcOutputs), i]
            getattr(L, "orc_render_" + sfx).restype = i
            getattr(L, "orc_qmul_" + sfx).argtypes = [pr, pr, pr]
            getattr(L, "orc_bulb_pow_" + sfx).argtypes = [pr, i, pr]
            getattr(L, "orc_de_" + sfx).argtypes = [P(OrcScene), pr, pi, pi, pr]
            getattr(L, "orc_de_" + sfx).restype = r
            getattr(L, "orc_camera_ray_" + sfx).argtypes = [P(OrcScene), i, i, i, pr, pr]
            getattr(L, "orc_trap_" + sfx).argtypes = [P(OrcScene), pr, pr]
            getattr(L, "orc_normal_scene_" + sfx).argtypes = [P(OrcScene), pr, pr, pr]
            getattr(L, "orc_quantize_" + sfx).argtypes = [r]
            getattr(L, "orc_quantize_" + sfx).restype = ctypes.c_uint32
        L.orc_qpow_d.argtypes = [pd, i, pd]
        L.orc_julia2d_escape_d.argtypes = [d, d, d, d, i, d]
        L.orc_julia2d_escape_d.restype = i
        L.orc_bounds_d.argtypes = [P(OrcScene), pd, pd, pd, pd, pi]
        L.orc_bounds_d.restype = i
        L.orc_splitmix64.argtypes = [ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_jitter.argtypes = [ctypes.c_uint32, i64, i, i, pd, pd]
        L.orc_march_field_d.argtypes = [i, pd, pd, pd, d, d, i, d, d, pd, pi]
        L.orc_march_field_d.restype = i
        L.orc_normal_field_d.argtypes = [i, pd, pd, i, d, pd, pd]
        L.orc_shade_d.argtypes = [P(OrcScene), pd, d, pd]
        L.orc_shade_phong_d.argtypes = [P(OrcScene), pd, pd, d, pd, pd]
        for fn in (L.orc_julia_grad_d, L.orc_bulb_grad_d):
            fn.argtypes = [P(OrcScene), pd, pd, ctypes.c_void_p, pd, i]
            fn.restype = i
        _lib = L
    return _lib


def _arr(x, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def _ptr(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def scene_struct(scene: dict) -> OrcScene:
    s = OrcScene()
    s.kind = JULIA if scene["kind"] == "julia" else BULB
    s.c[:] = [float(v) for v in scene["c"]]
    s.p = int(scene["p"])
    s.slice_w = float(scene["slice_w"])
    s.escape_r2 = float(scene["escape_r2"])
    s.n = int(scene["n"])
    s.bailout = float(scene["bailout"])
    s.max_iter = int(scene["max_iter"])
    s.bound_radius = float(scene["bound_radius"])
    s.max_steps = int(scene["max_steps"])
    s.eps = float(scene["eps"])
    s.max_step = float(scene["max_step"])
    s.normal_mode = {"tetra": NORMAL_TETRA, "central": NORMAL_CENTRAL,
                     "analytic": NORMAL_ANALYTIC}[scene["normal_mode"]]
    s.normal_h = float(scene["normal_h"])
    pl = scene.get("plane")
    s.plane_enabled = 1 if pl else 0
    if pl:
        s.plane_n[:] = [float(v) for v in pl["n"]]
        s.plane_o = float(pl["o"])
    cam = scene["camera"]
    s.eye[:] = [float(v) for v in cam["eye"]]
    s.target[:] = [float(v) for v in cam["target"]]
    s.up[:] = [float(v) for v in cam["up"]]
    s.fov_y_deg = float(cam["fov_y_deg"])
    s.width, s.height, s.spp = int(cam["width"]), int(cam["height"]), int(cam["spp"])
    s.seed = int(cam["seed"]) & 0xFFFFFFFF
    li = scene["light"]
    s.light_dir[:] = [float(v) for v in li["dir"]]
    s.albedo[:] = [float(v) for v in li["albedo"]]
    s.k_ambient = float(li["k_ambient"])
    s.k_diffuse = float(li["k_diffuse"])
    s.shadows = 1 if li["shadows"] else 0
    s.background[:] = [float(v) for v in li["background"]]
    s.shading = {"lambert": SHADE_LAMBERT, "phong": SHADE_PHONG}[li.get("shading", "lambert")]
    s.k_specular = float(li.get("k_specular", 0.0))
    s.shininess = float(li.get("shininess", 1.0))
    s.reflect_coef = float(li.get("reflect_coef", 0.0))
    return s


def render(scene: dict, pixels=None, precision: str = "f32", threads: int = 1) -> dict:
    """Render the listed pixels (linear indices y*W + x; None = whole image).

    Returns numpy arrays: rgba (n,4) float32 mean colour, rgba8 (n,) uint32,
    depth (n,) float32 (+inf on a miss), flags (n,) int32 (1 hit, 2 cut face,
    4 shadowed), stats (n,7) int64 (primary DE calls, normal DE calls, shadow DE
    calls, orbit iterations, shadow rays, reflection DE calls, reflection
    rays), trap (n,4) float32 orbit-trap colour
    parameters at the nearest hit, and for f64 also rgba64 / depth64."""
    L = lib()
    s = scene_struct(scene)
    if pixels is None:
        n = s.width * s.height
        px = None
    else:
        px = _arr(pixels, np.int64)
        n = px.size
    res = {
        "rgba": np.zeros((n, 4), np.float32),
        "rgba8": np.zeros(n, np.uint32),
        "depth": np.zeros(n, np.float32),
        "flags": np.zeros(n, np.int32),
        "stats": np.zeros((n, 7), np.int64),
        "trap": np.zeros((n, 4), np.float32),
    }
    out = OrcOutputs(res["rgba"].ctypes.data, res["rgba8"].ctypes.data, res["depth"].ctypes.data,
                     res["flags"].ctypes.data, res["stats"].ctypes.data, None, None,
                     res["trap"].ctypes.data)
    if precision == "f64":
        res["rgba64"] = np.zeros((n, 4), np.float64)
        res["depth64"] = np.zeros(n, np.float64)
        out.rgba64 = res["rgba64"].ctypes.data
        out.depth64 = res["depth64"].ctypes.data
    fn = L.orc_render_d if precision == "f64" else L.orc_render_f
    rc = fn(ctypes.byref(s), None if px is None else _ptr(px, ctypes.c_int64), n, ctypes.byref(out),
            int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the scene")
    return res


def de(scene: dict, points, precision: str = "f64"):
    """Distance estimate at each 3D point: (d, n_nonescaping, trips, m2)."""
    L = lib()
    s = scene_struct(scene)
    pts = np.asarray(points, np.float64).reshape(-1, 3)
    k = pts.shape[0]
    dt = np.float64 if precision == "f64" else np.float32
    ct = ctypes.c_double if precision == "f64" else ctypes.c_float
    fn = L.orc_de_d if precision == "f64" else L.orc_de_f
    d = np.zeros(k, dt)
    m2 = np.zeros(k, dt)
    nn = np.zeros(k, np.int32)
    tr = np.zeros(k, np.int32)
    pc = np.ascontiguousarray(pts.astype(dt))
    ni, ti, mv = ctypes.c_int(), ctypes.c_int(), ct()
    for j in range(k):
        d[j] = fn(ctypes.byref(s), _ptr(pc[j], ct), ctypes.byref(ni), ctypes.byref(ti), ctypes.byref(mv))
        nn[j], tr[j], m2[j] = ni.value, ti.value, mv.value
    return d, nn, tr, m2


def qmul(a, b, precision: str = "f64"):
    dt, ct = (np.float64, ctypes.c_double) if precision == "f64" else (np.float32, ctypes.c_float)
    fn = lib().orc_qmul_d if precision == "f64" else lib().orc_qmul_f
    a, b = _arr(a, dt), _arr(b, dt)
    o = np.zeros(4, dt)
    fn(_ptr(a, ct), _ptr(b, ct), _ptr(o, ct))
    return o


def qpow(q, p):
    q = _arr(q)
    o = np.zeros(4)
    lib().orc_qpow_d(_ptr(q), int(p), _ptr(o))
    return o


def bulb_pow(v, n, precision: str = "f64"):
    dt, ct = (np.float64, ctypes.c_double) if precision == "f64" else (np.float32, ctypes.c_float)
    fn = lib().orc_bulb_pow_d if precision == "f64" else lib().orc_bulb_pow_f
    v = _arr(v, dt)
    o = np.zeros(3, dt)
    fn(_ptr(v, ct), int(n), _ptr(o, ct))
    return o


def julia2d_escape(z, c, max_iter, escape_r2):
    return lib().orc_julia2d_escape_d(z.real, z.imag, c.real, c.imag, int(max_iter), float(escape_r2))


def bounds(scene, ro, rd):
    """(non-empty, t0, t1, from_plane) of the search interval."""
    s = scene_struct(scene)
    ro, rd = _arr(ro), _arr(rd)
    t0, t1, fp = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    ok = lib().orc_bounds_d(ctypes.byref(s), _ptr(ro), _ptr(rd), ctypes.byref(t0), ctypes.byref(t1),
                            ctypes.byref(fp))
    return bool(ok), t0.value, t1.value, bool(fp.value)


def camera_ray(scene, px, py, sample=0, precision: str = "f64"):
    s = scene_struct(scene)
    dt, ct = (np.float64, ctypes.c_double) if precision == "f64" else (np.float32, ctypes.c_float)
    fn = lib().orc_camera_ray_d if precision == "f64" else lib().orc_camera_ray_f
    ro, rd = np.zeros(3, dt), np.zeros(3, dt)
    fn(ctypes.byref(s), int(px), int(py), int(sample), _ptr(ro, ct), _ptr(rd, ct))
    return ro, rd


def splitmix64(state: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(state & 0xFFFFFFFFFFFFFFFF)))


def jitter(seed, pixel, spp, sample):
    sx, sy = ctypes.c_double(), ctypes.c_double()
    lib().orc_jitter(int(seed) & 0xFFFFFFFF, int(pixel), int(spp), int(sample), ctypes.byref(sx),
                     ctypes.byref(sy))
    return sx.value, sy.value


def march_field(kind, prm, ro, rd, t0, t1, max_steps, eps, max_step):
    """March a test field (0 sphere, 1 affine, 2 quadratic): (hit, t, steps)."""
    prm, ro, rd = _arr(prm), _arr(ro), _arr(rd)
    t, st = ctypes.c_double(), ctypes.c_int()
    hit = lib().orc_march_field_d(int(kind), _ptr(prm), _ptr(ro), _ptr(rd), float(t0), float(t1),
                                  int(max_steps), float(eps), float(max_step), ctypes.byref(t),
                                  ctypes.byref(st))
    return bool(hit), t.value, st.value


def normal_field(kind, prm, p, mode, h, rd=(0.0, 0.0, -1.0)):
    prm, p, rd = _arr(prm), _arr(p), _arr(rd)
    o = np.zeros(3)
    lib().orc_normal_field_d(int(kind), _ptr(prm), _ptr(p), int(mode), float(h), _ptr(rd), _ptr(o))
    return o


def shade(scene, n, vis=1.0):
    s = scene_struct(scene)
    n = _arr(n)
    o = np.zeros(4)
    lib().orc_shade_d(ctypes.byref(s), _ptr(n), float(vis), _ptr(o))
    return o


def shade_phong(scene, n, rd, vis=1.0, refl=(0.0, 0.0, 0.0)):
    """Phong colour of a hit with normal n seen along rd (visibility vis), plus
    reflect_coef * Fresnel-Schlick * refl (the colour along the mirror ray)."""
    s = scene_struct(scene)
    n, rd, refl = _arr(n), _arr(rd), _arr(refl)
    o = np.zeros(4)
    lib().orc_shade_phong_d(ctypes.byref(s), _ptr(n), _ptr(rd), float(vis), _ptr(refl), _ptr(o))
    return o


def normal_scene(scene, p, rd=(0.0, 0.0, -1.0), precision: str = "f64"):
    """Unit normal at p by the scene's normal mode."""
    dt, ct = (np.float64, ctypes.c_double) if precision == "f64" else (np.float32, ctypes.c_float)
    fn = lib().orc_normal_scene_d if precision == "f64" else lib().orc_normal_scene_f
    s = scene_struct(scene)
    pp, rr = _arr(p, dt), _arr(rd, dt)
    o = np.zeros(3, dt)
    fn(ctypes.byref(s), _ptr(pp, ct), _ptr(rr, ct), _ptr(o, ct))
    return o


def trap(scene, p, precision: str = "f64"):
    """Orbit-trap colour parameters of the DE at point p."""
    dt, ct = (np.float64, ctypes.c_double) if precision == "f64" else (np.float32, ctypes.c_float)
    fn = lib().orc_trap_d if precision == "f64" else lib().orc_trap_f
    s = scene_struct(scene)
    pp = _arr(p, dt)
    o = np.zeros(4, dt)
    fn(ctypes.byref(s), _ptr(pp, ct), _ptr(o, ct))
    return o


def quantize(x, precision: str = "f64") -> int:
    fn = lib().orc_quantize_d if precision == "f64" else lib().orc_quantize_f
    return int(fn(x))


def julia_grad(scene: dict, d_rgba, d_depth=None, mask=None, threads: int = 1) -> np.ndarray:
    """Reference vector-Jacobian product of the Julia render (double, forward-mode
    dual numbers, implicit differentiation at the hit).  Returns the 11-vector
    (dc[4], dplane_n[3], dplane_o, dlight_dir[3]).  A Mandelbulb scene gives
    the same vector with dc = 0 (the fractal has no parameter c)."""
    s = scene_struct(scene)
    W, H = s.width, s.height
    dr = _arr(d_rgba).reshape(W * H * 4)
    dd = None if d_depth is None else _arr(d_depth).reshape(W * H)
    mk = None if mask is None else np.ascontiguousarray(np.asarray(mask, np.uint8).reshape(W * H))
    g = np.zeros(11)
    fn = lib().orc_julia_grad_d if scene["kind"] == "julia" else lib().orc_bulb_grad_d
    rc = fn(ctypes.byref(s), _ptr(dr), None if dd is None else _ptr(dd),
                                None if mk is None else mk.ctypes.data, _ptr(g), int(threads))
    if rc != 0:
        raise ValueError("oracle gradient rejected the scene")
    return g
