"""The distance estimators' elementary functions (paper_2102_01747_gb300/csrc/
fr_math.cuh) replayed on the host: the polynomial coefficients are read from
the header, each routine's steps are redone in float32 with fused
multiply-adds emulated in double (a float product is exact in double, and the
sum is rounded once more to float), the hardware reciprocal and reciprocal-
square-root seeds taken as correctly rounded, and the results compared with
numpy's double-precision functions.  This pins the algorithms and their
constants without a GPU; tests/test_math_gpu.py measures the compiled
routines on the device.  The coefficients are also checked against a fresh
Remez fit by fr_math_fit.py where mpmath is installed."""
import math
import os
import re
import subprocess
import sys

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2102_01747_gb300", "csrc")
HEADER = open(os.path.join(CSRC, "fr_math.cuh")).read()
F32 = np.float32


def _body(name):
    """The source of the device routine `name` in the header."""
    i = re.search(r"__forceinline__ \w+ %s\(" % name, HEADER).start()
    return HEADER[i:HEADER.index("\n}\n", i)]


def _horner(body, acc):
    """[c_n, ..., c_0] of `acc = c_n; acc = fmaf(acc, v, c_k)` in a routine body."""
    first = re.search(r"float %s = (-?[0-9.e+-]+)f;" % acc, body)
    rest = re.findall(r"%s = fmaf\(%s, \w+, (-?[0-9.e+-]+)f\);" % (acc, acc), body)
    return [float(first.group(1))] + [float(c) for c in rest]


def fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def mul(a, b):
    with np.errstate(invalid="ignore"):  # 0 * inf of the reciprocal-square-root seed at x = 0
        return (np.asarray(a, F32) * np.asarray(b, F32)).astype(F32)


def horner(coefs, v):
    p = np.full(np.shape(v), F32(coefs[0]), F32)
    for c in coefs[1:]:
        p = fma(p, v, F32(c))
    return p


def quot(y, x):
    r = (1.0 / np.asarray(x, np.float64)).astype(F32)
    q = mul(y, r)
    e = fma(-np.asarray(x, F32), q, y)
    return fma(e, r, q)


def sqrt_rsqrt(x):
    x = np.asarray(x, F32)
    with np.errstate(divide="ignore"):
        y = (1.0 / np.sqrt(np.asarray(x, np.float64))).astype(F32)
    r = mul(x, y)
    hy = mul(F32(0.5), y)
    with np.errstate(invalid="ignore"):
        inv = fma(hy, fma(-r, y, F32(1.0)), y)
        q = fma(hy, fma(-r, r, x), r)
    return np.where(x >= F32(1.17549435e-38), q, F32(0.0)).astype(F32), inv


AT = _horner(_body("atan2pi"), "p")
AS = _horner(_body("acospi"), "p")
SN = _horner(_body("sincospi_own"), "ps")
CS = _horner(_body("sincospi_own"), "pc")
LG = _horner(_body("log_own"), "p")


def atan2pi(y, x):
    y, x = np.asarray(y, F32), np.asarray(x, F32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    q = quot(mn, np.maximum(mx, F32(1e-30)))
    t = mul(q, horner(AT, mul(q, q)))
    t = np.where(ay > ax, (F32(0.5) - t).astype(F32), t)
    t = np.where(np.signbit(x), (F32(1.0) - t).astype(F32), t)
    return np.copysign(t, y).astype(F32)


def acospi(x):
    x = np.asarray(x, F32)
    ax = np.abs(x)
    big = ax > F32(0.5)
    h = fma(F32(-0.5), ax, F32(0.5))
    s = np.where(big, sqrt_rsqrt(h)[0], ax)
    u = np.where(big, h, mul(ax, ax))
    a = mul(s, horner(AS, u))
    rbig = np.where(np.signbit(x), fma(F32(-2.0), a, F32(1.0)), mul(F32(2.0), a))
    rsmall = (F32(0.5) - np.copysign(a, x)).astype(F32)
    return np.where(big, rbig, rsmall).astype(F32)


def sincospi(x):
    x = np.asarray(x, F32)
    big = fma(x, F32(2.0), F32(12582912.0))
    j = (big - F32(12582912.0)).astype(F32)
    k = big.view(np.int32)
    f = fma(F32(-0.5), j, x)
    v = mul(f, f)
    sn = mul(f, horner(SN, v))
    cs = fma(horner(CS, v), v, F32(1.0))
    odd = (k & 1) == 1
    S, C = np.where(odd, cs, sn), np.where(odd, sn, cs)
    S = np.where((k & 2) != 0, -S, S).astype(F32)
    C = np.where(((k + 1) & 2) != 0, -C, C).astype(F32)
    return S, C


def log_own(x):
    i = np.maximum(np.asarray(x, F32), F32(1.17549435e-38)).view(np.int32).astype(np.int64)
    e = (i - 0x3f3504f3) >> 23
    f = (i - (e << 23)).astype(np.int32).view(F32)
    t = (f - F32(1.0)).astype(F32)
    sv = quot(t, (f + F32(1.0)).astype(F32))
    u = mul(sv, sv)
    lf = fma(sv, fma(u, horner(LG, u), -t), t)
    ef = e.astype(F32)
    return fma(ef, F32(0.693147182464599609375), fma(ef, F32(-1.9046542121259336e-09), lf))


def ulps(got, ref):
    ref = np.asarray(ref, np.float64)
    up = np.spacing(np.abs(ref).astype(F32)).astype(np.float64)
    return np.abs(np.asarray(got, np.float64) - ref) / up


RNG = np.random.default_rng(2102)


def test_atan2pi_error_and_signed_zeros():
    n = 400_000
    y = (RNG.uniform(-2, 2, n) * RNG.choice([1.0, 1e-3], n)).astype(F32)
    x = (RNG.uniform(-2, 2, n) * RNG.choice([1.0, 1e-3], n)).astype(F32)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64)) / math.pi
    assert ulps(atan2pi(y, x), ref).max() <= 3.0
    z = np.array([0.0, -0.0, 0.0, -0.0], F32)
    w = np.array([0.0, 0.0, -0.0, -0.0], F32)
    got = atan2pi(z, w)
    assert list(got) == [0.0, -0.0, 1.0, -1.0] and list(np.signbit(got)) == [False, True, False, True]
    assert list(atan2pi(np.array([1, 0, 1, -1], F32), np.array([0, -1, 1, -1], F32))) == [0.5, 1.0, 0.25, -0.75]


def test_acospi_error_and_ends():
    x = np.linspace(-1, 1, 400_001).astype(F32)
    assert ulps(acospi(x), np.arccos(x.astype(np.float64)) / math.pi).max() <= 3.0
    assert list(acospi(np.array([1, -1, 0], F32))) == [0.0, 1.0, 0.5]
    assert ulps(acospi(np.array([0.5, -0.5], F32)), np.array([1 / 3, 2 / 3])).max() <= 1.0


def test_sincospi_error_and_quarter_turns():
    x = np.linspace(-16, 16, 400_001).astype(F32)
    s, c = sincospi(x)
    xd = x.astype(np.float64)
    assert np.abs(s - np.sin(math.pi * xd)).max() <= 1e-7
    assert np.abs(c - np.cos(math.pi * xd)).max() <= 1e-7
    q = np.arange(-32, 33).astype(F32) * F32(0.5)  # multiples of a quarter turn
    s, c = sincospi(q)
    assert np.all(np.abs(s) == np.abs(np.round(np.sin(math.pi * q.astype(np.float64)))))
    assert np.all(np.abs(c) == np.abs(np.round(np.cos(math.pi * q.astype(np.float64)))))


def test_sqrt_log_quot():
    x = np.concatenate([np.exp2(RNG.uniform(-126, 20, 200_000)), RNG.uniform(0.5, 2.0, 200_000)]).astype(F32)
    r, inv = sqrt_rsqrt(x)
    xd = x.astype(np.float64)
    assert ulps(r, np.sqrt(xd)).max() <= 1.0
    assert ulps(inv, 1 / np.sqrt(xd)).max() <= 1.5
    assert ulps(log_own(x), np.log(xd)).max() <= 2.0
    y = RNG.uniform(-1, 1, 200_000).astype(F32)
    d = RNG.uniform(0.5, 2.0, 200_000).astype(F32)
    yy = np.where(np.abs(y) <= d, y, d).astype(F32)
    assert ulps(quot(yy, d), yy.astype(np.float64) / d.astype(np.float64)).max() <= 1.0
    assert list(sqrt_rsqrt(np.array([0.0, 4.0, 1e-40], F32))[0]) == [0.0, 2.0, 0.0]
    assert log_own(np.array([1.0], F32))[0] == 0.0


def test_coefficients_are_the_remez_fits():
    pytest.importorskip("mpmath")
    out = subprocess.run([sys.executable, os.path.join(CSRC, "fr_math_fit.py")], capture_output=True, text=True,
                         check=True, timeout=300).stdout
    fits = [[float(v) for v in re.findall(r"^\s+(-?[0-9.e+-]+)$", blk, re.M)] for blk in out.split(":")[1:]]
    assert [AT, AS, SN, CS] == fits[:4]
