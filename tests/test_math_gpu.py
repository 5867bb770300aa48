"""The distance estimators' own elementary functions (fr_math.cuh: atan2pi,
acospi, sincospi_own, quot, sqrt_own, sqrt_rsqrt_own, log_own) against double precision on
the device: the error bounds
the header states, and the library routines they replaced measured beside
them on the same arguments (tests/math_probe/math_probe.cu)."""
import math
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2102_01747_gb300", "csrc")


def _run_probe():
    from paper_2102_01747_gb300 import build as B

    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "math_probe")
        subprocess.run([B.nvcc(), "-O3", "-std=c++17", *B.ARCH, "-I", CSRC,
                        os.path.join(HERE, "math_probe", "math_probe.cu"), "-o", exe],
                       check=True, capture_output=True, text=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = dict(kv.split("=", 1) for kv in r.stdout.split())
    special = [float(v) for v in out.pop("special").split(",")]
    return {k: float(v) for k, v in out.items()}, special


def test_math_routines_error_bounds():
    m, sp = _run_probe()
    # the angles, in ulps of the result and absolutely (half-turns)
    assert m["atan2pi_ulp"] <= 3.0 and m["atan2pi_abs_e6"] <= 0.08, m
    assert m["acospi_ulp"] <= 3.0 and m["acospi_abs_e6"] <= 0.09, m
    # no worse than the library routines they replaced, scaled to half-turns, by more than 0.5 ulp
    assert m["atan2pi_ulp"] <= m["atan2f_ulp"] + 0.5 and m["acospi_ulp"] <= m["acosf_ulp"] + 0.5, m
    # sin and cos of pi x on [-16, 16]
    assert m["sinpi_abs_e6"] <= 0.09 and m["cospi_abs_e6"] <= 0.09, m
    assert m["quot_ulp"] <= 1.0 and m["sqrt_own_ulp"] <= 1.0, m
    assert m["log_own_ulp"] <= 2.0 and m["rsqrt_own_ulp"] <= 1.5, m
    # atan2 of signed zeros as IEEE atan2 has them, exact axis and diagonal values
    assert sp[:10] == [0.0, -0.0, 1.0, -1.0, 0.5, 1.0, 0.25, 0.0, 1.0, 0.5], sp
    assert [math.copysign(1.0, v) for v in sp[:4]] == [1.0, -1.0, 1.0, -1.0], sp
    assert [abs(v) for v in sp[10:14]] == [0.0, 1.0, 1.0, 0.0], sp  # sin, cos of 8 pi and of -1.5 pi
    # sqrt of 0, 4 and a subnormal (taken as 0); log of 1, 0 (taken as the smallest normal) and 2
    assert sp[14:18] == [0.0, 2.0, 0.0, 0.0], sp
    assert abs(sp[18] - math.log(2.0 ** -126)) < 1e-5 and abs(sp[19] - math.log(2.0)) < 1e-7, sp
