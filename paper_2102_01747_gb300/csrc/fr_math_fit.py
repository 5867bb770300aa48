"""Regenerate the polynomial coefficients of fr_math.cuh (not run at build time).

Each polynomial is a relative-error minimax fit found by the Remez exchange
algorithm in 40-digit arithmetic (mpmath), then rounded to float:

  atan(q) / (pi q)        = P(s), s = q^2 in [0, 1],     degree 8
  asin(s) / (pi s)        = Q(u), u = s^2 in [0, 1/4],   degree 5
  sin(pi f) / f           = S(v), v = f^2 in [0, 1/16],  degree 3
  (cos(pi f) - 1) / f^2   = C(v), v = f^2 in [0, 1/16],  degree 3

The Remez exchange: start from Chebyshev extrema, solve the linear system
p(x_i) + (-1)^i E f(x_i) = f(x_i) for the coefficients and the levelled error
E, move the reference points to the alternating extrema of the relative
error p / f - 1 on a dense grid, and repeat until the points settle.

    python fr_math_fit.py      # prints the coefficients, highest degree first
"""
import mpmath as mp

mp.mp.dps = 40


def remez(f, a, b, deg, iters=30, grid=4000):
    a, b = mp.mpf(a), mp.mpf(b)
    n = deg + 2
    xs = [a + (b - a) * (1 - mp.cos(mp.pi * i / (n - 1))) / 2 for i in range(n)]
    pts = [a + (b - a) * k / grid for k in range(grid + 1)]
    for _ in range(iters):
        A = mp.matrix(n, n)
        rhs = mp.matrix(n, 1)
        for i, x in enumerate(xs):
            for j in range(deg + 1):
                A[i, j] = x ** j
            A[i, deg + 1] = (-1) ** i * f(x)
            rhs[i] = f(x)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(deg + 1)]
        ev = [(mp.polyval(c[::-1], x) - f(x)) / f(x) for x in pts]
        ext = [k for k in range(len(pts))
               if k in (0, len(pts) - 1) or (ev[k] - ev[k - 1]) * (ev[k + 1] - ev[k]) <= 0]
        alt = []
        for k in ext:  # keep the largest of each run of equal sign
            if alt and mp.sign(ev[k]) == mp.sign(ev[alt[-1]]):
                if abs(ev[k]) > abs(ev[alt[-1]]):
                    alt[-1] = k
            else:
                alt.append(k)
        while len(alt) > n:  # drop the smaller end
            alt.pop(0 if abs(ev[alt[0]]) < abs(ev[alt[-1]]) else -1)
        if len(alt) < n:
            break
        new = [pts[k] for k in alt]
        if new == xs:  # the reference has settled: the next solve gives the same polynomial
            break
        xs = new
    return c, max(abs(e) for e in ev)


def atan_over_pi(s):
    return mp.atan(mp.sqrt(s)) / (mp.pi * mp.sqrt(s)) if s > 0 else 1 / mp.pi


def asin_over_pi(u):
    return mp.asin(mp.sqrt(u)) / (mp.pi * mp.sqrt(u)) if u > 0 else 1 / mp.pi


def sin_pi_over_f(v):
    return mp.sin(mp.pi * mp.sqrt(v)) / mp.sqrt(v) if v > 0 else mp.pi


def cos_pi_m1_over_f2(v):
    return (mp.cos(mp.pi * mp.sqrt(v)) - 1) / v if v > 0 else -mp.pi ** 2 / 2


def to_float(x):
    import struct
    return struct.unpack("f", struct.pack("f", float(x)))[0]


if __name__ == "__main__":
    for name, f, lo, hi, deg in (("atan2pi P(q^2)", atan_over_pi, 0, 1, 8),
                                 ("acospi Q(s^2)", asin_over_pi, 0, 0.25, 5),
                                 ("sincospi_own S(f^2)", sin_pi_over_f, 0, mp.mpf(1) / 16, 3),
                                 ("sincospi_own C(f^2)", cos_pi_m1_over_f2, 0, mp.mpf(1) / 16, 3)):
        c, err = remez(f, lo, hi, deg)
        print("%s: degree %d, relative error %.3e before rounding" % (name, deg, float(err)))
        for x in c[::-1]:
            print("    %r" % to_float(x))
