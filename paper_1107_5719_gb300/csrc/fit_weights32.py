"""Fit the polynomials of the FP32 segment weights (weights.cuh, seg_weights32).

Below x = 2 the FP32 march evaluates the linear-source weights through
  phi2(+-x) = E(z) +- x Q(z),  z = x^2,
  E(z) = sum_j z^j / (2j+2)! = (cosh x - 1) / z,
  Q(z) = sum_j z^j / (2j+3)! = (sinh x - x) / (x z),
as w_cur = x (E - x Q) and w_up = x e (E + x Q).  Truncated Taylor series
need seven terms each on z in [0, 4]; this script fits degree-4 polynomials
that minimise the maximum relative error on that interval (iteratively
reweighted least squares at 40 digits on Chebyshev nodes), rounds the
coefficients to FP32 and reports the error of the rounded polynomials.
Run it to regenerate the constants:  python fit_weights32.py
"""

import mpmath as mp
import numpy as np

mp.mp.dps = 40
Z_MAX = 4


def E(z):
    z = mp.mpf(z)
    if z == 0:
        return mp.mpf(1) / 2
    x = mp.sqrt(z)
    return (mp.cosh(x) - 1) / z


def Q(z):
    z = mp.mpf(z)
    if z == 0:
        return mp.mpf(1) / 6
    x = mp.sqrt(z)
    return (mp.sinh(x) - x) / (x * z)


def fit(f, deg, n=400, rounds=40):
    """Coefficients c[0..deg] of the polynomial with small maximum relative
    error against f on [0, Z_MAX]."""
    t = [mp.cos(mp.pi * (i + mp.mpf(1) / 2) / n) for i in range(n)]
    zs = [Z_MAX * (ti + 1) / 2 for ti in t]
    fv = [f(z) for z in zs]
    w = [mp.mpf(1)] * n
    c = None
    for _ in range(rounds):
        A = mp.matrix(n, deg + 1)
        y = mp.matrix(n, 1)
        for i, z in enumerate(zs):
            for j in range(deg + 1):
                A[i, j] = w[i] * z ** j / fv[i]
            y[i] = w[i]
        c = mp.lu_solve(A.T * A, A.T * y)
        err = [(sum(c[j] * z ** j for j in range(deg + 1)) - fv[i]) / fv[i]
               for i, z in enumerate(zs)]
        m = max(abs(e) for e in err)
        w = [wi * (1 + 10 * abs(e) / m) for wi, e in zip(w, err)]
        s = sum(w)
        w = [wi * n / s for wi in w]
    return [c[j] for j in range(deg + 1)]


def max_rel_err_fp32(coef, f, n=4000):
    """Maximum relative error of the FP32-rounded coefficients, evaluated
    exactly (so this is the fit plus coefficient rounding, not the FP32
    Horner rounding, which adds about one unit in the last place)."""
    cf = [mp.mpf(float(np.float32(float(c)))) for c in coef]
    worst = 0
    for i in range(n + 1):
        z = mp.mpf(Z_MAX) * i / n
        p = sum(cf[j] * z ** j for j in range(len(cf)))
        worst = max(worst, abs(p - f(z)) / f(z))
    return float(worst)


if __name__ == "__main__":
    for name, f in (("E", E), ("Q", Q)):
        c = fit(f, 4)
        print(f"{name}: max relative error {max_rel_err_fp32(c, f):.2e}")
        print("  " + ", ".join(f"{float(np.float32(float(x))):.9e}f" for x in c))
