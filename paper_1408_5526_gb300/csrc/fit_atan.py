"""Fit the polynomial coefficients of the library's FP32 arctangent (MBS prepayment).

Build-time generator for ``atan_coeffs.h`` (run: ``python fit_atan.py``).

Form: with a = |x| and t = min(a, 1/a) in [0, 1],
    atan(t) = t * P(t^2),      atan(x) = sign(x) * (a > 1 ? pi/2 - atan(t) : atan(t)),
the reflection atan(a) = pi/2 - atan(1/a) for a > 0.  P is our own fit of atan(sqrt(z))/sqrt(z)
on z in [0, 1]: least squares on Chebyshev nodes followed by Lawson iterations toward the
minimax relative error, reference values from mpmath at 40 digits.
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
DEG = 8


def target(z):
    if z == 0:
        return mp.mpf(1)
    r = mp.sqrt(z)
    return mp.atan(r) / r


def fit(deg, n=800, lawson=80):
    k = np.arange(n)
    z = 0.5 + 0.5 * np.cos(np.pi * (k + 0.5) / n)
    g = np.array([float(target(mp.mpf(x))) for x in z])
    A = np.vander(z, deg + 1, increasing=True)
    wt = np.ones(n)
    for _ in range(lawson):
        sw = np.sqrt(wt) / g
        c, *_ = np.linalg.lstsq(A * sw[:, None], g * sw, rcond=None)
        err = np.abs(A @ c - g) / g
        wt = wt * err
        wt /= wt.sum()
    err = np.abs(A @ c - g) / g
    return c, float(err.max())


def main():
    c, e = fit(DEG)
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "atan_coeffs.h"), "w") as f:
        f.write("// Generated by fit_atan.py -- do not edit.  atan(t) = t P(t^2) on t in [0, 1],\n")
        f.write(f"// P of degree {DEG} in t^2, max relative fit error {e:.2e}.\n")
        f.write("#pragma once\n")
        f.write(f"#define RQMC_ATAN_DEG {DEG}\n")
        f.write("#define RQMC_ATAN_C { " + ", ".join(f"{x:.17e}" for x in c) + " }\n")
    print("max relative error", e)


if __name__ == "__main__":
    main()
