"""Fit the polynomial coefficients of the library's inverse normal CDF.

Build-time generator for ``ndtri_coeffs.h`` (run: ``python fit_ndtri.py``).

Form (M. Giles, "Approximating the erfinv function", GPU Computing Gems,
2011): with y = 1 - 2q (q = min(u, 1-u)) and w = -ln((1-y)(1+y)) = -ln(4q(1-q)),
    erfinv(y) = y * P_c(w - W_MID)           for w < W_SPLIT     (|z| < ~2.9)
    erfinv(y) = y * P_t(sqrt(w) - T_MID)     for w < W_SPLIT2    (q > ~2.8e-8)
    erfinv(y) = y * P_u(sqrt(w) - U_MID)     otherwise
and Phi^-1(u) = +-sqrt(2) erfinv(y).  The FP32 routines take the central branch in the
variable v = log2(q(1-q)) itself, w = -ln 2 (v + 2):
    |Phi^-1(u)| = y * P_v(v)                for v > V_SPLIT = -2 - W_SPLIT/ln 2
with P_v(v) = sqrt(2) erfinv(y)/y, so the factors 4, -ln 2 and sqrt(2) and the shift by
W_MID cost no operation (evaluated uncentred in FP32 Horner it stays within 2e-7 relative).
The coefficients here are our own:
a weighted least-squares fit of erfinv(y)/y on Chebyshev nodes followed by
Lawson iterations toward the minimax relative error, reference values from
mpmath at 40 digits.  The tail covers q down to 1e-22.
"""
import math
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
W_SPLIT = 5.0
W_MID = 2.5
W_SPLIT2 = 16.0
W_TAIL_MAX = -math.log(4e-22)
T_MID = 3.3
U_MID = 5.5
DEG_C = 8
DEG_T = 8
DEG_U = 8


V_SPLIT = -2.0 - W_SPLIT / math.log(2.0)


def target(w):
    y = mp.sqrt(1 - mp.e ** (-w))
    return mp.erfinv(y) / y


def target_v(v):
    return mp.sqrt(2) * target(-mp.log(2) * (v + 2))


def fit(lo, hi, deg, xform, n=600, lawson=60, tgt=target):
    k = np.arange(n)
    w = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.pi * (k + 0.5) / n)
    g = np.array([float(tgt(mp.mpf(x))) for x in w])
    t = np.array([xform(x) for x in w])
    A = np.vander(t, deg + 1, increasing=True)
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
    cc, ec = fit(1e-12, W_SPLIT, DEG_C, lambda x: x - W_MID)
    ct, et = fit(W_SPLIT, W_SPLIT2, DEG_T, lambda x: math.sqrt(x) - T_MID)
    cu, eu = fit(W_SPLIT2, W_TAIL_MAX, DEG_U, lambda x: math.sqrt(x) - U_MID)
    cv, ev = fit(V_SPLIT, -2.0 - 1e-12, DEG_C, lambda x: x, tgt=target_v)
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "ndtri_coeffs.h"), "w") as f:
        f.write("/* Generated by fit_ndtri.py -- do not edit.  Polynomial coefficients (lowest\n")
        f.write(" * degree first) of erfinv(y)/y in the two-branch form described there.\n")
        f.write(f" * max relative fit error: central {ec:.2e}, tail {et:.2e}, far tail {eu:.2e},\n")
        f.write(f" * FP32 central in v = log2(q(1-q)) {ev:.2e}\n")
        f.write(" * (double evaluation). */\n")
        f.write("#pragma once\n")
        f.write(f"#define RQMC_NDTRI_W_SPLIT {W_SPLIT!r}\n#define RQMC_NDTRI_W_MID {W_MID!r}\n")
        f.write(f"#define RQMC_NDTRI_W_SPLIT2 {W_SPLIT2!r}\n")
        f.write(f"#define RQMC_NDTRI_T_MID {T_MID!r}\n#define RQMC_NDTRI_U_MID {U_MID!r}\n")
        f.write(f"#define RQMC_NDTRI_DEG_C {DEG_C}\n#define RQMC_NDTRI_DEG_T {DEG_T}\n")
        f.write(f"#define RQMC_NDTRI_DEG_U {DEG_U}\n")
        f.write(f"#define RQMC_NDTRI_V_SPLIT {V_SPLIT!r}\n")
        for name, c in (("RQMC_NDTRI_C", cc), ("RQMC_NDTRI_T", ct), ("RQMC_NDTRI_U", cu), ("RQMC_NDTRI_V", cv)):
            f.write(f"#define {name} {{ " + ", ".join(f"{x:.17e}" for x in c) + " }\n")
    print(f"central max rel err {ec:.3e}, tail {et:.3e}, far tail {eu:.3e}, FP32 central in v {ev:.3e}")


if __name__ == "__main__":
    main()
