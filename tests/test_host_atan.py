"""The FP32 arctangent of the MBS prepayment step (k_mbs.cuh), checked on the host: its
fitted coefficients (atan_coeffs.h) evaluated in float32 in the kernel's order against
numpy's double-precision arctangent over the whole real line."""
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_1408_5526_gb300", "csrc", "atan_coeffs.h")


def _coeffs():
    txt = open(HDR).read()
    body = re.search(r"RQMC_ATAN_C \{([^}]*)\}", txt).group(1)
    return np.array([float(v) for v in body.split(",")], dtype=np.float32)


def _atan32(x):
    C = _coeffs()
    x = np.asarray(x, dtype=np.float32)
    a = np.abs(x)
    with np.errstate(divide="ignore"):
        t = np.minimum(a, np.float32(1.0) / a)
    z = t * t
    p = np.full_like(z, C[-1])
    for c in C[-2::-1]:
        p = p * z + c
    r = t * p
    y = np.where(a > 1, np.float32(np.pi / 2) - r, r)
    return np.copysign(y, x)


def test_atan32_error_bound_on_the_real_line():
    x = np.concatenate([np.linspace(-4, 4, 200001), np.logspace(-30, 30, 20001), -np.logspace(-30, 30, 2001),
                        [0.0, 1.0, -1.0, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)]]).astype(np.float32)
    got = _atan32(x).astype(np.float64)
    ref = np.arctan(x.astype(np.float64))
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-38)
    assert err.max() < 4e-7                  # a few float32 ulp everywhere
    assert np.all(np.abs(got) <= np.pi / 2 + 1e-6)


def test_atan32_special_values():
    assert _atan32(np.float32(0.0)) == 0.0
    assert np.signbit(_atan32(np.float32(-0.0)))
    assert abs(_atan32(np.float32(np.inf)) - np.pi / 2) < 1e-7
    assert abs(_atan32(np.float32(-np.inf)) + np.pi / 2) < 1e-7
    assert np.isnan(_atan32(np.float32(np.nan)))
    # the MBS argument K3 i + K4 of the paper's constants (i near 0.7 %) lies near 0.57
    x = np.float32(10.0 * 0.007 + 0.5)
    assert abs(float(_atan32(x)) - np.arctan(float(x))) < 1e-7
