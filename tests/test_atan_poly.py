"""The FP32 arctangent polynomial the crossing kernels use (atan_poly.cuh,
written by csrc/gen_atan_poly.py) stays within its stated error bound against
float64 arctan; parsed from the header, evaluated the way the kernel does
(Horner, FP32, fused multiply-add emulated in float64 then rounded)."""
import os
import re

import numpy as np

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2411_09809_gb300", "csrc", "atan_poly.cuh")


def coefficients():
    text = open(HEADER).read()
    first = float(re.search(r"float p = ([-0-9.e]+)f;", text).group(1))
    rest = [float(v) for v in re.findall(r"p = fmaf\(p, u, ([-0-9.e]+)f\);", text)]
    bound = float(re.search(r"kAtanMaxAbsError = ([0-9.e-]+);", text).group(1))
    return [first] + rest, bound


def test_atan_polynomial_error_bound():
    coef, bound = coefficients()
    t = np.linspace(0.0, 1.0, 2_000_001).astype(np.float32)
    u = (t * t).astype(np.float32)
    p = np.full_like(t, np.float32(coef[0]))
    for c in coef[1:]:
        p = (p.astype(np.float64) * u + np.float32(c)).astype(np.float32)  # fma: one rounding
    a = (p * t).astype(np.float32).astype(np.float64)
    err = np.abs(a - np.arctan(t.astype(np.float64)))
    assert err.max() <= 1.05 * bound
    assert bound < 2e-7
    # the reflected branch pi/2 - atan(t) for t = x / y covers [pi/4, pi/2]
    b = np.float32(np.pi / 2) - a.astype(np.float32)
    assert np.abs(b.astype(np.float64) - (np.pi / 2 - np.arctan(t.astype(np.float64)))).max() < 3e-7
