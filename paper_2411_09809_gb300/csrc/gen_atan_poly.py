"""Writes atan_poly.cuh: a minimax polynomial for arctan on [0, 1].

atan(t) ~= t * P(t^2), P of degree N, with coefficients fitted here by the
Remez exchange algorithm (Remez 1934) on the absolute error, in float64.  The
kernel evaluates it in FP32 with Horner's rule and fused multiply-adds; the
acute crossing angle is atan(min/max) or pi/2 - atan(min/max).
Run: python gen_atan_poly.py  (prints the max errors; rewrites the header).
"""
import os

import numpy as np

N = 7  # degree of P in t^2 -> odd polynomial of degree 15


def fit(n_iter=40):
    m = N + 1  # coefficients; Remez needs m + 1 reference points
    # initial reference: Chebyshev extrema on [0, 1]
    k = np.arange(m + 1)
    ref = 0.5 - 0.5 * np.cos(np.pi * k / m)
    grid = np.linspace(0.0, 1.0, 200001)
    for _ in range(n_iter):
        # solve t P(t^2) + (-1)^i E = atan(t) on the reference points
        A = np.zeros((m + 1, m + 1))
        for j in range(m):
            A[:, j] = ref ** (2 * j + 1)
        A[:, m] = (-1.0) ** k
        sol = np.linalg.solve(A, np.arctan(ref))
        c = sol[:m]
        err = grid * np.polyval(c[::-1], grid * grid) - np.arctan(grid)
        # new reference: the extrema of the error between sign changes
        s = np.sign(err)
        s[s == 0] = 1
        idx = np.flatnonzero(np.diff(s) != 0)
        bounds = np.concatenate([[0], idx + 1, [len(grid)]])
        ext = [b0 + int(np.argmax(np.abs(err[b0:b1]))) for b0, b1 in zip(bounds[:-1], bounds[1:])]
        if len(ext) < m + 1:
            break
        # keep the m + 1 largest alternating extrema
        while len(ext) > m + 1:
            if abs(err[ext[0]]) < abs(err[ext[-1]]):
                ext = ext[1:]
            else:
                ext = ext[:-1]
        ref = grid[ext]
    return c, np.max(np.abs(err))


def fp32_error(c):
    t = np.linspace(0.0, 1.0, 1000001).astype(np.float32)
    u = (t * t).astype(np.float32)
    p = np.float32(c[-1])
    for cj in c[-2::-1]:
        p = (p * u + np.float32(cj)).astype(np.float32)
    a = (p * t).astype(np.float32)
    return float(np.max(np.abs(a.astype(np.float64) - np.arctan(t.astype(np.float64)))))


def main():
    c, e64 = fit()
    e32 = fp32_error(c)
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// atan_poly.cuh -- written by gen_atan_poly.py; do not edit.",
        f"// atan(t) ~= t * P(t^2) on [0, 1], P of degree {N}, Remez minimax fit of the",
        f"// absolute error: {e64:.3e} in exact arithmetic, {e32:.3e} evaluated in FP32.",
        "#pragma once",
        "",
        "namespace gr {",
        "constexpr double kAtanMaxAbsError = %.3e;" % max(e64, e32),
        "",
        "// arctan(t) for t in [0, 1], FP32, Horner's rule with fused multiply-adds.",
        "__device__ __forceinline__ float atan01(float t) {",
        "    const float u = t * t;",
        f"    float p = {float(np.float32(c[-1]))!r}f;",
    ]
    lines += [f"    p = fmaf(p, u, {float(np.float32(x))!r}f);" for x in c[-2::-1]]
    lines += ["    return p * t;", "}", "}  // namespace gr", ""]
    with open(os.path.join(here, "atan_poly.cuh"), "w") as f:
        f.write("\n".join(lines))
    print(f"max |error|: {e64:.3e} (float64), {e32:.3e} (float32 Horner)")


if __name__ == "__main__":
    main()
