// atan_poly.cuh -- written by gen_atan_poly.py; do not edit.
// atan(t) ~= t * P(t^2) on [0, 1], P of degree 7, Remez minimax fit of the
// absolute error: 3.748e-08 in exact arithmetic, 1.416e-07 evaluated in FP32.
#pragma once

namespace gr {
constexpr double kAtanMaxAbsError = 1.416e-07;

// arctan(t) for t in [0, 1], FP32, Horner's rule with fused multiply-adds.
__device__ __forceinline__ float atan01(float t) {
    const float u = t * t;
    float p = -0.004054567310959101f;
    p = fmaf(p, u, 0.021862957626581192f);
    p = fmaf(p, u, -0.0559123270213604f);
    p = fmaf(p, u, 0.0964219719171524f);
    p = fmaf(p, u, -0.1390862911939621f);
    p = fmaf(p, u, 0.19946566224098206f);
    p = fmaf(p, u, -0.33329859375953674f);
    p = fmaf(p, u, 0.9999993443489075f);
    return p * t;
}
}  // namespace gr
