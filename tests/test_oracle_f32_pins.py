"""Pins of the FP32 (differentiable) form of the oracle (CPU only)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2411_09809_gb300 import synth

IDEAL = 7 * math.pi / 18


def exact_orient(a, b, c):
    ax, ay, bx, by, cx, cy = (Fraction(float(np.float32(v))) for v in (*a, *b, *c))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


@pytest.mark.parametrize("lo,hi", [(-40, 1), (-120, 120)])
def test_orientation_is_exact_on_fp32_inputs(lo, hi):
    rng = np.random.default_rng(1)
    for _ in range(3000):
        e = rng.integers(lo, hi, size=6)
        v = (rng.choice([-1.0, 1.0], size=6) * rng.random(6) * 2.0 ** e).astype(np.float32)
        a, b, c = v[0:2], v[2:4], v[4:6]
        want = exact_orient(a, b, c)
        assert oracle.orient_f32(a, b, c) == want
        assert oracle.orient_f32_exact(a, b, c) == want


def test_orientation_on_exactly_collinear_and_one_ulp_off():
    rng = np.random.default_rng(2)
    zero = 0
    for _ in range(2000):
        # points a + t w with w and t dyadic: exactly collinear in FP32
        k = int(rng.integers(4, 20))
        a = rng.integers(0, 2 ** 10, size=2) / 2.0 ** 10
        w = rng.integers(-2 ** 6, 2 ** 6, size=2) / 2.0 ** k
        t = rng.integers(-8, 9, size=2)
        b, c = a + t[0] * w, a + t[1] * w
        pts = [np.float32(x) for x in (*a, *b, *c)]
        o = oracle.orient_f32(pts[0:2], pts[2:4], pts[4:6])
        assert o == exact_orient(pts[0:2], pts[2:4], pts[4:6])
        assert oracle.orient_f32_exact(pts[0:2], pts[2:4], pts[4:6]) == o
        zero += o == 0
        # one ulp away
        c2 = np.nextafter(np.float32(c[0]), np.float32(1.0))
        want = exact_orient(pts[0:2], pts[2:4], [c2, pts[5]])
        assert oracle.orient_f32(pts[0:2], pts[2:4], [c2, pts[5]]) == want
        assert oracle.orient_f32_exact(pts[0:2], pts[2:4], [c2, pts[5]]) == want
    assert zero > 1500


@pytest.mark.parametrize("seed", range(6))
def test_fp32_metrics_equal_the_integer_oracle_on_scaled_coordinates(seed):
    # coordinates k / 65536 are exact in FP32: the same geometry scaled by 2^-16
    rng = np.random.default_rng(seed)
    L = synth.tiny_degenerate_layout(rng, 60, 400, span=int(rng.integers(3, 30)), offset=int(rng.integers(0, 60000)))
    xyf = (L.xy.astype(np.float64) / 65536.0).astype(np.float32)
    ci, cf = oracle.crossings(L.xy, L.edges), oracle.crossings_f32(xyf, L.edges)
    assert (ci.proper, ci.touching, ci.collinear, ci.zero_length_edges) == \
        (cf.proper, cf.touching, cf.collinear, cf.zero_length_edges)
    assert cf.angle_dev_sum == pytest.approx(ci.angle_dev_sum, rel=1e-12, abs=1e-12)
    mi, mf = oracle.min_angle(L.xy, L.edges), oracle.min_angle_f32(xyf, L.edges)
    assert mi.n_vertices == mf.n_vertices and mf.M_a == pytest.approx(mi.M_a, rel=1e-12, abs=1e-12)
    assert oracle.edge_length_variation_f32(xyf, L.edges) == pytest.approx(
        oracle.edge_length_variation(L.xy, L.edges), rel=1e-12, abs=1e-15)


def _loss_terms(xy, edges):
    return oracle.diff_terms_and_grads(xy, edges)[0]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(4)
    checked = 0
    for trial in range(6):
        V = 40
        xy = rng.random((V, 2)).astype(np.float32)
        e = synth.knn_edges(xy, 3, 70)
        e = synth.add_random_edges(rng, V, e, 12)
        terms, g_eca, g_ml, g_ma = oracle.diff_terms_and_grads(xy, e)
        _, pairs0 = oracle.crossings_f32(xy, e, return_pairs=True)
        _, args0 = oracle.min_angle_f32(xy, e, return_args=True)
        for v in rng.choice(V, size=12, replace=False):
            for c in range(2):
                h = 1e-4
                xp, xm = xy.copy(), xy.copy()
                xp[v, c] = np.float32(xy[v, c] + h)
                xm[v, c] = np.float32(xy[v, c] - h)
                # only where the crossing set and the smallest gaps stay the same
                same = True
                for xq in (xp, xm):
                    _, pq = oracle.crossings_f32(xq, e, return_pairs=True)
                    _, aq = oracle.min_angle_f32(xq, e, return_args=True)
                    same &= np.array_equal(pq, pairs0) and np.array_equal(aq, args0)
                if not same:
                    continue
                step = float(xp[v, c]) - float(xm[v, c])
                fd = (_loss_terms(xp, e) - _loss_terms(xm, e)) / step
                for k, g in enumerate((g_eca, g_ml, g_ma)):
                    assert g[v, c] == pytest.approx(fd[k], rel=2e-4, abs=1e-6 * max(1.0, np.abs(g).max())), \
                        (trial, v, c, k)
                checked += 1
    assert checked > 30
