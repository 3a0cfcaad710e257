"""CPU pins of the strip oracle (the approximate algorithms of arXiv 2411.09809,
Sec. 3.2.2-3.2.3): the sweep against a pairwise brute force of the definition
in exact rationals, Eq. 1 against the direct per-pair sum, closed forms, the
exact count as an upper bound, and the exchange of the two orientations."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

IDEAL = 7 * math.pi / 18


def acute(ti, tj):
    d = abs(tj - ti)
    return min(d, math.pi - d)


def line_theta(dx, dy):
    t = math.atan2(dy, dx)
    if t < 0:
        t += math.pi
    if t >= math.pi:
        t -= math.pi
    return t


def brute_force(xy, edges, l, orient, ideal=IDEAL):
    """Every pair of segments that both cross both lines of a strip, compared
    by their exact rational y at the two lines: a strict reversal counts, with
    |ideal - angle| / ideal."""
    segs = []
    for a, b in edges:
        x0, y0 = int(xy[a][orient]), int(xy[a][1 - orient])
        x1, y1 = int(xy[b][orient]), int(xy[b][1 - orient])
        if x0 == x1:
            continue
        if x0 > x1:
            x0, y0, x1, y1 = x1, y1, x0, y0
        segs.append((x0, y0, x1, y1, line_theta(x1 - x0, y1 - y0)))
    count, term = 0, 0.0
    smax = 65536 // l + 1
    for s in range(smax + 1):
        XL, XR = s * l, (s + 1) * l
        inside = [g for g in segs if g[0] <= XL and XR <= g[2]]
        ys = [(Fraction(g[1]) + Fraction((XL - g[0]) * (g[3] - g[1]), g[2] - g[0]),
               Fraction(g[1]) + Fraction((XR - g[0]) * (g[3] - g[1]), g[2] - g[0]), g[4]) for g in inside]
        for i in range(len(ys)):
            for j in range(i + 1, len(ys)):
                li, ri, ti = ys[i]
                lj, rj, tj = ys[j]
                if (li < lj and ri > rj) or (li > lj and ri < rj):
                    count += 1
                    term += abs(ideal - acute(ti, tj)) / ideal
    return count, term


def small_layout(seed, V=40, E=70, span=200, offset=0):
    rng = np.random.default_rng(seed)
    xy = (offset + rng.integers(0, span, size=(V, 2))).astype(np.int32)
    a = rng.integers(0, V, size=E)
    b = (a + rng.integers(1, V, size=E)) % V
    return xy, np.stack([a, b], axis=1).astype(np.int32)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("orient", [0, 1])
def test_sweep_equals_pairwise_definition(seed, orient):
    xy, e = small_layout(seed, span=60 + 20 * seed)
    l = [3, 5, 7, 11][seed % 4]
    got = oracle.strip_crossings(xy, e, l, orient)
    c, t = brute_force(xy, e, l, orient)
    assert got.crossings == c
    assert got.term_sum == pytest.approx(t, rel=1e-12, abs=1e-12)


def test_degenerate_small_box():
    # shared endpoints, duplicates, collinear chains and crossings on strip lines
    rng = np.random.default_rng(7)
    xy = rng.integers(0, 9, size=(30, 2)).astype(np.int32)
    a = rng.integers(0, 30, size=120)
    e = np.stack([a, (a + rng.integers(1, 30, size=120)) % 30], axis=1).astype(np.int32)
    for l in (1, 2, 3):
        for orient in (0, 1):
            got = oracle.strip_crossings(xy, e, l, orient)
            c, t = brute_force(xy, e, l, orient)
            assert got.crossings == c and got.term_sum == pytest.approx(t, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("ideal", [IDEAL, math.pi / 2, math.pi / 6, 0.05])
def test_eq1_equals_direct_sum(ideal):
    rng = np.random.default_rng(int(ideal * 1000))
    for _ in range(200):
        ti = float(rng.uniform(0, math.pi))
        tj = rng.uniform(0, math.pi, size=int(rng.integers(1, 30)))
        n = np.zeros(8, np.int64)
        S = np.zeros(8, np.float64)
        for t in tj:
            g = oracle.strip_category(ti, float(t), ideal)
            n[g] += 1
            S[g] += t
        direct = sum(abs(ideal - acute(ti, float(t))) for t in tj)
        assert oracle.strip_eq1(ti, ideal, n, S) == pytest.approx(direct, rel=1e-9, abs=1e-9)


def test_eq1_categories_cover_their_ranges():
    v = IDEAL
    t = 1.0
    pi = math.pi
    for d, g in [(0.0, 0), (v - 1e-9, 0), (v, 1), (pi / 2 - 1e-9, 1), (pi / 2, 2), (pi - v, 3),
                 (-1e-9, 4), (-v, 4), (-v - 1e-9, 5), (-pi / 2, 5), (-pi / 2 - 1e-9, 6), (-pi + v, 6),
                 (-pi + v - 1e-9, 7)]:
        if 0 <= t + d < pi:
            assert oracle.strip_category(t, t + d, v) == g, d


def test_segments_spanning_all_strips_closed_form():
    # n segments from x = 0 to x = W (W a multiple of l): every pair that crosses
    # off the strip lines is counted; the crossing x is exact in rationals
    rng = np.random.default_rng(3)
    n, l, W = 120, 16, 16 * 40
    a = rng.choice(5000, size=n, replace=False)
    b = rng.choice(5000, size=n, replace=False)
    xy = np.concatenate([np.stack([np.zeros(n), a], 1), np.stack([np.full(n, W), b], 1)]).astype(np.int32)
    e = np.stack([np.arange(n), np.arange(n) + n], 1).astype(np.int32)
    want, term = 0, 0.0
    for i in range(n):
        for j in range(i + 1, n):
            if (a[i] - a[j]) * (b[i] - b[j]) < 0:
                # y_i(x) = a_i + (b_i - a_i) x / W; equal at x = W (a_j - a_i) / ((b_i - a_i) - (b_j - a_j))
                x = Fraction(W * int(a[j] - a[i]), int((b[i] - a[i]) - (b[j] - a[j])))
                if x.denominator == 1 and x.numerator % l == 0:
                    continue
                want += 1
                term += abs(IDEAL - acute(line_theta(W, int(b[i] - a[i])), line_theta(W, int(b[j] - a[j])))) / IDEAL
    got = oracle.strip_crossings(xy, e, l, 0)
    assert got.crossings == want
    assert got.term_sum == pytest.approx(term, rel=1e-10)
    assert want > 0.9 * oracle.crossings(xy, e).proper  # nearly every crossing is in a spanned strip


@pytest.mark.parametrize("seed", range(4))
def test_never_above_the_exact_count(seed):
    rng = np.random.default_rng(100 + seed)
    V, E = 400, 1200
    xy = rng.integers(0, 65536, size=(V, 2)).astype(np.int32)
    a = rng.integers(0, V, size=E)
    e = np.stack([a, (a + rng.integers(1, V, size=E)) % V], axis=1).astype(np.int32)
    exact = oracle.crossings(xy, e)
    prev = None
    for l in (4096, 1024, 256, 64):
        est = oracle.strip_crossings(xy, e, l, 0)
        assert est.crossings <= exact.proper
        prev = est
    # narrow strips: almost every crossing of long random segments is found
    assert prev.crossings >= 0.97 * exact.proper
    assert prev.E_ca == pytest.approx(exact.E_ca, abs=0.01)


def test_orientations_exchange_x_and_y():
    xy, e = small_layout(21, V=200, E=600, span=65536)
    for l in (512, 2048):
        h = oracle.strip_crossings(xy, e, l, 1)
        v = oracle.strip_crossings(np.ascontiguousarray(xy[:, ::-1]), e, l, 0)
        assert h.crossings == v.crossings and h.records == v.records
        assert h.term_sum == pytest.approx(v.term_sum, rel=1e-12)
        both = oracle.strip_crossings(xy, e, l, 2)
        assert both.crossings == max(h.crossings, oracle.strip_crossings(xy, e, l, 0).crossings)
