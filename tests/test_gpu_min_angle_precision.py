"""GPU: the FP64 minimum-angle gap (table-driven atan2) against the oracle's
FP64 atan2, vertex by vertex: one layout per vertex of degree 2 or 3 in a
batch, so that each layout's sum of d_v is one vertex's d_v (Algorithm 2).
Gaps are drawn at, near and halfway between the 256 sector angles of the
table, plus the axis directions and opposite pairs."""
import math

import numpy as np
import pytest

import oracle
from paper_2411_09809_gb300 import build, gr

pytestmark = pytest.mark.gpu
W = 2 * math.pi / 256


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gr.load()


def point(c, phi, r):
    return (int(round(c[0] + r * math.cos(phi))), int(round(c[1] + r * math.sin(phi))))


def star_layouts(rng, n):
    layouts = []
    for i in range(n):
        c = (int(rng.integers(25000, 40000)), int(rng.integers(25000, 40000)))
        alpha = float(rng.uniform(0, 2 * math.pi))
        kind = i % 4
        j = int(rng.integers(0, 129))
        if kind == 0:
            gap = j * W                                   # on a sector angle
        elif kind == 1:
            gap = (j + 0.5) * W                           # halfway between two
        elif kind == 2:
            gap = j * W + float(rng.uniform(-1e-4, 1e-4))  # near one
        else:
            gap = float(rng.uniform(0, math.pi))
        r1, r2 = float(rng.uniform(50, 20000)), float(rng.uniform(50, 20000))
        pts = [c, point(c, alpha, r1), point(c, alpha + gap, r2)]
        if i % 7 == 0:  # a third direction: degree 3
            pts.append(point(c, alpha - float(rng.uniform(0.1, 3.0)), float(rng.uniform(50, 20000))))
        if i % 11 == 0:  # axis-parallel and opposite directions
            pts = [c, (c[0] + 1000, c[1]), (c[0] - 37, c[1])] if i % 2 else [c, (c[0], c[1] + 5), (c[0] + 7, c[1])]
        xy = np.array(pts, np.int32)
        if len({tuple(p) for p in pts}) < len(pts):
            continue
        e = np.array([[0, k] for k in range(1, len(pts))], np.int32)
        layouts.append((xy, e))
    return layouts


def test_min_angle_fp64_gap_per_vertex():
    rng = np.random.default_rng(90)
    layouts = star_layouts(rng, 3000)
    v_off = np.concatenate([[0], np.cumsum([len(x) for x, _ in layouts])]).astype(np.int64)
    e_off = np.concatenate([[0], np.cumsum([len(e) for _, e in layouts])]).astype(np.int64)
    xy = np.concatenate([x for x, _ in layouts]).astype(np.int32)
    edges = np.concatenate([e for _, e in layouts]).astype(np.int32)
    with gr.Batch(v_off, e_off, xy, edges) as B:
        res = B.evaluate(gr.GR_METRIC_MIN_ANGLE, 70 * math.pi / 180, 0)
    worst = 0.0
    for i, (x, e) in enumerate(layouts):
        want = oracle.min_angle(x, e)
        got = res[i].min_angle
        assert got.n_vertices_counted == want.n_vertices == 1, i
        err = abs(got.sum_d - want.sum_d)
        worst = max(worst, err)
        assert err <= 4e-15 + 1e-13 * abs(want.sum_d), (i, got.sum_d, want.sum_d)
    assert worst < 1e-14


def test_min_angle_hub_above_warp_degree():
    # a vertex of degree 300 (the warp-shared path) with gaps near sector angles
    rng = np.random.default_rng(91)
    c = (32768, 32768)
    phis = np.sort(rng.uniform(0, 2 * math.pi, size=299))
    phis = np.append(phis, phis[0] + 3 * W + 1e-6)  # the smallest gap: three sectors and a bit
    pts = [c] + [point(c, float(p), float(rng.uniform(5000, 30000))) for p in phis]
    xy = np.array(pts, np.int32)
    keep = np.unique(xy, axis=0, return_index=True)[1]
    assert len(keep) == len(xy)
    e = np.array([[0, k] for k in range(1, len(pts))], np.int32)
    with gr.Layout(xy, e) as L:
        got = L.evaluate(gr.GR_METRIC_MIN_ANGLE, 70 * math.pi / 180, 0).min_angle
    want = oracle.min_angle(xy, e)
    assert got.n_vertices_counted == want.n_vertices == 1
    assert abs(got.sum_d - want.sum_d) <= 4e-15 + 1e-13 * abs(want.sum_d)
