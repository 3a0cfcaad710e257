"""Pins the CPU oracle to facts the paper and the mathematics fix (CPU only).

Each test names the definition it pins (arXiv 2411.09809, Sec. 2.1 and
Algorithms 1-5).  The closed forms are chosen so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_09809_gb300 import synth
from tests import brute

IDEAL = 7 * math.pi / 18


def _xy(pts):
    return np.asarray(pts, dtype=np.int32).reshape(-1, 2)


def _e(pairs):
    return np.asarray(pairs, dtype=np.int32).reshape(-1, 2)


# ------------------------------------------------------------------ E_c, E_ca

@pytest.mark.parametrize("n", [5, 9, 12])
def test_complete_graph_in_convex_position_has_n_choose_4_crossings(n):
    # Algorithm 4: every 4 points in strictly convex position contribute exactly one
    # crossing pair of disjoint edges; adjacent edges never cross.
    pts = [(i * 5000, i * i * 450) for i in range(n)]  # on a parabola: strictly convex
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    c = oracle.crossings(_xy(pts), _e(edges))
    assert c.proper == math.comb(n, 4)
    assert c.touching == 0 and c.collinear == 0 and c.zero_length_edges == 0
    assert c.crossings == math.comb(n, 4)


def test_axis_parallel_grid_crosses_at_right_angles():
    # h horizontal x v vertical segments: h*v crossings at pi/2, so
    # E_ca = 1 - |70 - 90| / 70 = 5/7 (Algorithm 5); with ideal 90 deg, E_ca = 1.
    h, v = 7, 9
    pts, edges = [], []
    for i in range(h):
        y = 1000 + 1000 * i
        pts += [(500, y), (1000 * v + 500, y)]
        edges.append((len(pts) - 2, len(pts) - 1))
    for j in range(v):
        x = 1000 + 1000 * j
        pts += [(x, 500), (x, 1000 * h + 500)]
        edges.append((len(pts) - 2, len(pts) - 1))
    c = oracle.crossings(_xy(pts), _e(edges))
    assert c.proper == h * v and c.crossings == h * v
    assert c.E_ca == pytest.approx(5.0 / 7.0, rel=1e-14)
    assert c.angle_dev_sum == pytest.approx(h * v * (math.pi / 2 - IDEAL), rel=1e-14)
    assert oracle.crossings(_xy(pts), _e(edges), ideal=math.pi / 2).E_ca == pytest.approx(1.0, abs=1e-15)


def test_45_degree_crossing():
    # a_c = 45 deg: E_ca = 1 - 25/70 = 9/14.
    pts = [(0, 100), (200, 100), (50, 50), (150, 150)]
    c = oracle.crossings(_xy(pts), _e([(0, 1), (2, 3)]))
    assert c.proper == 1
    assert c.E_ca == pytest.approx(9.0 / 14.0, rel=1e-14)


def test_crossing_angle_is_the_acute_angle_between_the_lines():
    # An obtuse pair of direction vectors (120 deg apart) crosses at 60 deg; reversing
    # either segment must not change it.
    pts = [(1000, 1000), (3000, 1000), (2500, 1000 - 866), (1500, 1000 + 866)]
    for e in ([(0, 1), (2, 3)], [(1, 0), (2, 3)], [(0, 1), (3, 2)]):
        c = oracle.crossings(_xy(pts), _e(e))
        ang = math.atan2(abs(2000 * 1732), abs(2000 * -1000))
        assert c.proper == 1
        assert c.angle_dev_sum == pytest.approx(abs(IDEAL - ang), rel=1e-14)
        assert ang < math.pi / 2


CLASS_CASES = [
    # (points, edges, proper, touching, collinear, zero)
    ("X", [(0, 0), (10, 10), (0, 10), (10, 0)], [(0, 1), (2, 3)], 1, 0, 0, 0),
    ("T-junction", [(0, 0), (10, 0), (5, 0), (5, 10)], [(0, 1), (2, 3)], 0, 1, 0, 0),
    ("endpoint contact, distinct ids", [(0, 0), (10, 0), (10, 0), (20, 10)], [(0, 1), (2, 3)], 0, 1, 0, 0),
    ("shared vertex", [(0, 0), (10, 0), (20, 10)], [(0, 1), (1, 2)], 0, 0, 0, 0),
    ("shared vertex, overlapping", [(0, 0), (10, 0), (20, 0)], [(0, 1), (0, 2)], 0, 0, 0, 0),
    ("collinear overlap", [(0, 0), (10, 0), (5, 0), (15, 0)], [(0, 1), (2, 3)], 0, 0, 1, 0),
    ("collinear single point", [(0, 0), (10, 0), (10, 0), (20, 0)], [(0, 1), (2, 3)], 0, 0, 1, 0),
    ("collinear disjoint", [(0, 0), (10, 0), (11, 0), (20, 0)], [(0, 1), (2, 3)], 0, 0, 0, 0),
    ("collinear containment, vertical", [(3, 0), (3, 20), (3, 5), (3, 7)], [(0, 1), (2, 3)], 0, 0, 1, 0),
    ("collinear diagonal overlap", [(0, 0), (6, 6), (6, 6), (9, 9)], [(0, 1), (3, 2)], 0, 0, 1, 0),
    ("parallel", [(0, 0), (10, 0), (0, 1), (10, 1)], [(0, 1), (2, 3)], 0, 0, 0, 0),
    ("near miss", [(0, 0), (10, 0), (5, 1), (5, 10)], [(0, 1), (2, 3)], 0, 0, 0, 0),
    ("zero length on a segment", [(0, 0), (10, 0), (5, 0), (5, 0)], [(0, 1), (2, 3)], 0, 0, 0, 1),
    ("zero length at a crossing", [(0, 0), (10, 10), (0, 10), (10, 0), (5, 5), (5, 5)],
     [(0, 1), (2, 3), (4, 5)], 1, 0, 0, 1),
    ("endpoint on endpoint, crossing lines", [(0, 0), (10, 10), (10, 10), (20, 0)], [(0, 1), (2, 3)], 0, 1, 0, 0),
]


@pytest.mark.parametrize("name,pts,edges,proper,touching,collinear,zero", CLASS_CASES,
                         ids=[c[0] for c in CLASS_CASES])
def test_pair_classes(name, pts, edges, proper, touching, collinear, zero):
    c = oracle.crossings(_xy(pts), _e(edges))
    assert (c.proper, c.touching, c.collinear, c.zero_length_edges) == (proper, touching, collinear, zero)
    assert c.crossings == proper + touching
    b = brute.crossings(_xy(pts), _e(edges), IDEAL)
    assert (b["proper"], b["touching"], b["collinear"], b["zero"]) == (proper, touching, collinear, zero)


def test_no_crossings_gives_E_ca_one():
    c = oracle.crossings(_xy([(0, 0), (10, 0), (0, 5), (10, 5)]), _e([(0, 1), (2, 3)]))
    assert c.crossings == 0 and c.E_ca == 1.0


def test_rational_brute_force_on_tiny_degenerate_layouts():
    # Exact rational parametric intersection (a different algorithm) on layouts where
    # collinear, touching, coincident and zero-length cases dominate.
    rng = np.random.default_rng(7)
    for trial in range(1500):
        V = int(rng.integers(3, 13))
        E = int(rng.integers(2, 21))
        L = synth.tiny_degenerate_layout(rng, V, E, span=int(rng.integers(3, 9)),
                                         offset=int(rng.integers(0, 65536 - 9)))
        c = oracle.crossings(L.xy, L.edges)
        b = brute.crossings(L.xy, L.edges, IDEAL)
        assert (c.proper, c.touching, c.collinear, c.zero_length_edges) == \
            (b["proper"], b["touching"], b["collinear"], b["zero"]), trial
        assert c.angle_dev_sum == pytest.approx(b["dev"], rel=1e-12, abs=1e-12), trial


def test_rational_brute_force_on_random_layouts():
    rng = np.random.default_rng(11)
    for trial in range(20):
        V = 40
        xy = rng.integers(0, 65536, size=(V, 2)).astype(np.int32)
        e = synth.add_random_edges(rng, V, np.zeros((0, 2), np.int32), 60)
        c = oracle.crossings(xy, e)
        b = brute.crossings(xy, e, IDEAL)
        assert (c.proper, c.touching, c.collinear) == (b["proper"], b["touching"], b["collinear"])
        assert c.angle_dev_sum == pytest.approx(b["dev"], rel=1e-12)


def test_random_segments_cross_with_probability_25_over_108():
    # Two segments with endpoints uniform in a square cross with probability 25/108.
    rng = np.random.default_rng(3)
    E = 4000
    xy = rng.integers(0, 65536, size=(2 * E, 2)).astype(np.int32)
    edges = np.arange(2 * E, dtype=np.int32).reshape(E, 2)
    c = oracle.crossings(xy, edges)
    frac = c.crossings / (E * (E - 1) / 2)
    assert abs(frac - 25 / 108) < 0.012, frac


def _transforms(xy):
    x, y = xy[:, 0].astype(np.int64), xy[:, 1].astype(np.int64)
    yield "translate", np.stack([x + 17, y + 301], 1)
    yield "rotate90", np.stack([y, 65535 - x], 1)
    yield "reflect", np.stack([65535 - x, y], 1)
    yield "transpose", np.stack([y, x], 1)
    yield "scale2", np.stack([2 * x, 2 * y], 1)


def test_invariances():
    rng = np.random.default_rng(5)
    V = 300
    base = synth.tiny_degenerate_layout(rng, V, 700, span=40)  # many degeneracies
    xy = (base.xy.astype(np.int64) * 97 + 1000).astype(np.int32)  # inside [1000, 5000)
    edges = base.edges
    ref = oracle.crossings(xy, edges)
    ref_occ = oracle.node_occlusion(xy, 200)
    ref_ma = oracle.min_angle(xy, edges)
    ref_ml = oracle.edge_length_variation(xy, edges)
    assert ref.proper > 0 and ref.touching > 0 and ref.collinear > 0 and ref.zero_length_edges > 0

    perm_v = rng.permutation(V)
    inv = np.empty(V, np.int64)
    inv[perm_v] = np.arange(V)
    xy_p = xy[perm_v]
    edges_p = inv[edges].astype(np.int32)
    edges_p = edges_p[rng.permutation(len(edges_p))]
    flip = rng.random(len(edges_p)) < 0.5
    edges_p[flip] = edges_p[flip][:, ::-1]
    variants = [("relabel+reorder+reverse", xy_p, edges_p)]
    variants += [(n, t.astype(np.int32), edges) for n, t in _transforms(xy)]
    for name, xv, ev in variants:
        c = oracle.crossings(xv, ev)
        assert (c.proper, c.touching, c.collinear, c.zero_length_edges) == \
            (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), name
        assert c.angle_dev_sum == pytest.approx(ref.angle_dev_sum, rel=1e-12), name
        ma = oracle.min_angle(xv, ev)
        assert ma.n_vertices == ref_ma.n_vertices, name
        assert ma.M_a == pytest.approx(ref_ma.M_a, rel=1e-12), name
        ml = oracle.edge_length_variation(xv, ev)
        assert ml == pytest.approx(ref_ml, rel=1e-12), name
        if name != "scale2":
            assert oracle.node_occlusion(xv, 200) == ref_occ, name
    assert oracle.node_occlusion(_transforms(xy).__next__()[1].astype(np.int32), 200) == ref_occ


def test_crossings_of_edges_sums_to_twice_the_totals():
    L = synth.plain_layout(V=300, knn_count=600, random_count=150, seed=99)
    c = oracle.crossings(L.xy, L.edges)
    per, dev = oracle.crossings_of_edges(L.xy, L.edges, np.arange(L.E))
    assert per[:, 0].sum() == 2 * c.proper
    assert per[:, 1].sum() == 2 * c.touching
    assert per[:, 2].sum() == 2 * c.collinear
    assert dev.sum() == pytest.approx(2 * c.angle_dev_sum, rel=1e-12)


# ----------------------------------------------------------------------- N_c

def _lattice(n, s, off=1000):
    return _xy([(off + i * s, off + j * s) for i in range(n) for j in range(n)])


@pytest.mark.parametrize("d,expected", [
    (0, 0), (100, 0), (101, 2 * 20 * 19), (141, 2 * 20 * 19),
    (142, 2 * 20 * 19 + 2 * 19 * 19), (200, 2 * 20 * 19 + 2 * 19 * 19),
    (201, 2 * 20 * 19 + 2 * 19 * 19 + 2 * 20 * 18),
])
def test_occlusion_on_a_lattice(d, expected):
    # Algorithm 1: ||p1 - p2||^2 < (2r)^2, strict.  Lattice spacing 100, n = 20.
    assert oracle.node_occlusion(_lattice(20, 100), d) == expected


def test_occlusion_coincident_points_and_all_pairs():
    xy = _xy([(5, 5)] * 6 + [(60000, 60000)])
    assert oracle.node_occlusion(xy, 0) == 0
    assert oracle.node_occlusion(xy, 1) == 15
    assert oracle.node_occlusion(xy, 100000) == 21
    with pytest.raises(ValueError):
        oracle.node_occlusion(xy, -1)


# ----------------------------------------------------------------------- M_a

def test_min_angle_stars():
    # Algorithm 2: d_v = (2 pi/deg - min gap) / (2 pi/deg), averaged over deg >= 2 vertices.
    c = (1000, 1000)
    four = [c, (1100, 1000), (1000, 1100), (900, 1000), (1000, 900)]
    r = oracle.min_angle(_xy(four), _e([(0, 1), (0, 2), (0, 3), (0, 4)]))
    assert (r.M_a, r.n_vertices) == (1.0, 1)
    eight = [c] + [(1000 + dx, 1000 + dy) for dx, dy in
                   [(7, 0), (3, 3), (0, 5), (-2, 2), (-9, 0), (-4, -4), (0, -1), (6, -6)]]
    r = oracle.min_angle(_xy(eight), _e([(0, k) for k in range(1, 9)]))
    assert r.M_a == pytest.approx(1.0, abs=1e-14) and r.sum_d == pytest.approx(0.0, abs=1e-14)
    three = [c, (1100, 1000), (1000, 1100), (900, 1000)]  # 0, 90, 180 deg: min 90, ideal 120
    r = oracle.min_angle(_xy(three), _e([(0, 1), (0, 2), (0, 3)]))
    assert r.M_a == pytest.approx(0.75, rel=1e-14) and r.sum_d == pytest.approx(0.25, rel=1e-14)
    same = [c, (1100, 1000), (1300, 1000)]  # same direction: gap 0, d_v = 1
    r = oracle.min_angle(_xy(same), _e([(0, 1), (0, 2)]))
    assert r.M_a == pytest.approx(0.0, abs=1e-15) and r.n_vertices == 1
    corner = [c, (1100, 1000), (1000, 1070)]  # 90 deg corner: gaps 90/270, ideal 180 -> 1/2
    r = oracle.min_angle(_xy(corner), _e([(0, 1), (0, 2)]))
    assert r.M_a == pytest.approx(0.5, rel=1e-14)


def test_min_angle_degenerate_cases():
    # degree-1 vertices only -> no vertex counted -> M_a = 1; zero-length edges ignored.
    r = oracle.min_angle(_xy([(0, 0), (5, 5), (9, 9), (9, 9)]), _e([(0, 1), (2, 3)]))
    assert (r.M_a, r.n_vertices) == (1.0, 0)
    r = oracle.min_angle(_xy([(0, 0), (10, 0), (0, 0), (0, 10)]), _e([(0, 1), (0, 2), (0, 3)]))
    assert r.n_vertices == 1 and r.M_a == pytest.approx(0.5, rel=1e-14)


def test_min_angle_against_the_literal_float_sort():
    rng = np.random.default_rng(13)
    for _ in range(30):
        V = 60
        xy = rng.integers(0, 65536, size=(V, 2)).astype(np.int32)
        e = synth.add_random_edges(rng, V, np.zeros((0, 2), np.int32), 150)
        r = oracle.min_angle(xy, e)
        ma, s, n = brute.min_angle_float_sort(xy, e)
        assert r.n_vertices == n
        assert r.M_a == pytest.approx(ma, rel=1e-12, abs=1e-12)


# ----------------------------------------------------------------------- M_l

def test_edge_length_variation_closed_forms():
    # Algorithm 3.  All lengths equal -> 0.
    pts = [(0, 0), (3, 4), (100, 100), (105, 100), (200, 200), (200, 195), (300, 300), (296, 297)]
    assert oracle.edge_length_variation(_xy(pts), _e([(0, 1), (2, 3), (4, 5), (6, 7)])) == pytest.approx(0.0, abs=1e-15)
    # lengths {l, 2l} -> mu = 1.5 l, S = l^2 / 2, M_l = sqrt(0.5 / (2 * 2.25)) / 1 = 1/3.
    pts = [(0, 0), (30, 40), (1000, 1000), (1060, 1080)]
    assert oracle.edge_length_variation(_xy(pts), _e([(0, 1), (2, 3)])) == pytest.approx(1 / 3, rel=1e-14)
    # lengths {3, 4, 5} -> mu = 4, S = 2, M_l = sqrt(2 / 48) / sqrt(2) = sqrt(1/48).
    pts = [(0, 0), (3, 0), (10, 10), (10, 14), (20, 20), (23, 24)]
    assert oracle.edge_length_variation(_xy(pts), _e([(0, 1), (2, 3), (4, 5)])) == pytest.approx(math.sqrt(1 / 48), rel=1e-14)
    # a single edge, or all zero lengths -> 0
    assert oracle.edge_length_variation(_xy(pts), _e([(0, 1)])) == 0.0
    assert oracle.edge_length_variation(_xy([(5, 5), (5, 5), (7, 7), (7, 7)]), _e([(0, 1), (2, 3)])) == 0.0
    # zero-length edges count with l = 0: lengths {0, 2} -> mu = 1, S = 2, sqrt(2/2)/1 = 1
    pts = [(5, 5), (5, 5), (0, 0), (2, 0)]
    assert oracle.edge_length_variation(_xy(pts), _e([(0, 1), (2, 3)])) == pytest.approx(1.0, rel=1e-14)


# ------------------------------------------------------------------ validate

def test_validate():
    xy = _xy([(0, 0), (65535, 65535), (3, 3)])
    assert oracle.validate(xy, _e([(0, 1), (1, 2)])) == 0
    assert oracle.validate(xy, _e([(0, 3)])) == 1
    assert oracle.validate(xy, _e([(1, 1)])) == 1
    assert oracle.validate(xy, _e([(-1, 1)])) == 1
    assert oracle.validate(_xy([(0, 65536), (1, 1)]), _e([(0, 1)])) == 2
    assert oracle.validate(_xy([(-1, 0), (1, 1)]), _e([(0, 1)])) == 2
