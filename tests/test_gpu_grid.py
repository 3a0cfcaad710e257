"""GPU: the uniform-grid paths (crossings a2-a6, occlusion a8) agree with the
all-pairs kernels and with the oracle for every cell size, including inputs
built to put intersections and segments exactly on cell boundaries."""
import math

import numpy as np
import pytest

import oracle
from paper_2411_09809_gb300 import build, gr, synth

pytestmark = pytest.mark.gpu
IDEAL = 7 * math.pi / 18
REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gr.load()


LONG = [gr.GR_LONG_ALLPAIRS, gr.GR_LONG_GRID]


def run(xy, edges, d, path, k=0, occl_path=0, long_pairs=gr.GR_LONG_AUTO):
    opt = gr.gr_options(path, k, occl_path, 0, long_pairs)
    with gr.Layout(np.ascontiguousarray(xy, np.int32), np.ascontiguousarray(edges, np.int32), opt) as L:
        return L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)


def counts(r):
    c = r.crossing.c
    return (c.proper, c.touching, c.collinear_overlaps, c.zero_length_edges)


def same_crossings(a, b, label):
    assert counts(a) == counts(b), label
    assert a.crossing.angle_dev_sum == pytest.approx(b.crossing.angle_dev_sum, rel=1e-12, abs=1e-9), label


def boundary_layout(rng, V, E, step, span_cells, offset_cells=0):
    """Vertices on a lattice of `step` (a divisor of the cell side), so crossings,
    endpoints and whole segments fall exactly on cell edges and corners."""
    n = span_cells * (64 // step)
    base = offset_cells * 64
    xy = base + step * rng.integers(0, n + 1, size=(V, 2))
    a = rng.integers(0, V, size=E)
    b = (a + rng.integers(1, V, size=E)) % V
    return np.clip(xy, 0, 65535).astype(np.int32), np.stack([a, b], 1).astype(np.int32)


@pytest.mark.parametrize("long_pairs", LONG)
@pytest.mark.parametrize("k", [6, 7, 8, 9, 10, 12, 16])
def test_grid_equals_allpairs_and_oracle_for_every_cell_size(k, long_pairs):
    L = synth.plain_layout(V=800, knn_count=1600, random_count=500, seed=31)
    ref = oracle.crossings(L.xy, L.edges)
    ap = run(L.xy, L.edges, 300, gr.GR_PATH_ALLPAIRS)
    g = run(L.xy, L.edges, 300, gr.GR_PATH_GRID, k, long_pairs=long_pairs)
    assert g.crossing_path == gr.GR_PATH_GRID and g.cell_log2 == k
    assert ap.crossing_path == gr.GR_PATH_ALLPAIRS
    same_crossings(g, ap, f"k={k}")
    assert counts(g) == (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges)
    assert g.crossing.E_ca == pytest.approx(ref.E_ca, rel=REL)
    assert g.grid_records >= L.E - ref.zero_length_edges


@pytest.mark.parametrize("long_pairs", LONG)
@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("k", [6, 7])
def test_grid_on_cell_boundaries(seed, k, long_pairs):
    rng = np.random.default_rng(500 + seed)
    step = [8, 16, 32, 64][seed % 4]
    xy, e = boundary_layout(rng, 120, 500, step, span_cells=6, offset_cells=int(rng.integers(0, 1000)))
    # plus axis-parallel segments lying on grid lines, sharing no vertex
    extra_pts, extra_e = [], []
    for i in range(20):
        x = 64 * int(rng.integers(0, 8)) + int(xy[:, 0].min() // 64 * 64)
        y0, y1 = sorted(int(v) for v in rng.integers(0, 8, size=2) * 64 + int(xy[:, 1].min() // 64 * 64))
        extra_pts += [(x, y0), (x, y1 + 64)]
        extra_e.append((len(xy) + len(extra_pts) - 2, len(xy) + len(extra_pts) - 1))
    xy = np.concatenate([xy, np.clip(np.array(extra_pts), 0, 65535).astype(np.int32)])
    e = np.concatenate([e, np.array(extra_e, np.int32)])
    ref = oracle.crossings(xy, e)
    g = run(xy, e, 64, gr.GR_PATH_GRID, k, long_pairs=long_pairs)
    assert counts(g) == (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), f"seed {seed}"
    assert g.crossing.angle_dev_sum == pytest.approx(ref.angle_dev_sum, rel=REL, abs=1e-6)
    assert ref.touching + ref.collinear > 0


@pytest.mark.parametrize("seed", range(6))
def test_grid_on_tiny_degenerate_layouts(seed):
    rng = np.random.default_rng(900 + seed)
    L = synth.tiny_degenerate_layout(rng, 50, 600, span=int(rng.integers(3, 40)),
                                     offset=64 * int(rng.integers(1, 1000)) - int(rng.integers(0, 20)))
    ref = oracle.crossings(L.xy, L.edges)
    for k in (6, 8):
        for lp in LONG:
            g = run(L.xy, L.edges, 3, gr.GR_PATH_GRID, k, long_pairs=lp)
            assert counts(g) == (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), (seed, k, lp)


def test_heavy_cell_spans_many_tiles():
    # 3,000 segments in one 64-wide cell: about 94 tiles of 32, 4,465 tile pairs
    rng = np.random.default_rng(2)
    xy = (1024 + rng.integers(0, 64, size=(2500, 2))).astype(np.int32)
    e = synth.add_random_edges(rng, 2500, np.zeros((0, 2), np.int32), 3000)
    ref = oracle.crossings(xy, e)
    g = run(xy, e, 5, gr.GR_PATH_GRID, 6)
    assert counts(g) == (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges)


@pytest.mark.parametrize("k", [6, 9])
def test_cells_mixing_short_and_long_segments(k):
    # a dense cluster of short edges crossed by many long edges: cells with
    # several tiles of short records followed by several tiles of long ones
    rng = np.random.default_rng(71 + k)
    cluster = (30000 + rng.integers(0, 1 << k, size=(1500, 2))).astype(np.int32)
    far = rng.integers(0, 65536, size=(600, 2)).astype(np.int32)
    xy = np.concatenate([cluster, far])
    short = synth.knn_edges(cluster, 3, 3000)
    lines = []
    for i in range(300):  # long edges through the cluster cell
        a = 1500 + 2 * i
        xy[a] = (30000 - 9000 + rng.integers(0, 200), 30000 + rng.integers(0, 1 << k))
        xy[a + 1] = (30000 + 9000 + rng.integers(0, 200), 30000 + rng.integers(0, 1 << k))
        lines.append((a, a + 1))
    e = np.concatenate([short, np.array(lines, np.int32)]).astype(np.int32)
    ref = oracle.crossings(xy, e)
    for lp in LONG:
        g = run(xy, e, 5, gr.GR_PATH_GRID, k, long_pairs=lp)
        assert counts(g) == (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), lp
        assert g.crossing.angle_dev_sum == pytest.approx(ref.angle_dev_sum, rel=REL, abs=1e-6)


@pytest.mark.parametrize("d", [1, 2, 63, 64, 65, 100, 128, 129, 1000, 5000])
def test_occlusion_grid_matches_oracle(d):
    rng = np.random.default_rng(d)
    pts = synth.gaussian_mixture_points(rng, 6000, 8, 400.0)
    lattice = np.array([(20000 + 64 * i, 20000 + 64 * j) for i in range(30) for j in range(30)], np.int32)
    xy = np.concatenate([pts, lattice, pts[:50]])  # coincident points too
    e = np.array([[0, 1]], np.int32)
    ref = oracle.node_occlusion(xy, d)
    g = run(xy, e, d, gr.GR_PATH_ALLPAIRS, 0, gr.GR_PATH_GRID)
    assert g.occlusion_path == gr.GR_PATH_GRID
    assert g.occlusion_pairs == ref
    a = run(xy, e, d, gr.GR_PATH_ALLPAIRS, 0, gr.GR_PATH_ALLPAIRS)
    assert a.occlusion_pairs == ref


@pytest.mark.parametrize("long_pairs", LONG)
def test_grid_per_edge_output_matches_oracle(long_pairs):
    import torch
    L = synth.plain_layout(V=600, knn_count=1200, random_count=300, seed=44)
    xy = torch.from_numpy(L.xy).cuda()
    ed = torch.from_numpy(L.edges).cuda()
    c = torch.empty((L.E, 3), dtype=torch.int64, device="cuda")
    dv = torch.empty(L.E, dtype=torch.float64, device="cuda")
    with gr.Layout(xy, ed, gr.gr_options(gr.GR_PATH_GRID, 7, 0, 0, long_pairs)) as lay:
        gr.gr_crossings_per_edge(lay.handle, IDEAL, c, dv)
    ref_c, ref_d = oracle.crossings_of_edges(L.xy, L.edges, np.arange(L.E))
    assert np.array_equal(c.cpu().numpy(), ref_c)
    np.testing.assert_allclose(dv.cpu().numpy(), ref_d, rtol=REL, atol=1e-6)


def test_auto_path_choices_on_the_workloads():
    sparse = synth.large_sparse_layout()
    r = run(sparse.xy, sparse.edges, 64, gr.GR_PATH_AUTO)
    assert r.crossing_path == gr.GR_PATH_GRID and r.occlusion_path == gr.GR_PATH_GRID
    dense = synth.dense_long_edge_layout(V=4000, E=40_000)
    r = run(dense.xy, dense.edges, 256, gr.GR_PATH_AUTO)
    assert r.crossing_path == gr.GR_PATH_ALLPAIRS


def test_repeated_evaluations_after_updates_match_oracle():
    # later evaluations reuse the plan and buffers of the first; an update that
    # outgrows them (short edges -> long edges, same cell size) is re-run
    rng = np.random.default_rng(12)
    V = 3000
    xy0 = synth.uniform_points(rng, V)
    e = synth.add_random_edges(rng, V, synth.knn_edges(xy0, 3, 6000), 300)
    steps = [xy0, np.clip(xy0 + rng.integers(-300, 300, size=xy0.shape), 0, 65535).astype(np.int32),
             synth.uniform_points(rng, V), (xy0 // 16).astype(np.int32), xy0]
    with gr.Layout(xy0, e, gr.gr_options(gr.GR_PATH_GRID, 9, 0, 0)) as L:
        for i, xy in enumerate(steps):
            L.update(np.ascontiguousarray(xy, np.int32))
            r = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 100)
            ref = oracle.crossings(xy, e)
            assert counts(r) == (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), i
            assert r.crossing.angle_dev_sum == pytest.approx(ref.angle_dev_sum, rel=REL, abs=1e-6), i
            assert r.occlusion_pairs == oracle.node_occlusion(xy, 100), i
            assert r.min_angle.M_a == pytest.approx(oracle.min_angle(xy, e).M_a, rel=REL, abs=REL), i


def test_update_with_invalid_coordinates_reports_erange():
    rng = np.random.default_rng(13)
    V = 5000
    xy = synth.uniform_points(rng, V)
    e = synth.knn_edges(xy, 3, 9000)
    bad = xy.copy()
    bad[17] = (70000, 5)
    bad[4000] = (-3, 100)
    for opt in (gr.gr_options(0, 0, gr.GR_PATH_GRID, 0), gr.gr_options(0, 0, gr.GR_PATH_ALLPAIRS, 0)):
        with gr.Layout(xy, e, opt) as L:
            L.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
            L.update(bad)
            with pytest.raises(gr.GrError) as ei:
                L.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
            assert ei.value.status == gr.GR_ERANGE
            L.update(xy)  # and it recovers
            r = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
            assert r.occlusion_pairs == oracle.node_occlusion(xy, 64)
    v_off = np.array([0, 2000, V], np.int64)
    e_off = np.array([0, 0, 0], np.int64)
    edges = np.zeros((0, 2), np.int32)
    with gr.Batch(v_off, e_off, xy, edges) as B:
        B.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
        B.update(bad)
        with pytest.raises(gr.GrError) as ei:
            B.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
        assert ei.value.status == gr.GR_ERANGE


def same_result(a, b, label):
    assert counts(a) == counts(b), label
    assert a.crossing.angle_dev_sum == b.crossing.angle_dev_sum, label
    assert a.occlusion_pairs == b.occlusion_pairs, label
    assert a.min_angle.M_a == b.min_angle.M_a and a.M_l == b.M_l, label
    # (the plan may differ: repeated evaluations keep the plan of the previous statistics)


@pytest.mark.parametrize("opt", [gr.gr_options(0, 0, 0, 0), gr.gr_options(gr.GR_PATH_GRID, 9, 0, 0),
                                 gr.gr_options(gr.GR_PATH_ALLPAIRS, 0, gr.GR_PATH_ALLPAIRS, 0)])
def test_replayed_evaluations_follow_every_change(opt):
    # repeated evaluations replay a captured graph; a change of metrics,
    # parameters, profiling or buffers must give what a fresh layout gives
    rng = np.random.default_rng(31)
    V = 6000
    xy0 = synth.uniform_points(rng, V)
    e = synth.add_random_edges(rng, V, synth.knn_edges(xy0, 3, 12000), 600)
    far = synth.uniform_points(rng, V)
    calls = [(xy0, gr.GR_METRIC_ALL, IDEAL, 64, False), (xy0, gr.GR_METRIC_ALL, IDEAL, 64, False),
             (xy0, gr.GR_METRIC_ALL, IDEAL, 128, False), (xy0, gr.GR_METRIC_CROSSINGS, IDEAL, 128, False),
             (xy0, gr.GR_METRIC_ALL, math.radians(45), 64, True), (xy0, gr.GR_METRIC_ALL, math.radians(45), 64, True),
             (far, gr.GR_METRIC_ALL, IDEAL, 64, False),  # long edges: buffers outgrown, re-run, new capture
             (far, gr.GR_METRIC_ALL, IDEAL, 64, False), (xy0, gr.GR_METRIC_OCCLUSION | gr.GR_METRIC_MIN_ANGLE,
                                                        IDEAL, 300, False), (xy0, gr.GR_METRIC_ALL, IDEAL, 64, False)]
    with gr.Layout(xy0, e, opt) as L:
        for i, (xy, m, ideal, d, prof) in enumerate(calls):
            gr.gr_profile_enable(L.handle, prof)
            L.update(xy)
            r = L.evaluate(m, ideal, d)
            with gr.Layout(xy, e, opt) as F:
                same_result(r, F.evaluate(m, ideal, d), f"call {i}")
            if prof:
                assert L.profile()["finalize"][1] > 0
