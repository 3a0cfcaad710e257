"""GPU: the batched evaluator (gr_batch_*) against the oracle and against the
single-layout entry points, layout by layout."""
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


def mixed_layouts(seed=0, n=90):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 6
        if kind == 0:
            out.append(synth.tiny_degenerate_layout(rng, int(rng.integers(3, 40)), int(rng.integers(2, 200)),
                                                    span=int(rng.integers(2, 20)),
                                                    offset=int(rng.integers(0, 65000))))
        elif kind == 1:
            V = int(rng.integers(50, 900))
            xy = synth.uniform_points(rng, V)
            e = synth.knn_edges(xy, 4, 2 * V)
            out.append(synth.Layout(xy, synth.add_random_edges(rng, V, e, V // 2)))
        elif kind == 2:  # empty layout, or vertices without edges
            V = int(rng.integers(0, 5))
            out.append(synth.Layout(synth.uniform_points(rng, V), np.zeros((0, 2), np.int32)))
        elif kind == 3:  # clustered
            V = int(rng.integers(100, 600))
            xy = synth.gaussian_mixture_points(rng, V, 3, 300.0)
            e = synth.knn_edges(xy, 5, int(2.5 * V))
            out.append(synth.Layout(xy, synth.add_random_edges(rng, V, e, V // 20)))
        elif kind == 4:  # a single edge, or a zero-length edge
            xy = np.array([[5, 5], [5, 5], [900, 40]], np.int32)
            out.append(synth.Layout(xy, np.array([[0, 1], [1, 2]], np.int32)))
        else:  # long random edges only
            V = int(rng.integers(20, 300))
            out.append(synth.Layout(synth.uniform_points(rng, V),
                                    synth.add_random_edges(rng, V, np.zeros((0, 2), np.int32), 2 * V)))
    return out


def check_layout(r, L, d, label):
    ref = oracle.crossings(L.xy, L.edges)
    c = r.crossing.c
    assert (c.proper, c.touching, c.collinear_overlaps, c.zero_length_edges) == \
        (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), label
    assert abs(r.crossing.angle_dev_sum - ref.angle_dev_sum) <= REL * max(1.0, ref.angle_dev_sum), label
    assert r.crossing.E_ca == pytest.approx(ref.E_ca, rel=REL, abs=REL), label
    assert r.occlusion_pairs == oracle.node_occlusion(L.xy, d), label
    ma = oracle.min_angle(L.xy, L.edges)
    assert r.min_angle.n_vertices_counted == ma.n_vertices, label
    assert r.min_angle.M_a == pytest.approx(ma.M_a, rel=REL, abs=REL), label
    assert r.M_l == pytest.approx(oracle.edge_length_variation(L.xy, L.edges), rel=REL, abs=1e-12), label


def test_mixed_batch_matches_oracle_and_replays_bitwise():
    layouts = mixed_layouts()
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    with gr.Batch(v_off, e_off, xy, edges) as B:
        res = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 200)
        again = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 200)  # graph replay
    for i, L in enumerate(layouts):
        check_layout(res[i], L, 200, f"layout {i}")
        assert bytes(memoryview(res[i])) == bytes(memoryview(again[i]))


def test_batch_equals_single_layout_entry_points():
    layouts = mixed_layouts(seed=3, n=36)
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    with gr.Batch(v_off, e_off, xy, edges) as B:
        res = B.evaluate(gr.GR_METRIC_ALL, math.radians(60), 90)
    for i, L in enumerate(layouts):
        if L.E == 0 and L.V < 2:
            continue
        with gr.Layout(L.xy, L.edges) as one:
            r = one.evaluate(gr.GR_METRIC_ALL, math.radians(60), 90)
        a, b = res[i], r
        assert (a.crossing.c.proper, a.crossing.c.touching, a.crossing.c.collinear_overlaps) == \
            (b.crossing.c.proper, b.crossing.c.touching, b.crossing.c.collinear_overlaps), i
        assert a.crossing.angle_dev_sum == pytest.approx(b.crossing.angle_dev_sum, rel=1e-12, abs=1e-9), i
        assert a.occlusion_pairs == b.occlusion_pairs, i
        assert a.min_angle.M_a == pytest.approx(b.min_angle.M_a, rel=1e-12), i
        assert a.M_l == pytest.approx(b.M_l, rel=1e-12, abs=1e-15), i


@pytest.mark.parametrize("long_pairs", [1, 2])
def test_batch_long_pair_forms_match_oracle(long_pairs):
    layouts = mixed_layouts(seed=9, n=48)
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    with gr.Batch(v_off, e_off, xy, edges, gr.gr_options(0, 0, 0, 0, long_pairs)) as B:
        res = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 128)
    for i, L in enumerate(layouts):
        check_layout(res[i], L, 128, f"layout {i}")


def test_batch_update_subsets_and_fixed_offsets():
    layouts = mixed_layouts(seed=5, n=24)
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    rng = np.random.default_rng(8)
    xy2 = rng.integers(0, 65536, size=xy.shape).astype(np.int32)
    for opt in (None, gr.gr_options(0, -1, 0, 0)):
        with gr.Batch(v_off, e_off, xy, edges, opt) as B:
            B.update(xy2)
            res = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 500)
            only = B.evaluate(gr.GR_METRIC_CROSSINGS, IDEAL, 500)
        for i, L in enumerate(layouts):
            L2 = synth.Layout(xy2[v_off[i]:v_off[i + 1]], L.edges)
            check_layout(res[i], L2, 500, f"layout {i}")
            assert only[i].crossing.c.crossings == res[i].crossing.c.crossings
            assert only[i].occlusion_pairs == 0 and only[i].min_angle.M_a == 1.0 and only[i].M_l == 0.0


def test_batch_errors():
    xy = np.array([[0, 0], [10, 10], [0, 10], [5, 5]], np.int32)
    v_off = np.array([0, 2, 4], np.int64)
    e_off = np.array([0, 1, 2], np.int64)
    with pytest.raises(gr.GrError) as ei:
        gr.Batch(v_off, e_off, xy, np.array([[0, 1], [0, 2]], np.int32))  # id 2 outside layout 1
    assert ei.value.status == gr.GR_EINVAL
    with pytest.raises(gr.GrError) as ei:
        gr.Batch(v_off, e_off, np.array([[0, 0], [10, 70000], [0, 10], [5, 5]], np.int32),
                 np.array([[0, 1], [0, 1]], np.int32))
    assert ei.value.status == gr.GR_ERANGE
    with pytest.raises(gr.GrError) as ei:
        gr.Batch(np.array([0, 2, 1], np.int64), e_off, xy, np.array([[0, 1], [0, 1]], np.int32))
    assert ei.value.status == gr.GR_EINVAL


def test_batched_workload_full_size():
    layouts = synth.batched_layouts()
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    import torch
    dxy, ded = torch.from_numpy(xy).cuda(), torch.from_numpy(edges).cuda()
    with gr.Batch(v_off, e_off, dxy, ded) as B:
        res = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 256)
    # every layout against the single-layout API (exact counts, same float terms)
    for i, L in enumerate(layouts):
        with gr.Layout(dxy[v_off[i]:v_off[i + 1]], ded[e_off[i]:e_off[i + 1]]) as one:
            r = one.evaluate(gr.GR_METRIC_ALL, IDEAL, 256)
        assert (res[i].crossing.c.proper, res[i].crossing.c.touching, res[i].crossing.c.collinear_overlaps) == \
            (r.crossing.c.proper, r.crossing.c.touching, r.crossing.c.collinear_overlaps), i
        assert res[i].crossing.angle_dev_sum == pytest.approx(r.crossing.angle_dev_sum, rel=1e-12), i
        assert res[i].occlusion_pairs == r.occlusion_pairs, i
        assert res[i].min_angle.M_a == pytest.approx(r.min_angle.M_a, rel=1e-12), i
        assert res[i].M_l == pytest.approx(r.M_l, rel=1e-12), i
    # a sample of layouts, stratified by size, against the oracle
    order = np.argsort(v_off[1:] - v_off[:-1])
    for i in list(order[::256][:14]):
        check_layout(res[i], layouts[i], 256, f"layout {i}")


@pytest.mark.parametrize("long_pairs", [1, 2])
def test_batch_tile_heights_agree(long_pairs, monkeypatch):
    # the pair kernel's items with 16-segment tiles (two items per warp) and
    # with 32-segment tiles give the same tallies, layout by layout, and both
    # match the oracle; the autotuner's cache keeps the tile height it chose
    layouts = mixed_layouts(seed=21, n=60)
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    res = {}
    for tile in ("16", "32"):  # the same cell sizes (a fixed offset), so the same results bit for bit
        monkeypatch.setenv("GR_BATCH_TILE", tile)
        with gr.Batch(v_off, e_off, xy, edges, gr.gr_options(0, -1, 0, 0, long_pairs)) as B:
            res[tile] = [bytes(memoryview(r)) for r in B.evaluate(gr.GR_METRIC_ALL, IDEAL, 160)]
    assert res["16"] == res["32"]
    monkeypatch.delenv("GR_BATCH_TILE")
    with gr.Batch(v_off, e_off, xy, edges, gr.gr_options(0, 0, 0, 0, long_pairs)) as B:  # autotuned
        got = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 160)
    for i, L in enumerate(layouts):
        check_layout(got[i], L, 160, f"layout {i}")


def test_autotuner_caches_offset_and_tile(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("GR_TUNE_CACHE", str(cache))
    monkeypatch.delenv("GR_BATCH_TILE", raising=False)
    layouts = mixed_layouts(seed=22, n=30)
    v_off, e_off, xy, edges = synth.pack_layouts(layouts)
    with gr.Batch(v_off, e_off, xy, edges) as B:
        first = [bytes(memoryview(r)) for r in B.evaluate(gr.GR_METRIC_ALL, IDEAL, 200)]
    key, delta, tile = cache.read_text().split()
    assert key.startswith("batch_tiled_") and int(delta) in (-1, 0, 1) and int(tile) in (16, 32)
    with gr.Batch(v_off, e_off, xy, edges) as B:  # from the cache: the same plan, the same results
        assert [bytes(memoryview(r)) for r in B.evaluate(gr.GR_METRIC_ALL, IDEAL, 200)] == first
    assert len(cache.read_text().splitlines()) == 1
