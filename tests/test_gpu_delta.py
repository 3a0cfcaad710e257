"""GPU: incremental re-evaluation after moving vertices (gr_move_vertices)
equals a full evaluation of the moved layout -- counts and the integer
crossing-angle sum bit for bit -- and the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2411_09809_gb300 import build, gr, synth

pytestmark = pytest.mark.gpu
IDEAL = 7 * math.pi / 18


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gr.load()


def full(xy, e, d, ideal=IDEAL):
    with gr.Layout(np.ascontiguousarray(xy, np.int32), e) as L:
        return L.evaluate(gr.GR_METRIC_ALL, ideal, d)


def same(a, b, label):
    ca, cb = a.crossing.c, b.crossing.c
    assert (ca.proper, ca.touching, ca.collinear_overlaps, ca.zero_length_edges) == \
        (cb.proper, cb.touching, cb.collinear_overlaps, cb.zero_length_edges), label
    assert a.crossing.angle_dev_sum == b.crossing.angle_dev_sum, label  # the same integer sum
    assert a.occlusion_pairs == b.occlusion_pairs, label
    assert a.min_angle.M_a == pytest.approx(b.min_angle.M_a, rel=1e-12, abs=1e-15), label
    assert a.M_l == pytest.approx(b.M_l, rel=1e-12, abs=1e-15), label


def test_moves_match_full_evaluation_and_oracle():
    rng = np.random.default_rng(3)
    L0 = synth.plain_layout(V=1500, knn_count=3000, random_count=600, seed=77)
    xy = L0.xy.copy()
    d = 300
    with gr.Layout(xy, L0.edges) as L:
        L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
        for step, n in enumerate([1, 3, 17, 120, 1, 400]):
            ids = rng.choice(L0.V, size=n, replace=False).astype(np.int32)
            new = rng.integers(0, 65536, size=(n, 2)).astype(np.int32)
            if step == 4:  # onto another vertex: zero-length edges, coincident points
                new[:] = xy[(ids + 1) % L0.V]
            xy[ids] = new
            r = L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, d)
            assert r.crossing_path == gr.GR_PATH_DELTA and r.occlusion_path == gr.GR_PATH_DELTA
            same(r, full(xy, L0.edges, d), f"step {step}")
        ref = oracle.crossings(xy, L0.edges)
        c = r.crossing.c
        assert (c.proper, c.touching, c.collinear_overlaps) == (ref.proper, ref.touching, ref.collinear)
        assert r.occlusion_pairs == oracle.node_occlusion(xy, d)


def test_degenerate_moves_on_a_small_box():
    # every vertex in a 12 x 12 box: moves create collinear overlaps and touching pairs
    rng = np.random.default_rng(5)
    L0 = synth.tiny_degenerate_layout(rng, 60, 400, span=12, offset=40000)
    xy = L0.xy.copy()
    with gr.Layout(xy, L0.edges) as L:
        L.evaluate(gr.GR_METRIC_ALL, IDEAL, 3)
        for step in range(6):
            ids = rng.choice(60, size=int(rng.integers(1, 20)), replace=False).astype(np.int32)
            new = (40000 + rng.integers(0, 12, size=(len(ids), 2))).astype(np.int32)
            xy[ids] = new
            same(L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, 3), full(xy, L0.edges, 3), f"step {step}")


def test_parameter_change_falls_back_and_errors_leave_the_layout():
    L0 = synth.plain_layout(V=800, knn_count=1600, random_count=200, seed=5)
    xy = L0.xy.copy()
    with gr.Layout(xy, L0.edges) as L:
        L.evaluate(gr.GR_METRIC_CROSSINGS, IDEAL, 0)
        ids = np.array([3, 9], np.int32)
        new = np.array([[10, 10], [60000, 60000]], np.int32)
        xy[ids] = new
        r = L.move(ids, new, gr.GR_METRIC_ALL, math.radians(60), 100)  # other metrics and angle: full
        assert r.crossing_path in (gr.GR_PATH_GRID, gr.GR_PATH_ALLPAIRS)
        same(r, full(xy, L0.edges, 100, math.radians(60)), "fallback")
        for bad_ids, bad_xy, status in [([5, 5], [[1, 1], [2, 2]], gr.GR_EINVAL),
                                        ([800], [[1, 1]], gr.GR_EINVAL),
                                        ([-1], [[1, 1]], gr.GR_EINVAL),
                                        ([7], [[70000, 1]], gr.GR_ERANGE)]:
            with pytest.raises(gr.GrError) as ei:
                L.move(np.array(bad_ids, np.int32), np.array(bad_xy, np.int32), gr.GR_METRIC_ALL,
                       math.radians(60), 100)
            assert ei.value.status == status
        # unchanged by the errors, and the next move is incremental again
        ids = np.array([11], np.int32)
        new = np.array([[123, 456]], np.int32)
        xy[ids] = new
        r = L.move(ids, new, gr.GR_METRIC_ALL, math.radians(60), 100)
        assert r.crossing_path == gr.GR_PATH_DELTA
        same(r, full(xy, L0.edges, 100, math.radians(60)), "after errors")


def test_move_on_the_large_sparse_layout():
    import torch
    L0 = synth.large_sparse_layout()
    xy = L0.xy.copy()
    rng = np.random.default_rng(9)
    with gr.Layout(torch.from_numpy(xy).cuda(), torch.from_numpy(L0.edges).cuda()) as L:
        L.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
        ids = rng.choice(L0.V, size=64, replace=False).astype(np.int32)
        new = rng.integers(0, 65536, size=(64, 2)).astype(np.int32)
        xy[ids] = new
        r = L.move(torch.from_numpy(ids).cuda(), torch.from_numpy(new).cuda(), gr.GR_METRIC_ALL, IDEAL, 64)
        assert r.crossing_path == gr.GR_PATH_DELTA
        assert r.crossing.c.pairs_tested < L0.E * (L0.E - 1) // 100  # far below a full evaluation
        same(r, full(xy, L0.edges, 64), "large sparse")


def test_subset_metrics_empty_moves_and_errors_before_the_first_evaluation():
    rng = np.random.default_rng(11)
    L0 = synth.plain_layout(V=900, knn_count=1800, random_count=300, seed=8)
    xy = L0.xy.copy()
    with gr.Layout(xy, L0.edges) as L:
        # no evaluation yet: an invalid move is refused and changes nothing
        with pytest.raises(gr.GrError) as ei:
            L.move(np.array([2, 2], np.int32), np.array([[5, 5], [6, 6]], np.int32), gr.GR_METRIC_ALL, IDEAL, 50)
        assert ei.value.status == gr.GR_EINVAL
        r = L.move(np.zeros(0, np.int32), np.zeros((0, 2), np.int32), gr.GR_METRIC_ALL, IDEAL, 50)
        same(r, full(xy, L0.edges, 50), "empty move, full evaluation")
        r = L.move(np.zeros(0, np.int32), np.zeros((0, 2), np.int32), gr.GR_METRIC_ALL, IDEAL, 50)
        assert r.crossing_path == gr.GR_PATH_DELTA
        same(r, full(xy, L0.edges, 50), "empty move, incremental")
        for step in range(4):  # crossings only: still incremental after an evaluation of all five
            ids = rng.choice(L0.V, size=9, replace=False).astype(np.int32)
            new = rng.integers(0, 65536, size=(9, 2)).astype(np.int32)
            xy[ids] = new
            r = L.move(ids, new, gr.GR_METRIC_CROSSINGS, IDEAL, 50)
            assert r.crossing_path == gr.GR_PATH_DELTA
            f = full(xy, L0.edges, 50)
            assert (r.crossing.c.proper, r.crossing.c.touching, r.crossing.c.collinear_overlaps) == \
                (f.crossing.c.proper, f.crossing.c.touching, f.crossing.c.collinear_overlaps)
            assert r.crossing.angle_dev_sum == f.crossing.angle_dev_sum
        # the occlusion total was not kept up by crossing-only moves: a full evaluation again
        r = L.move(np.zeros(0, np.int32), np.zeros((0, 2), np.int32), gr.GR_METRIC_ALL, IDEAL, 50)
        assert r.crossing_path != gr.GR_PATH_DELTA
        same(r, full(xy, L0.edges, 50), "after crossing-only moves")


def grid_opt(k, long_pairs=gr.GR_LONG_AUTO):
    return gr.gr_options(crossing_path=gr.GR_PATH_GRID, cell_log2=k, long_pairs=long_pairs)


@pytest.mark.parametrize("k,long_pairs", [(6, gr.GR_LONG_AUTO), (9, gr.GR_LONG_ALLPAIRS), (9, gr.GR_LONG_GRID),
                                          (12, gr.GR_LONG_AUTO)])
def test_moves_through_the_crossing_grid(k, long_pairs):
    # the last full evaluation's grid indexes the unmoved edges; moved ones
    # accumulate in the dirty list across moves
    rng = np.random.default_rng(21 + k)
    L0 = synth.plain_layout(V=1500, knn_count=3000, random_count=600, seed=78)
    xy = L0.xy.copy()
    d = 300
    with gr.Layout(xy, L0.edges, opt=grid_opt(k, long_pairs)) as L:
        r = L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
        assert r.crossing_path == gr.GR_PATH_GRID and r.cell_log2 == k
        for step, n in enumerate([1, 5, 2, 40, 1, 3, 150]):
            ids = rng.choice(L0.V, size=n, replace=False).astype(np.int32)
            if step % 2:  # small steps, as a layout optimiser takes them
                new = np.clip(xy[ids] + rng.integers(-300, 301, size=(n, 2)), 0, 65535).astype(np.int32)
            else:
                new = rng.integers(0, 65536, size=(n, 2)).astype(np.int32)
            if step == 4:  # onto a neighbour: a zero-length edge and coincident points
                nb = L0.edges[L0.edges[:, 0] == ids[0], 1]
                new[0] = xy[nb[0]] if len(nb) else xy[(ids[0] + 1) % L0.V]
            xy[ids] = new
            r = L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, d)
            assert r.crossing_path == gr.GR_PATH_DELTA
            same(r, full(xy, L0.edges, d), f"k {k} step {step}")
        ref = oracle.crossings(xy, L0.edges)
        c = r.crossing.c
        assert (c.proper, c.touching, c.collinear_overlaps) == (ref.proper, ref.touching, ref.collinear)


def test_degenerate_moves_through_a_grid_across_cell_borders():
    # a 12 x 12 box across the cell lines x, y = 40000 (cells of side 64):
    # owner rules on cell borders and corners, collinear chains, touching pairs
    rng = np.random.default_rng(6)
    L0 = synth.tiny_degenerate_layout(rng, 80, 500, span=12, offset=39994)
    xy = L0.xy.copy()
    with gr.Layout(xy, L0.edges, opt=grid_opt(6, gr.GR_LONG_GRID)) as L:
        assert L.evaluate(gr.GR_METRIC_ALL, IDEAL, 3).crossing_path == gr.GR_PATH_GRID
        for step in range(8):
            ids = rng.choice(80, size=int(rng.integers(1, 12)), replace=False).astype(np.int32)
            new = (39994 + rng.integers(0, 12, size=(len(ids), 2))).astype(np.int32)
            xy[ids] = new
            r = L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, 3)
            assert r.crossing_path == gr.GR_PATH_DELTA
            same(r, full(xy, L0.edges, 3), f"step {step}")


def test_dirty_list_overflow_rebuilds_the_grid():
    # the dirty list holds max(4096, E / 32) edges: moving more falls back to a
    # full evaluation (a new grid), after which moves are incremental again
    rng = np.random.default_rng(12)
    L0 = synth.plain_layout(V=3000, knn_count=6000, random_count=1000, seed=13)
    xy = L0.xy.copy()
    with gr.Layout(xy, L0.edges, opt=grid_opt(10)) as L:
        L.evaluate(gr.GR_METRIC_ALL, IDEAL, 100)
        paths = []
        for step in range(5):
            ids = rng.choice(L0.V, size=700, replace=False).astype(np.int32)
            new = rng.integers(0, 65536, size=(700, 2)).astype(np.int32)
            xy[ids] = new
            r = L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, 100)
            paths.append(r.crossing_path)
            same(r, full(xy, L0.edges, 100), f"step {step}")
        assert gr.GR_PATH_GRID in paths[1:]  # a rebuild
        assert paths[0] == gr.GR_PATH_DELTA and paths[-1] == gr.GR_PATH_DELTA


@pytest.mark.parametrize("opt", [None, grid_opt(9), grid_opt(11, gr.GR_LONG_ALLPAIRS)])
def test_long_random_move_sequence_with_interleaved_evaluations(opt):
    # 60 moves of 1-60 vertices (local steps, jumps, onto other vertices), with
    # synchronous and asynchronous full evaluations in between: every state
    # transition (incremental, full, dirty-list growth) against fresh layouts
    import torch
    rng = np.random.default_rng(71)
    L0 = synth.plain_layout(V=3000, knn_count=6000, random_count=1200, seed=72)
    xy = L0.xy.copy()
    d = 150
    buf = gr.result_buffer(1)
    with gr.Layout(torch.from_numpy(xy).cuda(), torch.from_numpy(L0.edges).cuda(), opt=opt) as L:
        L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
        for step in range(60):
            n = int(rng.integers(1, 61))
            ids = rng.choice(L0.V, size=n, replace=False).astype(np.int32)
            kind = step % 3
            if kind == 0:
                new = np.clip(xy[ids] + rng.integers(-150, 151, size=(n, 2)), 0, 65535).astype(np.int32)
            elif kind == 1:
                new = rng.integers(0, 65536, size=(n, 2)).astype(np.int32)
            else:
                new = xy[rng.integers(0, L0.V, size=n)].astype(np.int32)
            xy[ids] = new
            r = L.move(torch.from_numpy(ids).cuda(), torch.from_numpy(new).cuda(), gr.GR_METRIC_ALL, IDEAL, d)
            if step % 10 == 4:
                L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
            if step % 10 == 7:
                L.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, d)
                torch.cuda.synchronize()
                got = gr.results_from_device(buf)[0]
                if got.metrics == 0:
                    # the moves outgrew the buffers planned at the last synchronous evaluation: the
                    # asynchronous result says so, a synchronous evaluation re-plans, and then it works
                    L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
                    L.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, d)
                    torch.cuda.synchronize()
                    got = gr.results_from_device(buf)[0]
                same(got, full(xy, L0.edges, d), f"async after step {step}")
            if step % 5 == 0 or step == 59:
                same(r, full(xy, L0.edges, d), f"step {step}")
