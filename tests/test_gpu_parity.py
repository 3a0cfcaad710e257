"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Counts must match exactly; float metrics within 1e-5 relative (the stated
tolerance; the FP32 angle terms are typically ~1e-7 off the FP64 oracle).
"""
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


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def check_crossings(res, ref, label=""):
    c = res.crossing.c
    assert (c.proper, c.touching, c.collinear_overlaps, c.zero_length_edges) == \
        (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), label
    assert c.crossings == ref.crossings, label
    tol = REL * max(abs(ref.angle_dev_sum), 1.0)
    assert abs(res.crossing.angle_dev_sum - ref.angle_dev_sum) <= tol, label
    assert res.crossing.E_ca == pytest.approx(ref.E_ca, rel=REL, abs=REL), label


def evaluate_all(xy, edges, d, device=True, ideal=IDEAL):
    if device:
        torch = torch_cuda()
        xy = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
        edges = torch.from_numpy(np.ascontiguousarray(edges)).cuda()
    with gr.Layout(xy, edges) as L:
        return L.evaluate(gr.GR_METRIC_ALL, ideal, d)


def check_all(xy, edges, d, res, label=""):
    check_crossings(res, oracle.crossings(xy, edges), label)
    assert res.occlusion_pairs == oracle.node_occlusion(xy, d), label
    ma = oracle.min_angle(xy, edges)
    assert res.min_angle.n_vertices_counted == ma.n_vertices, label
    assert res.min_angle.M_a == pytest.approx(ma.M_a, rel=REL, abs=REL), label
    assert res.min_angle.sum_d == pytest.approx(ma.sum_d, rel=REL, abs=REL), label
    assert res.M_l == pytest.approx(oracle.edge_length_variation(xy, edges), rel=REL, abs=1e-12), label


def test_plain_layout_all_five_metrics():
    L = synth.plain_layout()
    res = evaluate_all(L.xy, L.edges, 256)
    check_all(L.xy, L.edges, 256, res)
    assert res.crossing.c.crossings > 100_000


def test_host_and_device_inputs_agree_and_repeat_bitwise():
    L = synth.plain_layout(V=700, knn_count=1400, random_count=400, seed=5)
    a = evaluate_all(L.xy, L.edges, 300, device=True)
    b = evaluate_all(L.xy, L.edges, 300, device=False)
    c = evaluate_all(L.xy, L.edges, 300, device=True)
    for r in (b, c):
        assert bytes(memoryview(r)) == bytes(memoryview(a))  # deterministic, bit for bit


@pytest.mark.parametrize("seed", range(12))
def test_degenerate_layouts_many_tiles(seed):
    # coordinates in a tiny box: collinear, touching, coincident and zero-length
    # pairs dominate; E spans one to three 256-wide tiles with ragged tails.
    rng = np.random.default_rng(1000 + seed)
    V = int(rng.integers(3, 60))
    E = int(rng.integers(2, 700))
    L = synth.tiny_degenerate_layout(rng, V, E, span=int(rng.integers(2, 12)),
                                     offset=int(rng.integers(0, 65536 - 12)))
    d = int(rng.integers(0, 6))
    res = evaluate_all(L.xy, L.edges, d)
    check_all(L.xy, L.edges, d, res, f"seed {seed}")


def test_random_long_edges_across_tiles():
    rng = np.random.default_rng(42)
    V = 1300
    xy = synth.uniform_points(rng, V)
    e = synth.add_random_edges(rng, V, np.zeros((0, 2), np.int32), 1500)
    res = evaluate_all(xy, e, 3000)
    check_all(xy, e, 3000, res)


def test_extreme_coordinates_and_full_range_occlusion():
    # corners of the coordinate range: largest cross products and distances
    xy = np.array([[0, 0], [65535, 65535], [0, 65535], [65535, 0], [32768, 0], [32768, 65535],
                   [0, 32768], [65535, 32768], [65535, 65535]], np.int32)
    e = np.array([[0, 1], [2, 3], [4, 5], [6, 7], [0, 8], [1, 3], [2, 8]], np.int32)
    for d in (0, 1, 32768, 65536, 92682, 92683, 10**9):
        res = evaluate_all(xy, e, d)
        check_all(xy, e, d, res, f"d={d}")


def test_empty_and_trivial_layouts():
    z = np.zeros((0, 2), np.int32)
    res = evaluate_all(z, z, 5, device=False)
    assert res.crossing.c.crossings == 0 and res.crossing.E_ca == 1.0
    assert res.occlusion_pairs == 0 and res.min_angle.M_a == 1.0 and res.M_l == 0.0
    xy = np.array([[5, 5], [5, 5], [9, 9]], np.int32)
    e = np.array([[0, 1], [1, 2]], np.int32)
    res = evaluate_all(xy, e, 1)
    check_all(xy, e, 1, res)
    assert res.crossing.c.zero_length_edges == 1


def test_per_edge_crossings_match_the_oracle():
    torch = torch_cuda()
    L = synth.plain_layout(V=900, knn_count=1800, random_count=500, seed=77)
    xy = torch.from_numpy(L.xy).cuda()
    ed = torch.from_numpy(L.edges).cuda()
    counts = torch.empty((L.E, 3), dtype=torch.int64, device="cuda")
    dev = torch.empty(L.E, dtype=torch.float64, device="cuda")
    with gr.Layout(xy, ed) as lay:
        gr.gr_crossings_per_edge(lay.handle, IDEAL, counts, dev)
    ref_c, ref_d = oracle.crossings_of_edges(L.xy, L.edges, np.arange(L.E))
    assert np.array_equal(counts.cpu().numpy(), ref_c)
    np.testing.assert_allclose(dev.cpu().numpy(), ref_d, rtol=REL, atol=1e-6)


def _sampled_parity(L, n_sample, seed, d):
    torch = torch_cuda()
    xy = torch.from_numpy(L.xy).cuda()
    ed = torch.from_numpy(L.edges).cuda()
    counts = torch.empty((L.E, 3), dtype=torch.int64, device="cuda")
    dev = torch.empty(L.E, dtype=torch.float64, device="cuda")
    with gr.Layout(xy, ed) as lay:
        res = lay.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
        gr.gr_crossings_per_edge(lay.handle, IDEAL, counts, dev)
    c = counts.cpu().numpy()
    dv = dev.cpu().numpy()
    # every pair is seen from both of its edges
    assert c[:, 0].sum() == 2 * res.crossing.c.proper
    assert c[:, 1].sum() == 2 * res.crossing.c.touching
    assert c[:, 2].sum() == 2 * res.crossing.c.collinear_overlaps
    assert dv.sum() == pytest.approx(2 * res.crossing.angle_dev_sum, rel=1e-9)
    rng = np.random.default_rng(seed)
    sample = rng.choice(L.E, size=n_sample, replace=False)
    ref_c, ref_d = oracle.crossings_of_edges(L.xy, L.edges, sample)
    assert np.array_equal(c[sample], ref_c)
    np.testing.assert_allclose(dv[sample], ref_d, rtol=REL, atol=1e-6)
    # O(E) and O(V deg^2) metrics run in full on the oracle
    ma = oracle.min_angle(L.xy, L.edges)
    assert res.min_angle.n_vertices_counted == ma.n_vertices
    assert res.min_angle.M_a == pytest.approx(ma.M_a, rel=REL)
    assert res.M_l == pytest.approx(oracle.edge_length_variation(L.xy, L.edges), rel=REL)
    return res


def test_dense_long_edge_layout_full_size_sampled():
    L = synth.dense_long_edge_layout()
    res = _sampled_parity(L, 48, 3, 256)
    E = L.E
    frac = res.crossing.c.crossings / (E * (E - 1) / 2)
    assert abs(frac - 25 / 108) < 0.01  # random segments cross w.p. 25/108


def test_large_sparse_layout_full_size_sampled():
    L = synth.large_sparse_layout()
    _sampled_parity(L, 64, 4, 64)


def test_dense_long_edge_layout_full_size_totals():
    # every one of the 2.0e10 edge pairs on the oracle (tens of seconds of host work)
    L = synth.dense_long_edge_layout()
    res = evaluate_all(L.xy, L.edges, 256)
    check_crossings(res, oracle.crossings(L.xy, L.edges), "dense long-edge, all pairs")
    assert res.occlusion_pairs == oracle.node_occlusion(L.xy, 256)


def test_large_sparse_layout_full_size_totals():
    # occlusion over all 2.0e10 vertex pairs and crossings over all 1.25e11 edge
    # pairs on the oracle (about two minutes of host work on the GPU machine)
    L = synth.large_sparse_layout()
    res = evaluate_all(L.xy, L.edges, 64)
    assert res.occlusion_pairs == oracle.node_occlusion(L.xy, 64)
    check_crossings(res, oracle.crossings(L.xy, L.edges), "large sparse, all pairs")


def _expect_error(status, fn):
    with pytest.raises(gr.GrError) as ei:
        fn()
    assert ei.value.status == status


def test_error_codes():
    xy = np.array([[0, 0], [10, 10], [0, 10]], np.int32)
    _expect_error(gr.GR_EINVAL, lambda: gr.Layout(xy, np.array([[0, 3]], np.int32)))
    _expect_error(gr.GR_EINVAL, lambda: gr.Layout(xy, np.array([[1, 1]], np.int32)))
    _expect_error(gr.GR_EINVAL, lambda: gr.Layout(xy, np.array([[-1, 1]], np.int32)))
    _expect_error(gr.GR_ERANGE, lambda: gr.Layout(np.array([[0, 65536], [1, 1]], np.int32),
                                                  np.array([[0, 1]], np.int32)))
    _expect_error(gr.GR_ERANGE, lambda: gr.Layout(np.array([[0, 5], [1, 1], [-3, 0]], np.int32),
                                                  np.array([[0, 1]], np.int32)))
    with gr.Layout(xy, np.array([[0, 1], [1, 2]], np.int32)) as L:
        _expect_error(gr.GR_EINVAL, lambda: L.evaluate(gr.GR_METRIC_ALL, 0.0, -1))
        _expect_error(gr.GR_EINVAL, lambda: L.evaluate(gr.GR_METRIC_ALL, 2.0, 1))
        _expect_error(gr.GR_EINVAL, lambda: L.evaluate(1 << 7, 0.0, 1))
        # a bad update is reported by the next evaluation
        L.update(np.array([[0, 0], [70000, 1], [0, 10]], np.int32))
        _expect_error(gr.GR_ERANGE, lambda: L.evaluate())
        L.update(xy)
        assert L.evaluate().crossing.c.crossings == 0


def test_update_replaces_coordinates():
    A = synth.plain_layout(V=500, knn_count=1000, random_count=200, seed=8)
    rng = np.random.default_rng(9)
    xy2 = synth.uniform_points(rng, A.V)
    with gr.Layout(A.xy, A.edges) as L:
        r1 = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 500)
        L.update(xy2)
        r2 = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 500)
    check_all(A.xy, A.edges, 500, r1)
    check_all(xy2, A.edges, 500, r2)


def test_single_metric_entry_points():
    L = synth.plain_layout(V=400, knn_count=800, random_count=200, seed=10)
    ref = oracle.crossings(L.xy, L.edges)
    with gr.Layout(L.xy, L.edges) as lay:
        c = gr.gr_edge_crossings(lay.handle)
        assert (c.proper, c.touching, c.crossings) == (ref.proper, ref.touching, ref.crossings)
        a = gr.gr_crossing_angle(lay.handle, math.radians(45))
        assert a.E_ca == pytest.approx(oracle.crossings(L.xy, L.edges, math.radians(45)).E_ca, rel=REL)
        assert gr.gr_node_occlusion(lay.handle, 700) == oracle.node_occlusion(L.xy, 700)
        assert gr.gr_min_angle(lay.handle).M_a == pytest.approx(oracle.min_angle(L.xy, L.edges).M_a, rel=REL)
        assert gr.gr_edge_length_variation(lay.handle) == pytest.approx(
            oracle.edge_length_variation(L.xy, L.edges), rel=REL)


def test_empty_and_trivial_layouts_on_every_entry_point():
    # repeated evaluations (the replayed graph), the strip estimate and moves on
    # layouts with no edge, one vertex, or only coincident points
    z = np.zeros((0, 2), np.int32)
    cases = [(z, z), (np.array([[7, 7]], np.int32), z),
             (np.array([[5, 5], [5, 5], [9, 9]], np.int32), np.array([[0, 1], [1, 2]], np.int32)),
             (np.array([[0, 0], [65535, 65535], [0, 65535], [65535, 0]], np.int32),
              np.array([[0, 1], [2, 3]], np.int32))]
    for xy, e in cases:
        with gr.Layout(xy, e) as L:
            for _ in range(3):
                r = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 3)
                if len(xy):
                    check_all(xy, e, 3, r)
                else:
                    assert (r.crossing.c.crossings, r.occlusion_pairs, r.M_l) == (0, 0, 0.0)
            for w in (1, 1000, 65535):
                st = L.strips(w, gr.GR_STRIP_BOTH, IDEAL)
                assert st.crossings == oracle.strip_crossings(xy, e, w, 2, IDEAL).crossings
            if len(xy):
                ids = np.array([0], np.int32)
                new = np.array([[65535, 0]], np.int32)
                r = L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, 3)
                moved = xy.copy()
                moved[0] = new[0]
                check_all(moved, e, 3, r)
            r = L.move(np.zeros(0, np.int32), np.zeros((0, 2), np.int32), gr.GR_METRIC_ALL, IDEAL, 3)
            assert r.crossing.c.crossings == (oracle.crossings(moved, e).crossings if len(xy) else 0)
