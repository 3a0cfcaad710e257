"""GPU test of gr_crossing_angle_noalloc, the entry point that allocates no
device memory (for callers that cannot call cudaMalloc: a process whose
device memory is committed to its own pool allocator, or a latency-critical
caller that cannot afford cudaMalloc / cudaFree).  It works in a fixed
scratch array inside the library, reused by every call, so this test calls it
twice in a row on different layouts and checks each result against
gr_crossing_angle on a regular layout evaluated by the same all-pairs kernel
(so even the number of pairs tested must agree).  Collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_2411_09809_gb300 import build, gr, synth

pytestmark = pytest.mark.gpu
REL = 1e-5


def _cuda(a):
    import torch
    assert torch.cuda.is_available(), "needs CUDA"
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_gr_crossing_angle_on_two_calls_in_a_row():
    build.build()
    gr.load()
    first = synth.plain_layout()                                  # 5,000 edges
    second = synth.dense_long_edge_layout(V=3000, E=20_000)       # more edges, more crossings
    for L, ideal in [(first, 0.0), (second, math.radians(60.0))]:
        xy, ed = _cuda(L.xy), _cuda(L.edges)
        got = gr.gr_crossing_angle_noalloc(xy, ed, ideal)
        with gr.Layout(xy, ed, gr.gr_options(gr.GR_PATH_ALLPAIRS, 0, 0, 0)) as lay:
            ref = gr.gr_crossing_angle(lay.handle, ideal)
        for f in ("crossings", "proper", "touching", "collinear_overlaps", "zero_length_edges", "pairs_tested"):
            assert getattr(got.c, f) == getattr(ref.c, f), f
        assert got.c.crossings > 0
        assert got.angle_dev_sum == pytest.approx(ref.angle_dev_sum, rel=REL)
        assert got.E_ca == pytest.approx(ref.E_ca, rel=REL)
        assert got.ideal_rad == pytest.approx(ref.ideal_rad, rel=1e-15)


def test_noalloc_rejects_layouts_above_its_limit():
    build.build()
    lib = gr.load()
    rng = np.random.default_rng(0)
    E = gr.GR_NOALLOC_MAX_EDGES + 1
    xy = _cuda(rng.integers(0, 65536, size=(100, 2)).astype(np.int32))
    ed = _cuda(np.stack([np.zeros(E), np.ones(E)], 1).astype(np.int32))
    out = gr.gr_crossing_angle_result()
    st = lib.gr_crossing_angle_noalloc(xy.data_ptr(), 100, ed.data_ptr(), E, 0.0, ctypes.byref(out), None)
    assert st == gr.GR_EINVAL
    assert "limit" in gr.gr_last_error()


def test_noalloc_reports_bad_inputs_and_recovers():
    # the device-side checks come back through the shared scratch accumulator:
    # a self-loop (GR_EINVAL) and a coordinate of 65536 (GR_ERANGE); a valid
    # call right after each must still equal gr_crossing_angle
    build.build()
    lib = gr.load()
    L = synth.plain_layout(V=800, knn_count=1600, random_count=400, seed=21)
    xy, ed = _cuda(L.xy), _cuda(L.edges)
    with gr.Layout(xy, ed, gr.gr_options(gr.GR_PATH_ALLPAIRS, 0, 0, 0)) as lay:
        ref = gr.gr_crossing_angle(lay.handle, 0.0)
    bad_e = L.edges.copy()
    bad_e[17] = [5, 5]
    bad_xy = L.xy.copy()
    bad_xy[3] = [65536, 10]
    for xs, es, status in [(L.xy, bad_e, gr.GR_EINVAL), (bad_xy, L.edges, gr.GR_ERANGE)]:
        bx, be = _cuda(xs), _cuda(es)
        out = gr.gr_crossing_angle_result()
        st = lib.gr_crossing_angle_noalloc(bx.data_ptr(), len(xs), be.data_ptr(), len(es), 0.0,
                                           ctypes.byref(out), None)
        assert st == status, gr.gr_last_error()
        got = gr.gr_crossing_angle_noalloc(xy, ed, 0.0)
        for f in ("crossings", "proper", "touching", "collinear_overlaps", "zero_length_edges", "pairs_tested"):
            assert getattr(got.c, f) == getattr(ref.c, f), f
        assert got.angle_dev_sum == pytest.approx(ref.angle_dev_sum, rel=REL)
