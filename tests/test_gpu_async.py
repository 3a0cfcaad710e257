"""GPU: the asynchronous evaluations (gr_evaluate_async, gr_batch_evaluate_async)
write the same results as the synchronous calls into device memory, follow
updates in stream order, run on a caller's stream, mark failures with
metrics = 0, and can be captured into the caller's CUDA graph."""
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


def torch_cuda():
    import torch
    return torch


def same(a, b, label=""):
    assert a.metrics == b.metrics, label
    ca, cb = a.crossing.c, b.crossing.c
    assert (ca.proper, ca.touching, ca.collinear_overlaps, ca.zero_length_edges) == \
        (cb.proper, cb.touching, cb.collinear_overlaps, cb.zero_length_edges), label
    assert a.crossing.angle_dev_sum == b.crossing.angle_dev_sum, label
    assert a.occlusion_pairs == b.occlusion_pairs and a.min_angle.M_a == b.min_angle.M_a and a.M_l == b.M_l, label


@pytest.mark.parametrize("opt", [None, gr.gr_options(gr.GR_PATH_ALLPAIRS, 0, gr.GR_PATH_ALLPAIRS, 0)])
def test_async_evaluations_follow_updates(opt):
    torch = torch_cuda()
    rng = np.random.default_rng(41)
    L0 = synth.plain_layout(V=3000, knn_count=6000, random_count=1500, seed=42)
    steps = [L0.xy] + [np.clip(L0.xy + rng.integers(-500, 501, size=L0.xy.shape), 0, 65535).astype(np.int32)
                       for _ in range(4)]
    buf = gr.result_buffer(len(steps))
    size = buf.numel() // len(steps)
    with gr.Layout(torch.from_numpy(L0.xy).cuda(), torch.from_numpy(L0.edges).cuda(), opt) as L:
        # the first call plans (one synchronisation); the rest only enqueue
        for i, xy in enumerate(steps):
            L.update(torch.from_numpy(xy).cuda())
            L.evaluate_async(buf[i * size:(i + 1) * size], gr.GR_METRIC_ALL, IDEAL, 200)
        torch.cuda.synchronize()
        got = gr.results_from_device(buf, len(steps))
    for i, xy in enumerate(steps):
        with gr.Layout(xy, L0.edges) as F:
            same(got[i], F.evaluate(gr.GR_METRIC_ALL, IDEAL, 200), f"step {i}")
    ref = oracle.crossings(steps[-1], L0.edges)
    assert got[-1].crossing.c.proper == ref.proper


def test_async_on_a_caller_stream_and_failure_marking():
    torch = torch_cuda()
    L0 = synth.plain_layout(V=2000, knn_count=4000, random_count=1000, seed=43)
    side = torch.cuda.Stream()
    buf = gr.result_buffer(1)
    with gr.Layout(torch.from_numpy(L0.xy).cuda(), torch.from_numpy(L0.edges).cuda()) as L:
        want = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 256)
        with torch.cuda.stream(side):
            buf.zero_()
            L.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, 256, stream=side)
        side.synchronize()
        same(gr.results_from_device(buf)[0], want, "caller stream")
        # invalid coordinates: the asynchronous result says so, the synchronous call gives the error
        bad = L0.xy.copy()
        bad[5] = (70000, 3)
        L.update(bad)
        L.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, 256)
        torch.cuda.synchronize()
        assert gr.results_from_device(buf)[0].metrics == 0
        with pytest.raises(gr.GrError) as ei:
            L.evaluate(gr.GR_METRIC_ALL, IDEAL, 256)
        assert ei.value.status == gr.GR_ERANGE


def test_async_evaluation_in_a_captured_cuda_graph():
    torch = torch_cuda()
    L0 = synth.plain_layout(V=2500, knn_count=5000, random_count=800, seed=44)
    rng = np.random.default_rng(45)
    xy_dev = torch.from_numpy(L0.xy).cuda()
    buf = gr.result_buffer(1)
    with gr.Layout(xy_dev, torch.from_numpy(L0.edges).cuda()) as L:
        L.evaluate(gr.GR_METRIC_ALL, IDEAL, 128)   # plans and sizes the buffers
        L.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, 128)  # the layout's own graph of this configuration
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            L.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, 128, stream=torch.cuda.current_stream())
        for step in range(3):
            xy = np.clip(L0.xy + rng.integers(-300, 301, size=L0.xy.shape), 0, 65535).astype(np.int32)
            L.update(torch.from_numpy(xy).cuda())
            torch.cuda.synchronize()  # the inputs are in place before the replay
            g.replay()
            torch.cuda.synchronize()
            with gr.Layout(xy, L0.edges) as F:
                same(gr.results_from_device(buf)[0], F.evaluate(gr.GR_METRIC_ALL, IDEAL, 128), f"replay {step}")


def test_batch_async_matches_sync():
    torch = torch_cuda()
    rng = np.random.default_rng(46)
    layouts = [synth.plain_layout(V=int(v), knn_count=int(2 * v), random_count=int(v // 2), seed=50 + i)
               for i, v in enumerate(rng.integers(60, 1500, size=12))]
    v_off = np.concatenate([[0], np.cumsum([l.V for l in layouts])]).astype(np.int64)
    e_off = np.concatenate([[0], np.cumsum([l.E for l in layouts])]).astype(np.int64)
    xy = np.concatenate([l.xy for l in layouts]).astype(np.int32)
    edges = np.concatenate([l.edges for l in layouts]).astype(np.int32)
    with gr.Batch(v_off, e_off, xy, edges) as B:
        want = B.evaluate(gr.GR_METRIC_ALL, IDEAL, 256)
        buf = gr.result_buffer(len(layouts))
        B.evaluate_async(buf, gr.GR_METRIC_ALL, IDEAL, 256)
        torch.cuda.synchronize()
        got = gr.results_from_device(buf, len(layouts))
    for i in range(len(layouts)):
        same(got[i], want[i], f"layout {i}")
