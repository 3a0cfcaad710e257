"""GPU: the differentiable (FP32) form through the C ABI against the oracle's FP32
form -- exact crossing counts, terms within 1e-5, gradients within 1e-5 in norm
of the oracle's FP64 gradients -- and the torch.autograd wrapper."""
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


def cuda(a):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def random_float_layout(seed, V, knn, extra, scale=1.0, offset=0.0):
    rng = np.random.default_rng(seed)
    xy = (offset + scale * rng.random((V, 2))).astype(np.float32)
    e = synth.knn_edges(xy, 5, knn)
    return xy, synth.add_random_edges(rng, V, e, extra)


def check_forward(xy, edges, res, label, ideal=IDEAL):
    ref = oracle.crossings_f32(xy, edges, ideal)
    c = res.crossing.c
    assert (c.proper, c.touching, c.collinear_overlaps, c.zero_length_edges) == \
        (ref.proper, ref.touching, ref.collinear, ref.zero_length_edges), label
    assert abs(res.crossing.angle_dev_sum - ref.angle_dev_sum) <= REL * max(1.0, ref.angle_dev_sum), label
    assert res.crossing.E_ca == pytest.approx(ref.E_ca, rel=REL, abs=REL), label
    ma = oracle.min_angle_f32(xy, edges)
    assert res.min_angle.n_vertices_counted == ma.n_vertices, label
    assert res.min_angle.M_a == pytest.approx(ma.M_a, rel=REL, abs=REL), label
    assert res.M_l == pytest.approx(oracle.edge_length_variation_f32(xy, edges), rel=REL, abs=1e-12), label


FWD = gr.GR_METRIC_CROSSINGS | gr.GR_METRIC_MIN_ANGLE | gr.GR_METRIC_EDGE_LENGTH


@pytest.mark.parametrize("seed", range(4))
def test_fp32_evaluate_matches_oracle(seed):
    xy, e = random_float_layout(seed, 3000, 6500, 1500, scale=float(10.0 ** (seed - 1)), offset=seed * 100.0)
    with gr.Layout(cuda(xy), cuda(e), coord_type=gr.GR_COORD_F32) as L:
        check_forward(xy, e, L.evaluate(FWD, IDEAL), f"seed {seed}")
        check_forward(xy, e, L.evaluate(FWD, math.radians(45)), f"seed {seed} 45", math.radians(45))


def test_fp32_degenerate_layouts_exact():
    # coordinates k / 64 on a tiny span: collinear overlaps, touching, zero-length,
    # duplicate edges; host buffers this time
    rng = np.random.default_rng(11)
    for t in range(12):
        L0 = synth.tiny_degenerate_layout(rng, int(rng.integers(3, 50)), int(rng.integers(1, 300)),
                                          span=int(rng.integers(2, 12)))
        xy = (L0.xy.astype(np.float64) / 64.0 - 0.5).astype(np.float32)
        with gr.Layout(xy, L0.edges, coord_type=gr.GR_COORD_F32) as L:
            check_forward(xy, L0.edges, L.evaluate(FWD, IDEAL), f"trial {t}")


def test_fp32_layout_rejects_non_finite_and_occlusion():
    xy = np.array([[0.0, 0.0], [1.0, np.inf], [0.5, 0.5]], np.float32)
    e = np.array([[0, 1], [1, 2]], np.int32)
    with pytest.raises(gr.GrError) as ei:
        gr.Layout(xy, e, coord_type=gr.GR_COORD_F32)
    assert ei.value.status == gr.GR_ERANGE
    xy[1, 1] = 2.0
    with gr.Layout(xy, e, coord_type=gr.GR_COORD_F32) as L:
        with pytest.raises(gr.GrError) as ei:
            L.evaluate(gr.GR_METRIC_OCCLUSION, IDEAL, 10)
        assert ei.value.status == gr.GR_ENOTSUP
        with pytest.raises(gr.GrError) as ei:
            gr.gr_diff_backward(L.handle, np.ones(3, np.float32), cuda(np.zeros((3, 2), np.float32)))
        assert ei.value.status == gr.GR_EINVAL  # no forward yet
    with gr.Layout(xy.astype(np.int32), e) as L:
        with pytest.raises(gr.GrError) as ei:
            gr.gr_diff_forward(L.handle, IDEAL)
        assert ei.value.status == gr.GR_ENOTSUP


def grad_close(g, ref, label):
    """The gradient matches the FP64 oracle gradient in norm (relative 1e-5) and
    coordinate by coordinate: |g - g_ref| <= 1e-5 |g_ref| + 1e-6 max |g_ref|, so
    a few wrong coordinates (a mis-scattered endpoint of one pair, a vertex whose
    smallest gap was taken at another pair of directions) cannot hide under the
    norm of the rest."""
    g = g.astype(np.float64)
    err = np.linalg.norm(g - ref)
    assert err <= REL * max(np.linalg.norm(ref), 1e-30), (label, err, np.linalg.norm(ref))
    floor = 1e-6 * max(float(np.abs(ref).max(initial=0.0)), 1e-30)
    bad = np.abs(g - ref) > REL * np.abs(ref) + floor
    if bad.any():
        i = np.flatnonzero(bad.reshape(-1))[:5]
        raise AssertionError(f"{label}: {int(bad.sum())} coordinates off, first {i.tolist()}: "
                             f"{g.reshape(-1)[i].tolist()} vs {ref.reshape(-1)[i].tolist()}")


@pytest.mark.parametrize("seed", range(3))
def test_diff_forward_and_gradients_match_oracle(seed):
    xy, e = random_float_layout(100 + seed, 4000, 9000, 2000)
    terms, g_eca, g_ml, g_ma = oracle.diff_terms_and_grads(xy, e, IDEAL)
    with gr.Layout(cuda(xy), cuda(e), coord_type=gr.GR_COORD_F32) as L:
        out = gr.gr_diff_forward(L.handle, IDEAL)
        assert out == pytest.approx(terms, rel=REL, abs=REL)
        grads = []
        for k in range(3):
            gout = np.zeros(3, np.float32)
            gout[k] = 1.0
            d = cuda(np.full((len(xy), 2), np.nan, np.float32))
            gr.gr_diff_backward(L.handle, gout, d)  # host gout: synchronous
            grads.append(d.cpu().numpy())
        for k, (g, ref) in enumerate(zip(grads, (g_eca, g_ml, g_ma))):
            grad_close(g, ref, f"term {k}")
        # a combination equals the combination of the parts (device gout, stream-ordered)
        w = np.array([-1.0, 2.0, 0.5], np.float32)
        d = cuda(np.zeros((len(xy), 2), np.float32))
        gr.gr_diff_backward(L.handle, cuda(w), d)
        grad_close(d.cpu().numpy(), w[0] * g_eca + w[1] * g_ml + w[2] * g_ma, "combination")


def test_diff_many_crossings_and_update_invalidates():
    # many crossings (long random edges, far more than edges), then an update
    # that invalidates the forward the backward would use
    rng = np.random.default_rng(7)
    V = 1500
    xy = rng.random((V, 2)).astype(np.float32)
    e = synth.add_random_edges(rng, V, np.zeros((0, 2), np.int32), 4000)
    with gr.Layout(cuda(xy), cuda(e), coord_type=gr.GR_COORD_F32) as L:
        for it in range(2):
            terms, g_eca, _, _ = oracle.diff_terms_and_grads(xy, e, IDEAL)
            out = gr.gr_diff_forward(L.handle, IDEAL)
            assert out == pytest.approx(terms, rel=REL, abs=REL)
            d = cuda(np.zeros((V, 2), np.float32))
            gr.gr_diff_backward(L.handle, np.array([1, 0, 0], np.float32), d)
            grad_close(d.cpu().numpy(), g_eca, f"iteration {it}")
            xy = (xy * np.float32(0.5) + np.float32(0.25)).astype(np.float32)
            L.update(cuda(xy))
            with pytest.raises(gr.GrError):
                gr.gr_diff_backward(L.handle, np.array([1, 0, 0], np.float32), d)


def test_autograd_loss_gradient_and_descent():
    import torch
    from paper_2411_09809_gb300.autograd import ReadabilityTerms, readability_loss
    xy_np, e = random_float_layout(5, 2000, 4500, 800)
    terms_ref, g_eca, g_ml, g_ma = oracle.diff_terms_and_grads(xy_np, e, IDEAL)
    mod = ReadabilityTerms(cuda(e), IDEAL)
    xy = cuda(xy_np).requires_grad_(True)
    terms = mod(xy)
    loss = readability_loss(terms)
    loss.backward()
    assert terms.detach().cpu().numpy() == pytest.approx(terms_ref, rel=REL, abs=REL)
    grad_close(xy.grad.cpu().numpy(), -g_eca + g_ml - g_ma, "loss gradient")
    # a few small gradient steps lower the loss
    opt = torch.optim.SGD([xy], lr=1e-5)
    first = float(loss)
    for _ in range(5):
        opt.zero_grad()
        loss = readability_loss(mod(xy))
        loss.backward()
        opt.step()
    assert float(readability_loss(mod(xy.detach()))) < first
    # a second forward before the first backward is an error, not a wrong gradient
    t1 = mod(xy)
    mod(xy)
    with pytest.raises(RuntimeError):
        readability_loss(t1).backward()
    mod.close()


def test_differentiable_workload_full_size():
    L0 = synth.differentiable_layout()
    xy, e = L0.xy, L0.edges
    # one oracle pass (about a minute of host work): counts, terms and gradients
    terms, g_eca, g_ml, g_ma, counts = oracle.diff_terms_and_grads(xy, e, IDEAL, return_counts=True)
    with gr.Layout(cuda(xy), cuda(e), coord_type=gr.GR_COORD_F32) as L:
        r = L.evaluate(FWD, IDEAL)
        c = r.crossing.c
        assert [c.proper, c.touching, c.collinear_overlaps, c.zero_length_edges, c.crossings] == list(counts)
        assert r.crossing.E_ca == pytest.approx(terms[0], rel=REL)
        assert r.M_l == pytest.approx(terms[1], rel=REL)
        assert r.min_angle.M_a == pytest.approx(terms[2], rel=REL)
        out = gr.gr_diff_forward(L.handle, IDEAL)
        assert out == pytest.approx(terms, rel=REL, abs=REL)
        d = cuda(np.zeros((len(xy), 2), np.float32))
        gr.gr_diff_backward(L.handle, np.array([-1, 1, -1], np.float32), d)
        grad_close(d.cpu().numpy(), -g_eca + g_ml - g_ma, "full size")


def f32_forward(xy, e, path=0):
    with gr.Layout(cuda(xy), cuda(e), gr.gr_options(path, 0, 0, 0), coord_type=gr.GR_COORD_F32) as L:
        return L.evaluate(FWD, IDEAL)


@pytest.mark.parametrize("seed", range(6))
def test_fp32_grid_on_degenerate_layouts(seed):
    # enough edges for the grid; coordinates k / 64 in a small box: collinear
    # overlaps, touching, coincident endpoints, duplicate edges, lines along cell edges
    rng = np.random.default_rng(300 + seed)
    L0 = synth.tiny_degenerate_layout(rng, 400, 3000, span=int(rng.integers(3, 60)))
    xy = (L0.xy.astype(np.float64) / 64.0 + [0.0, 3.0, -7.5, 1e3, 0.25, -1e4][seed]).astype(np.float32)
    r = f32_forward(xy, L0.edges)
    check_forward(xy, L0.edges, r, f"seed {seed}")
    a = f32_forward(xy, L0.edges, gr.GR_PATH_ALLPAIRS)
    assert r.crossing.angle_dev_sum == pytest.approx(a.crossing.angle_dev_sum, rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("case", ["lattice", "offset", "wide", "clustered"])
def test_fp32_grid_matches_allpairs_and_oracle(case):
    rng = np.random.default_rng({"lattice": 1, "offset": 2, "wide": 3, "clustered": 4}[case])
    V = 2500
    if case == "lattice":  # vertices on the grid's own lines (the bounding box is [0, 1])
        xy = (rng.integers(0, 65, size=(V, 2)) / 64.0).astype(np.float32)
        xy[0], xy[1] = (0.0, 0.0), (1.0, 1.0)
    elif case == "offset":  # coordinates far from the origin: cells a few FP32 ulps wide
        xy = (1.0e5 + rng.random((V, 2)) * 0.25).astype(np.float32)
    elif case == "wide":  # exponents over many binades
        xy = (np.sign(rng.random((V, 2)) - 0.5) * 2.0 ** rng.uniform(-30, 30, size=(V, 2))).astype(np.float32)
    else:
        xy = (rng.normal(0.5, 0.01, size=(V, 2))).astype(np.float32)
        xy[: V // 10] = rng.random((V // 10, 2)).astype(np.float32)
    e = synth.add_random_edges(rng, V, synth.knn_edges(xy.astype(np.float64), 3, 5000), 600)
    r = f32_forward(xy, e)
    check_forward(xy, e, r, case)
    a = f32_forward(xy, e, gr.GR_PATH_ALLPAIRS)
    assert (r.crossing.c.proper, r.crossing.c.touching, r.crossing.c.collinear_overlaps) == \
        (a.crossing.c.proper, a.crossing.c.touching, a.crossing.c.collinear_overlaps)


def test_fp32_grid_gradients_equal_allpairs_gradients():
    xy, e = random_float_layout(77, 6000, 14000, 900)
    grads = []
    for path in (0, gr.GR_PATH_ALLPAIRS):
        with gr.Layout(cuda(xy), cuda(e), gr.gr_options(path, 0, 0, 0), coord_type=gr.GR_COORD_F32) as L:
            out = gr.gr_diff_forward(L.handle, IDEAL)
            d = cuda(np.zeros((len(xy), 2), np.float32))
            gr.gr_diff_backward(L.handle, np.array([-1, 1, -1], np.float32), d)
            grads.append((out.copy(), d.cpu().numpy().astype(np.float64)))
    assert np.array_equal(grads[0][0], grads[1][0])
    g0, g1 = grads[0][1], grads[1][1]
    assert np.linalg.norm(g0 - g1) <= 1e-6 * np.linalg.norm(g1)


def test_diff_calls_on_a_caller_stream_and_in_a_captured_graph():
    # the backward ordered on another stream without a host synchronisation, and
    # captured into a CUDA graph whose replays follow the last forward before them,
    # also after a forward with far more crossings
    import torch
    xy, e = random_float_layout(55, 3000, 6500, 300)
    V = len(xy)
    s = torch.cuda.Stream()
    gout = cuda(np.array([-1.0, 1.0, -1.0], np.float32))
    with gr.Layout(cuda(xy), cuda(e), coord_type=gr.GR_COORD_F32) as L:
        out = cuda(np.zeros(3, np.float32))
        gr.gr_diff_forward(L.handle, IDEAL, out, s.cuda_stream)
        terms, g_eca, g_ml, g_ma = oracle.diff_terms_and_grads(xy, e, IDEAL)
        assert out.cpu().numpy() == pytest.approx(terms, rel=REL, abs=REL)
        want = -g_eca + g_ml - g_ma
        d = cuda(np.full((V, 2), np.nan, np.float32))
        with torch.cuda.stream(s):
            gr.gr_diff_backward(L.handle, gout, d, s.cuda_stream)
            d2 = d * 2.0  # later work on the same stream sees the gradient
        torch.cuda.synchronize()
        grad_close(d.cpu().numpy(), want, "caller stream")
        grad_close(d2.cpu().numpy() / 2.0, want, "after, on the caller stream")
        g = torch.cuda.CUDAGraph()
        gd = cuda(np.zeros((V, 2), np.float32))
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            gr.gr_diff_backward(L.handle, gout, gd, torch.cuda.current_stream().cuda_stream)
        gd.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        grad_close(gd.cpu().numpy(), want, "graph replay")
        # random positions turn the nearest-neighbour edges into long ones: millions of
        # crossings
        xy2 = np.random.default_rng(56).random((V, 2)).astype(np.float32)
        L.update(cuda(xy2))
        gr.gr_diff_forward(L.handle, IDEAL, None)
        terms2, h_eca, h_ml, h_ma = oracle.diff_terms_and_grads(xy2, e, IDEAL)
        gd.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        grad_close(gd.cpu().numpy(), -h_eca + h_ml - h_ma, "graph replay after a forward with millions of crossings")
        with pytest.raises(gr.GrError) as ei:
            with torch.cuda.graph(torch.cuda.CUDAGraph(), stream=s, capture_error_mode="relaxed"):
                gr.gr_diff_forward(L.handle, IDEAL, out, torch.cuda.current_stream().cuda_stream)
        assert ei.value.status == gr.GR_ENOTSUP
