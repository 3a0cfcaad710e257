"""GPU: one layout's evaluation in parts (gr_evaluate_part), the parts summed
and combined (gr_combine_parts) on one GPU, against gr_evaluate of the whole
layout -- bit for bit, on every path the parts split (the rotation kernel's
work items, the tile kernel's items with long pairs on all-pairs tiles, the
all-pairs tiles, both occlusion paths) -- and the layout's later full
evaluations and moves unaffected."""
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


def cuda(a):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def combined(L, n_parts, d, others=()):
    """Parts 0 .. n_parts-1, part p evaluated on layout ([L] + others)[p % ...]:
    separate layouts of the same inputs stand in for the ranks (each gathers
    its segments and fills its grid in its own order)."""
    lays = [L] + list(others)
    parts = [gr.gr_evaluate_part(lays[p % len(lays)].handle, p, n_parts, gr.GR_METRIC_ALL, IDEAL, d)
             for p in range(n_parts)]
    total = gr.partial_from_list([sum(v) for v in zip(*(gr.partial_to_list(p) for p in parts))])
    return gr.gr_combine_parts(total, IDEAL, d), parts


CASES = {
    "plain": (lambda: synth.plain_layout(), gr.gr_options(0, 0, 0, 0), 256),
    "long_pairs_on_tiles": (lambda: synth.plain_layout(V=3000, knn_count=6000, random_count=3000, seed=9),
                            gr.gr_options(gr.GR_PATH_GRID, 0, 0, 0, gr.GR_LONG_ALLPAIRS), 300),
    "all_pairs": (lambda: synth.dense_long_edge_layout(V=3000, E=20_000), gr.gr_options(gr.GR_PATH_ALLPAIRS, 0, 0, 0),
                  2000),
    "occlusion_grid": (lambda: synth.plain_layout(V=9000, knn_count=18000, random_count=2000, seed=4),
                       gr.gr_options(0, 0, gr.GR_PATH_GRID, 0), 700),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_parts_combine_to_the_whole_evaluation(case):
    make, opt, d = CASES[case]
    L0 = make()
    with gr.Layout(cuda(L0.xy), cuda(L0.edges), opt) as L, gr.Layout(cuda(L0.xy), cuda(L0.edges), opt) as L2, \
            gr.Layout(L0.xy, L0.edges, opt) as L3:
        whole = L.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
        for n_parts in (1, 2, 3, 7):
            r, parts = combined(L, n_parts, d, (L2, L3))
            assert bytes(memoryview(r)) == bytes(memoryview(whole)), (case, n_parts)
            if n_parts > 1 and whole.crossing.c.crossings > 100:
                assert all(p.proper + p.touching < whole.crossing.c.crossings for p in parts)  # really split
        # a whole evaluation after the parts, and a move, see all of the work again
        assert bytes(memoryview(L.evaluate(gr.GR_METRIC_ALL, IDEAL, d))) == bytes(memoryview(whole))
        ids = np.array([1, 2], np.int32)
        new = np.array([[100, 100], [60000, 31000]], np.int32)
        rm = L.move(ids, new, gr.GR_METRIC_ALL, IDEAL, d)
        xy = L0.xy.copy()
        xy[ids] = new
        ref = oracle.crossings(xy, L0.edges, IDEAL)
        assert (rm.crossing.c.proper, rm.crossing.c.touching) == (ref.proper, ref.touching)


def test_large_sparse_layout_in_parts():
    L0 = synth.large_sparse_layout()
    with gr.Layout(cuda(L0.xy), cuda(L0.edges)) as L, gr.Layout(cuda(L0.xy), cuda(L0.edges)) as L2:
        whole = L.evaluate(gr.GR_METRIC_ALL, IDEAL, 64)
        assert whole.crossing_path == 1
        for n_parts in (2, 5):
            r, _ = combined(L, n_parts, 64, (L2,))
            assert bytes(memoryview(r)) == bytes(memoryview(whole)), n_parts


def test_part_errors():
    L0 = synth.plain_layout(V=300, knn_count=600, random_count=100, seed=2)
    with gr.Layout(cuda(L0.xy), cuda(L0.edges)) as L:
        for part, n in ((0, 0), (2, 2), (-1, 3)):
            with pytest.raises(gr.GrError) as ei:
                gr.gr_evaluate_part(L.handle, part, n)
            assert ei.value.status == gr.GR_EINVAL
    xy = np.random.default_rng(0).random((50, 2)).astype(np.float32)
    with gr.Layout(cuda(xy), cuda(np.array([[0, 1], [2, 3]], np.int32)), coord_type=gr.GR_COORD_F32) as L:
        with pytest.raises(gr.GrError) as ei:
            gr.gr_evaluate_part(L.handle, 0, 2)
        assert ei.value.status == gr.GR_ENOTSUP
