"""CPU: one layout's evaluation split into parts over two gloo ranks (no GPU).

Each rank takes the part of the all-pairs tiles that the library's kernels
would take (the part range and the tile order restated from the CUDA
sources), tallies that part's pairs with the oracle, and the ranks combine
their integer tallies with one all-reduce (paper_2411_09809_gb300.shard) and
libgr's host-side gr_combine_parts.  The combined counts must equal the
oracle's on the whole layout exactly; the angle sum, quantised to the
library's units per part, within that quantisation."""
import math
import os
import re
import socket
import struct
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
CSRC = os.path.join(ROOT, "paper_2411_09809_gb300", "csrc")
IDEAL = 7 * math.pi / 18
UNIT = math.pi / 2.0 ** 32


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def small_tile_rows():
    src = open(os.path.join(CSRC, "allpairs_common.cuh")).read()
    t = int(re.search(r"constexpr int AS_THREADS = (\d+);", src).group(1))
    r = int(re.search(r"constexpr int AS_RPT = (\d+);", src).group(1))
    return t * r


def part_range(units, p, n):
    # gr_internal.cuh part_range
    return units * p // n, units * (p + 1) // n


def decode_tile(t):
    # allpairs_common.cuh decode_tile: lower-triangular order, bi <= bj
    r = int((math.sqrt(8.0 * t + 1.0) - 1.0) * 0.5)
    while r * (r + 1) // 2 > t:
        r -= 1
    while (r + 1) * (r + 2) // 2 <= t:
        r += 1
    return t - r * (r + 1) // 2, r


def layout():
    from paper_2411_09809_gb300 import synth
    L = synth.plain_layout(V=420, knn_count=840, random_count=360, seed=3)
    a, b = L.xy[L.edges[:, 0]], L.xy[L.edges[:, 1]]
    assert np.all(np.any(a != b, axis=1))  # no zero-length edges: segments are the edge list
    return L


def part_tallies(L, part, n_parts):
    """(proper, touching, collinear, angle sum in radians) of the pairs in this
    part's tiles, each tile's pairs tallied by the oracle."""
    import oracle
    rows = small_tile_rows()
    E = L.E
    nb = (E + rows - 1) // rows
    lo, hi = part_range(nb * (nb + 1) // 2, part, n_parts)
    blocks = [L.edges[i * rows:(i + 1) * rows] for i in range(nb)]

    def tally(edges):
        r = oracle.crossings(L.xy, edges, IDEAL)
        return np.array([r.proper, r.touching, r.collinear]), r.angle_dev_sum

    c, dev = np.zeros(3, np.int64), 0.0
    for t in range(lo, hi):
        bi, bj = decode_tile(t)
        if bi == bj:
            k, d = tally(blocks[bi])
        else:
            k, d = tally(np.concatenate([blocks[bi], blocks[bj]]))
            for blk in (blocks[bi], blocks[bj]):
                k2, d2 = tally(blk)
                k, d = k - k2, d - d2
        c += k
        dev += d
    return c, dev


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def make_partial(L, part, n_parts):
    import oracle
    from paper_2411_09809_gb300 import gr
    c, dev = part_tallies(L, part, n_parts)
    units = int(round(dev / UNIT))
    p = gr.gr_partial()
    p.proper, p.touching, p.collinear_overlaps = (int(v) for v in c)
    p.occlusion_pairs = 0
    p.dev_hi32, p.dev_lo32 = units >> 32, units & 0xFFFFFFFF
    if part == 0:
        ma = oracle.min_angle(L.xy, L.edges)
        p.metrics, p.crossing_path, p.cell_log2, p.occlusion_path = gr.GR_METRIC_CROSSINGS | 12, 2, 0, 0
        p.zero_length_edges, p.pairs_tested = 0, L.E * (L.E - 1) // 2
        p.n_vertices_counted = ma.n_vertices
        p.min_angle_sum_d_bits, p.M_a_bits = _bits(ma.sum_d), _bits(ma.M_a)
        p.M_l_bits = _bits(oracle.edge_length_variation(L.xy, L.edges))
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build, gr, shard
    build.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = layout()
        mine = make_partial(L, rank, world)
        total = shard.reduce_partials(mine)
        r = gr.gr_combine_parts(total, IDEAL, 0)
        q.put((rank, gr.partial_to_list(mine), gr.partial_to_list(total), bytes(memoryview(r))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_whole_layout():
    import torch.multiprocessing as mp

    import oracle
    from paper_2411_09809_gb300 import build, gr
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {r: (mine, total, res) for r, mine, total, res in (q.get(timeout=300) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the all-reduce is the field-wise sum, and both ranks hold the same result
    want = [a + b for a, b in zip(got[0][0], got[1][0])]
    assert got[0][1] == got[1][1] == want
    assert got[0][2] == got[1][2]
    r = gr.gr_result.from_buffer_copy(got[0][2])
    L = layout()
    ref = oracle.crossings(L.xy, L.edges, IDEAL)
    c = r.crossing.c
    assert (c.proper, c.touching, c.collinear_overlaps, c.crossings) == \
        (ref.proper, ref.touching, ref.collinear, ref.crossings)
    assert c.pairs_tested == L.E * (L.E - 1) // 2
    # the two parts' angle sums each rounded to the library's unit
    assert abs(r.crossing.angle_dev_sum - ref.angle_dev_sum) <= 2 * UNIT
    assert r.crossing.E_ca == pytest.approx(ref.E_ca, rel=1e-12)
    ma = oracle.min_angle(L.xy, L.edges)
    assert (r.min_angle.M_a, r.min_angle.sum_d, r.min_angle.n_vertices_counted) == (ma.M_a, ma.sum_d, ma.n_vertices)
    assert r.M_l == oracle.edge_length_variation(L.xy, L.edges)


def test_part_ranges_cover_every_unit_once():
    for units in (0, 1, 2, 7, 15, 1000, 2 ** 40 + 3):
        for n in (1, 2, 3, 5, 8):
            spans = [part_range(units, p, n) for p in range(n)]
            assert spans[0][0] == 0 and spans[-1][1] == units
            assert all(spans[i][1] == spans[i + 1][0] for i in range(n - 1))


def test_combine_carries_the_angle_sum_across_halves():
    # low halves that overflow 32 bits when summed: the 128-bit total is rebuilt
    from paper_2411_09809_gb300 import build, gr
    build.build()
    parts = [gr.gr_partial(), gr.gr_partial(), gr.gr_partial()]
    units = [0xFFFFFFFF + (7 << 32), 0xFFFFFFFE + (2 ** 40 << 32), 5]
    for p, u in zip(parts, units):
        p.proper = 3
        p.dev_hi32, p.dev_lo32 = u >> 32, u & 0xFFFFFFFF
    tot = gr.partial_from_list([sum(v) for v in zip(*(gr.partial_to_list(p) for p in parts))])
    r = gr.gr_combine_parts(tot, IDEAL, 0)
    assert r.crossing.c.crossings == 9
    assert r.crossing.angle_dev_sum == float(sum(units)) * UNIT
