"""CPU: the integer arithmetic of three kernels restated in Python with the
constants read from their sources, checked against plain definitions: the
Barrett-reduced visiting order of the DDA passes (a bijection equal to
i * (2^31 - 1) mod n), the cells each thread of the offsets cluster reads and
writes (every cell of [0, C) exactly once, 16-byte accesses aligned), and the
integer scaling of a line direction to units of pi / 2^32 (the FP64 product
rounded to the nearest integer); and the minimum angle's table-driven FP64
gap against atan2 (with NumPy's FP32 atan2 standing in for the device's)."""
import math
import os
import re
from decimal import Decimal, getcontext

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2411_09809_gb300", "csrc")


def source(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def spread(i, n):
    # k_grid.cu spread_setup / spread_index
    if n >= 0x7FFFFFFF:
        return i
    m = 0x7FFFFFFF % n
    inv = ((1 << 64) - 1) // n
    p = i * m
    r = p - ((p * inv) >> 64) * n
    assert 0 <= r < 2 * n
    return r - n if r >= n else r


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000, 4093, 65536])
def test_spread_is_the_modular_bijection(n):
    got = [spread(i, n) for i in range(n)]
    assert got == [(i * (0x7FFFFFFF % n)) % n for i in range(n)]
    assert sorted(got) == list(range(n))


def test_spread_on_large_n():
    rng = np.random.default_rng(5)
    for n in list(rng.integers(1, 0x7FFFFFFE, size=200)) + [0x7FFFFFFE]:
        n = int(n)
        for i in [0, n - 1] + [int(x) for x in rng.integers(0, n, size=50)]:
            assert spread(i, n) == (i * (0x7FFFFFFF % n)) % n


def offsets_constants():
    s = source("k_grid.cu")
    m = re.search(r"kOffsetsThreads = (\d+), kOffsetsPer = (\d+), kOffsetsCluster = (\d+);", s)
    return tuple(int(x) for x in m.groups())


@pytest.mark.parametrize("log2_side", [0, 1, 2, 4, 6, 7, 8])
def test_offsets_cluster_touches_every_cell_once(log2_side):
    T, P, K = offsets_constants()
    C = (1 << log2_side) ** 2  # G = 65536 >> k cells a side
    if C > K * T * P:
        pytest.skip("larger grids take the three-kernel scans")
    seen = np.zeros(C, np.int64)
    for r in range(K):
        for t in range(T):
            c0 = r * T * P + t * P
            full = c0 + P <= C
            if full:
                assert c0 % 4 == 0  # 16-byte aligned uint4 accesses
            for j in range(P):
                c = c0 + j
                if full or c < C:
                    assert 0 <= c < C
                    seen[c] += 1
    assert (seen == 1).all()


def test_line_direction_scaling_equals_the_fp64_product():
    s = source("pair_math.cuh")
    K = int(re.search(r"constexpr uint64_t K = (\d+)ull;", s).group(1))
    getcontext().prec = 60
    pi = Decimal("3.14159265358979323846264338327950288419716939937510582097494")
    assert K == int((Decimal(2) ** 62 / pi).to_integral_value())  # round(2^62 / pi), exactly
    rng = np.random.default_rng(6)
    dx = rng.integers(-65535, 65536, size=200000)
    dy = rng.integers(1, 65536, size=200000)
    t = np.arctan2(dy.astype(np.float32), dx.astype(np.float32)).astype(np.float32)
    bits = t.view(np.uint32).astype(np.int64)
    want = np.rint(t.astype(np.float64) * (4294967296.0 / math.pi)).astype(np.int64)
    for b, w in zip(bits[:20000], want[:20000]):
        be = int(b) >> 23
        m = (int(b) & 0x7FFFFF) | 0x800000
        sh = 180 - be
        got = (m * K + (1 << (sh - 1))) >> sh if be >= 90 else 0
        assert got == int(w)


def sector_gap(a, b, tab, w):
    # k_minangle.cu ccw_gap_d, FP64 steps in the same order
    cr = a[0] * b[1] - a[1] * b[0]
    dt = a[0] * b[0] + a[1] * b[1]
    g = np.arctan2(np.float32(cr), np.float32(dt))
    j = int(np.rint(np.float32(g) * np.float32(len(tab) / (2 * math.pi)))) & (len(tab) - 1)
    c, s_ = tab[j]
    X, Y = float(dt), float(cr)
    x = X * c + Y * s_
    y = Y * c - X * s_
    t = y / x
    t2 = t * t
    p = (((t2 / 9.0 - 1.0 / 7.0) * t2 + 1.0 / 5.0) * t2 - 1.0 / 3.0) * t2 + 1.0
    th = t * p + j * w
    if th < 0.0:
        th += 2 * math.pi
    if th >= 2 * math.pi:
        th -= 2 * math.pi
    return th


def test_min_angle_sector_gap_matches_atan2():
    s = source("k_minangle.cu")
    n = int(re.search(r"constexpr int kSectors = (\d+);", s).group(1))
    w = 2.0 * math.pi / n
    tab = [(math.cos(j * w), math.sin(j * w)) for j in range(n)]
    rng = np.random.default_rng(7)
    vecs = [tuple(int(v) for v in rng.integers(-65535, 65536, size=2)) for _ in range(4000)]
    vecs += [(1, 0), (-1, 0), (0, 1), (0, -1), (65535, 1), (-65535, 1), (3, 4), (-4, 3)]
    worst = 0.0
    for i in range(len(vecs) - 1):
        a, b = vecs[i], vecs[i + 1]
        if a == (0, 0) or b == (0, 0):
            continue
        ref = math.atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1])
        ref = ref + 2 * math.pi if ref < 0 else ref
        d = abs(sector_gap(a, b, tab, w) - ref)
        worst = max(worst, min(d, 2 * math.pi - d))
    assert worst < 2e-15
