"""CPU: the integer arithmetic of three kernels restated in Python with the
constants read from their sources, checked against plain definitions: the
Barrett-reduced visiting order of the DDA passes (a bijection equal to
i * (2^31 - 1) mod n), the cells each thread of the offsets cluster reads and
writes (every cell of [0, C) exactly once, 16-byte accesses aligned), and the
integer scaling of a line direction to units of pi / 2^32 (the FP64 product
rounded to the nearest integer)."""
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
