"""CPU: the integer and filtered floating-point arithmetic of the kernels
restated in Python with the constants read from their sources, checked
against plain definitions: the Barrett-reduced visiting order of the DDA
passes (a bijection equal to i * (2^31 - 1) mod n), the cells each thread of
the offsets cluster reads and writes (every cell of [0, C) exactly once,
16-byte accesses aligned), the integer scaling of a line direction to units
of pi / 2^32 (the FP64 product rounded to the nearest integer), the minimum
angle's table-driven FP64 gap against atan2 (with NumPy's FP32 atan2 standing
in for the device's), the rotation work items (every pair of a cell once),
the FP32 and FP16 clip tests of the pair kernel and the FP32 orientation
filter of the differentiable kernels against exact rational arithmetic."""
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


def rotation_constants():
    src = source("grid_common.cuh")
    get = lambda name: int(re.search(r"constexpr int %s = (\d+);" % name, src).group(1))
    return get("RQ"), get("RSTREAMS"), get("RWIN")


def rot_streams(m, P, RS):
    # grid_common.cuh rot_streams
    return 1 if m >= 32 else min(RS, max(1, 32 // m), max(1, P))


def rot_items(n, RQ, RS):
    # grid_common.cuh rot_item_count / rot_item_words
    if n < 2:
        return []
    Q, Ff, m = n >> 1, n >> 5, n & 31
    P = (Q + RQ - 1) // RQ
    words = [(c << 16) | p for c in range(Ff) for p in range(P)]
    if m:
        s = rot_streams(m, min(P, RS), RS)
        words += [(Ff << 16) | p for p in range((P + s - 1) // s)]
    return words


def rot_lane(n, w, lane, RQ, RS):
    # grid_common.cuh rot_lane: (row, first offset, offsets taken, window slot, m, s, first window row)
    Q, c, p = n >> 1, (w >> 16) & 0x7FFF, w & 0xFFFF
    P = (Q + RQ - 1) // RQ
    m = min(32, n - 32 * c)
    s = rot_streams(m, min(P, RS), RS)
    sig, row = lane // m, lane % m
    pbase = p if m == 32 else p * s
    piece = pbase + sig
    i, q0 = 32 * c + row, 1 + piece * RQ
    first = 32 * c + 1 + pbase * RQ
    slot = sig * (m + RQ - 1) + row
    Qi = Q - 1 if (n % 2 == 0 and i >= n // 2) else Q
    cnt = max(0, min(Qi, q0 + RQ - 1) - q0 + 1) if (sig < s and piece < P) else 0
    if cnt == 0:
        i, slot = 0, 0
    return i, q0, cnt, slot, m, s, first


@pytest.mark.parametrize("n", list(range(0, 70)) + [95, 96, 97, 127, 128, 129, 255, 256, 299, 300, 513, 1000])
def test_rotation_items_cover_every_pair_of_a_cell_once(n):
    # every unordered pair {i, j} of the cell's n records is met exactly once by
    # the lanes of its rotation work items, each lane within the cell's rows, and
    # the window slot a lane reads at each offset (staged as the kernel stages
    # it, within RWIN slots) holds that pair's column
    RQ, RS, RWIN = rotation_constants()
    seen = {}
    for w in rot_items(n, RQ, RS):
        lanes = [rot_lane(n, w, lane, RQ, RS) for lane in range(32)]
        _, _, _, _, m, s, first = lanes[0]
        span = m + RQ - 1
        assert s * span <= RWIN
        window = [(first + (u // span) * RQ + (u % span)) % n for u in range(s * span)]
        for i, q0, cnt, slot, *_ in lanes:
            assert cnt <= RQ
            for t in range(cnt):
                j = (i + q0 + t) % n
                assert window[slot + t] == j
                key = (min(i, j), max(i, j))
                seen[key] = seen.get(key, 0) + 1
    assert len(seen) == n * (n - 1) // 2
    assert all(v == 1 for v in seen.values())


def test_rotation_items_use_most_lanes():
    # lane slots of a cell's items (32 lanes x RQ offsets) against its pairs:
    # the streams of a short last chunk keep most lanes busy
    RQ, RS, _ = rotation_constants()
    sizes = range(33, 400)
    pairs = sum(n * (n - 1) // 2 for n in sizes)
    slots = sum(32 * RQ * len(rot_items(n, RQ, RS)) for n in sizes)
    assert pairs >= 0.8 * slots


def f32(x):
    return float(np.float32(x))


def fmaf(a, b, c):
    # one rounding of the exact a * b + c to FP32
    from fractions import Fraction
    return f32(Fraction(a) * Fraction(b) + Fraction(c)) if not any(map(math.isnan, (a, b, c))) else math.nan


def div_fast(a, b, rng=None):
    # the device's fast division: within 2 ulp of the quotient (modelled as the
    # correctly rounded quotient moved by up to 2 ulp either way)
    from fractions import Fraction
    q = f32(Fraction(a) / Fraction(b))
    if rng is not None and q != 0.0:
        q = float(np.float32(q) + np.float32(rng.integers(-2, 3)) * np.spacing(np.float32(abs(q))))
    return q


def make_clip(ax, ay, bx, by, w, rng=None):
    # grid_common.cuh make_rgeo: the clip points and {ux, uy, nk, v}
    ux, uy = bx - ax, by - ay
    m = max(abs(ax), abs(ay), abs(bx), abs(by))
    exact = abs(ux) <= 1024 and abs(uy) <= 1024 and m <= 4096
    whole = min(ax, ay, bx, by) >= 0 and max(ax, ay, bx, by) <= w
    line = (float(ux), float(uy), -f32(ux * ay - uy * ax), (0.0 if whole else 64.0) if exact else 8192.0)
    if (uy == 0 and ay in (0, w)) or (ux == 0 and ax in (0, w)):
        return (math.nan,) * 4, line
    if whole:
        return (float(ax), float(ay), float(bx), float(by)), line
    t0, t1 = 0.0, 1.0
    if ux:
        ta, tb = div_fast(-ax, ux, rng), div_fast(w - ax, ux, rng)
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    if uy:
        ta, tb = div_fast(-ay, uy, rng), div_fast(w - ay, uy, rng)
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    if t1 < t0:
        t1 = t0
    return (fmaf(t0, ux, ax), fmaf(t0, uy, ay), fmaf(t1, ux, ax), fmaf(t1, uy, ay)), line


def fmin(a, b):
    # IEEE minNum (fminf): a NaN operand yields the other
    return b if math.isnan(a) else (a if math.isnan(b) else min(a, b))


def fmax(a, b):
    return b if math.isnan(a) else (a if math.isnan(b) else max(a, b))


def clip_test(rb, rc, cb, cc):
    # grid_common.cuh clip_test: (out, in)
    def s(line, p):
        return fmaf(line[0], p[1], fmaf(-line[1], p[0], line[2]))
    s0, s1 = s(cb, rc[:2]), s(cb, rc[2:])
    s2, s3 = s(rb, cc[:2]), s(rb, cc[2:])
    M01 = fmax(cb[3], min(rb[3], 64.0))
    M23 = fmax(rb[3], min(cb[3], 64.0))
    lo01, hi01, lo23, hi23 = fmin(s0, s1), fmax(s0, s1), fmin(s2, s3), fmax(s2, s3)
    out = lo01 > M01 or hi01 < -M01 or lo23 > M23 or hi23 < -M23
    inside = lo01 < -M01 and hi01 > M01
    return out, inside


def exact_owner(r, c, w):
    # the half-open cell [0, w)^2 holds the intersection point of the two lines
    from fractions import Fraction
    ax, ay, bx, by = r
    cx, cy, dx, dy = c
    ux, uy, vx, vy = bx - ax, by - ay, dx - cx, dy - cy
    den = ux * vy - uy * vx
    t = Fraction((cx - ax) * vy - (cy - ay) * vx, den)
    X, Y = ax + ux * t, ay + uy * t
    return int(0 <= X < w and 0 <= Y < w)


def crossing(r, c):
    from fractions import Fraction
    def o(p, q, s):
        return (q[0] - p[0]) * (s[1] - p[1]) - (q[1] - p[1]) * (s[0] - p[0])
    a, b, p, q = r[:2], r[2:], c[:2], c[2:]
    o1, o2, o3, o4 = o(a, b, p), o(a, b, q), o(p, q, a), o(p, q, b)
    return o1 * o2 <= 0 and o3 * o4 <= 0 and not (o1 == 0 and o2 == 0)


def meets_cell(r, w):
    # the closed segment meets the closed cell [0, w]^2 (exact, Liang-Barsky)
    from fractions import Fraction
    lo, hi = Fraction(0), Fraction(1)
    for a0, u in ((r[0], r[2] - r[0]), (r[1], r[3] - r[1])):
        if u == 0:
            if not 0 <= a0 <= w:
                return False
        else:
            ta, tb = Fraction(-a0, u), Fraction(w - a0, u)
            lo, hi = max(lo, min(ta, tb)), min(hi, max(ta, tb))
    return lo <= hi


def test_clip_test_never_drops_a_pair_this_cell_owns():
    # pairs of crossing segments in the coordinates of one cell, among them long
    # ones reaching far outside it, intersections near the cell's corners and
    # borders, and segments along its border lines: the FP32 clip test (both
    # clipped parts against the other's line) never rejects a pair whose exact
    # intersection point lies in the half-open cell, and whenever it places the
    # point inside, the exact owner is this cell
    rng = np.random.default_rng(123)
    owned = rejected = inside = 0
    for trial in range(8000):
        k = int(rng.choice([6, 8, 10, 12]))
        w = 1 << k
        x0 = int(rng.integers(1, 65536 // w - 1)) * w
        y0 = int(rng.integers(1, 65536 // w - 1)) * w
        P = rng.uniform(-0.25 * w, 1.25 * w, size=2)
        if rng.random() < 0.3:
            P = np.array([float(rng.choice([0, w])), float(rng.choice([0, w]))])
        elif rng.random() < 0.3:
            P[int(rng.integers(0, 2))] = float(rng.choice([0, w]))

        def seg():
            th = rng.uniform(0, math.pi)
            if rng.random() < 0.15:
                th = float(rng.choice([0.0, math.pi / 2]))  # axis-parallel, possibly along a cell line
            d = np.array([math.cos(th), math.sin(th)])
            la, lb = (rng.uniform(0, 40000, size=2) if rng.random() < 0.4 else rng.uniform(0, 1.5 * w, size=2))
            p = np.rint(np.concatenate([P - la * d, P + lb * d]) + [x0, y0, x0, y0])
            p = np.clip(p, 0, 65535).astype(np.int64)
            return tuple(int(v) for v in (p[0] - x0, p[1] - y0, p[2] - x0, p[3] - y0))
        r, c = seg(), seg()
        if (r[0], r[1]) == (r[2], r[3]) or (c[0], c[1]) == (c[2], c[3]) or not crossing(r, c):
            continue
        ux, uy, vx, vy = r[2] - r[0], r[3] - r[1], c[2] - c[0], c[3] - c[1]
        if ux * vy - uy * vx == 0:
            continue
        if not (meets_cell(r, w) and meets_cell(c, w)):  # the grid only emits such records
            continue
        rc, rb = make_clip(*r, w, rng)
        cc, cb = make_clip(*c, w, rng)
        out, ins = clip_test(rb, rc, cb, cc)
        own = exact_owner(r, c, w)
        owned += own
        if own:
            assert not out, (trial, r, c, w)
        else:
            rejected += out
        if ins:
            inside += 1
            assert own, (trial, r, c, w)
    assert owned > 500 and rejected > 500 and inside > 300


def half_margin(w):
    src = source("grid_common.cuh")
    a, b = re.search(r"half_margin\(int w\) \{ return ([0-9.]+)f \+ ([0-9.]+)f / \(float\)w; \}", src).groups()
    m = float(np.float32(np.float32(a) + np.float32(b) / np.float32(w)))
    h = np.float16(m)
    if float(h) < m:  # rounded up to FP16, as the kernel takes it
        h = np.nextafter(h, np.float16(np.inf))
    return float(h)


def make_half(line, clip, w):
    # grid_common.cuh make_hgeo, in FP32 then rounded to FP16, centred on the
    # cell (NaN records: None)
    f = np.float32
    ux, uy, nk = f(line[0]), f(line[1]), f(line[2])
    inv_w = f(1.0) / f(w)
    ln = np.sqrt(ux * ux + uy * uy)
    with np.errstate(divide="ignore", invalid="ignore"):
        hx, hy = ux / ln, -uy / ln
        hc = nk * inv_w / ln + f(0.5) * (hx + hy)
    if not ln > 0 or not abs(hc) <= 0.75 or any(map(math.isnan, clip)):
        return None
    h = lambda v: float(np.float16(v))
    return (h(hx), h(hy), h(hc)), tuple(h(f(v) * inv_w - f(0.5)) for v in clip)


def hfma(a, b, c):
    # one rounding of a * b + c to FP16 (exact in FP64 for FP16 operands)
    return float(np.float16(a * b + c))


def half_test(r, c, M):
    # k_cell_pairs' FP16 test of one pair: (dropped, counted); None records: undecided
    if r is None or c is None:
        return False, False
    def s(line, p):
        return hfma(line[0], p[1], hfma(line[1], p[0], line[2]))
    (rl, rp), (cl, cp) = r, c
    s0, s1, s2, s3 = s(cl, rp[:2]), s(cl, rp[2:]), s(rl, cp[:2]), s(rl, cp[2:])
    t01 = fmax(fmin(s0, s1), -fmax(s0, s1))
    t23 = fmax(fmin(s2, s3), -fmax(s2, s3))
    tt = max(t01, t23)
    return tt > M, tt < -M


def proper(r, c):
    def o(p, q, s):
        return (q[0] - p[0]) * (s[1] - p[1]) - (q[1] - p[1]) * (s[0] - p[0])
    a, b, p, q = r[:2], r[2:], c[:2], c[2:]
    return o(a, b, p) * o(a, b, q) < 0 and o(p, q, a) * o(p, q, b) < 0


def test_half_test_is_sound():
    # pairs of segments meeting one cell: crossing, touching, sharing an
    # endpoint, nearly touching, collinear, long ones reaching far outside
    # the cell, points on its corners and border lines.  The FP16 first test
    # of the pair kernel never drops a pair that counts in this cell (a
    # crossing or touching whose exact intersection point lies in the
    # half-open cell, or a collinear overlap), and every pair it counts at
    # once is a proper crossing whose point lies in the cell.
    rng = np.random.default_rng(321)
    dropped = counted = kept_owned = 0
    for trial in range(9000):
        k = int(rng.choice([3, 5, 8, 10, 12]))
        w = 1 << k
        M = half_margin(w)
        x0 = int(rng.integers(1, 65536 // w - 1)) * w
        y0 = int(rng.integers(1, 65536 // w - 1)) * w
        P = rng.uniform(-0.25 * w, 1.25 * w, size=2)
        u = rng.random()
        if u < 0.25:
            P = np.array([float(rng.choice([0, w])), float(rng.choice([0, w]))])
        elif u < 0.5:
            P[int(rng.integers(0, 2))] = float(rng.choice([0, w]))

        def seg(off):
            th = rng.uniform(0, math.pi)
            if rng.random() < 0.15:
                th = float(rng.choice([0.0, math.pi / 2]))
            d = np.array([math.cos(th), math.sin(th)])
            nrm = np.array([-d[1], d[0]])
            la, lb = (rng.uniform(0, 40000, size=2) if rng.random() < 0.3 else rng.uniform(0, 1.5 * w, size=2))
            if rng.random() < 0.25:
                la = 0.0  # the segment ends at P
            Q = P + off * nrm
            p = np.rint(np.concatenate([Q - la * d, Q + lb * d]) + [x0, y0, x0, y0])
            p = np.clip(p, 0, 65535).astype(np.int64)
            return tuple(int(v) for v in (p[0] - x0, p[1] - y0, p[2] - x0, p[3] - y0))
        off = 0.0 if rng.random() < 0.5 else float(rng.choice([-1, 1])) * rng.uniform(0, 4) * w / 256
        r, c = seg(0.0), seg(off)
        if rng.random() < 0.1:
            c = (r[0], r[1], c[2], c[3])  # an endpoint shared
        if rng.random() < 0.05:
            t = int(rng.integers(-3, 4))  # collinear, overlapping or not
            c = (r[0] + t * (r[2] - r[0]) // 4, r[1] + t * (r[3] - r[1]) // 4, r[2], r[3])
        if (r[0], r[1]) == (r[2], r[3]) or (c[0], c[1]) == (c[2], c[3]):
            continue
        if not (meets_cell(r, w) and meets_cell(c, w)):
            continue
        rc, rb = make_clip(*r, w, rng)
        cc, cb = make_clip(*c, w, rng)
        out, sure = half_test(make_half(rb, rc, w), make_half(cb, cc, w), M)
        ux, uy, vx, vy = r[2] - r[0], r[3] - r[1], c[2] - c[0], c[3] - c[1]
        par = ux * vy - uy * vx == 0
        counts = crossing(r, c) and (par or exact_owner(r, c, w))
        if out:
            dropped += 1
            assert not counts, (trial, r, c, w)
        if sure:
            counted += 1
            assert proper(r, c) and exact_owner(r, c, w), (trial, r, c, w)
        kept_owned += counts and not sure
    assert dropped > 1000 and counted > 500 and kept_owned > 100


def orient_filter(ux, uy, px, py, rx, ry):
    # k_diff.cu orient_f32_filter in FP32 (products and differences rounded
    # one by one; the device may fuse the last subtraction, which only makes
    # d more accurate): +-1 when decided, 0 otherwise
    f = np.float32
    t1 = f(ux) * (f(ry) - f(py))
    t2 = f(uy) * (f(rx) - f(px))
    d = t1 - t2
    mag = abs(t1) + abs(t2)
    e32 = f(5.9604645e-08)
    b32 = (f(3.0) + f(16.0) * e32) * e32 * mag
    if not mag >= f(2.0 ** -100):
        return 0
    return 1 if d > b32 else (-1 if -d > b32 else 0)


def test_fp32_orientation_filter_decides_only_exact_signs():
    # FP32 points near and on common lines (collinear up to a few ulp, wide
    # exponent ranges, shared coordinates): whenever the branch-free FP32 filter
    # of the differentiable pair kernels decides a sign, it is the sign of the
    # exact orientation of the FP32 inputs
    from fractions import Fraction
    rng = np.random.default_rng(77)
    decided = undecided = 0
    for trial in range(20000):
        scale = float(2.0 ** rng.integers(-20, 20))
        p = rng.uniform(-1, 1, 2) * scale
        q = rng.uniform(-1, 1, 2) * scale
        t = rng.uniform(-2, 3)
        r = p + t * (q - p)
        if rng.random() < 0.7:  # nudge off the line by a few ulp
            r = r + rng.integers(-4, 5, 2) * np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
        else:
            r = r + rng.normal(0, 1e-3 * scale, 2)
        p, q, r = (np.asarray(v, np.float32) for v in (p, q, r))
        ux, uy = np.float32(q[0] - p[0]), np.float32(q[1] - p[1])
        s = orient_filter(ux, uy, p[0], p[1], r[0], r[1])
        F = lambda v: Fraction(float(v))
        exact = (F(q[0]) - F(p[0])) * (F(r[1]) - F(p[1])) - (F(q[1]) - F(p[1])) * (F(r[0]) - F(p[0]))
        if s == 0:
            undecided += 1
            continue
        decided += 1
        assert (exact > 0 and s == 1) or (exact < 0 and s == -1), (trial, p, q, r, s, exact)
    assert decided > 5000 and undecided > 1000
