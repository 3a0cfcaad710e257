"""Independent rational-arithmetic brute force for small layouts (tests only).

It decides every edge pair by solving the two parametric line equations
a + t u = c + s v exactly with `fractions.Fraction` (Cramer's rule), instead of
the orientation-sign products the oracle uses, and it measures the crossing
angle from the two lines' angles with the x-axis (Sec. 3.2.3 defines theta_i in
[0, pi) that way), instead of from the cross and dot products.  It follows the
same readings of the paper as the oracle: shared-id pairs and zero-length edges
never cross, collinear pairs that meet are counted apart from E_c.
"""
from fractions import Fraction
import math


def classify(p, e, f):
    """Returns (kind, angle) with kind in {None, 'proper', 'touching', 'collinear'}."""
    a_id, b_id = e
    c_id, d_id = f
    if len({a_id, b_id} & {c_id, d_id}) > 0:
        return None, 0.0
    a, b, c, d = p[a_id], p[b_id], p[c_id], p[d_id]
    if a == b or c == d:
        return None, 0.0
    ux, uy = b[0] - a[0], b[1] - a[1]
    vx, vy = d[0] - c[0], d[1] - c[1]
    wx, wy = c[0] - a[0], c[1] - a[1]
    den = ux * vy - uy * vx
    if den == 0:
        if wx * uy - wy * ux != 0:
            return None, 0.0  # parallel, distinct lines
        uu = ux * ux + uy * uy
        t0 = Fraction(wx * ux + wy * uy, uu)
        t1 = Fraction((d[0] - a[0]) * ux + (d[1] - a[1]) * uy, uu)
        lo, hi = min(t0, t1), max(t0, t1)
        if hi < 0 or lo > 1:
            return None, 0.0
        return "collinear", 0.0
    t = Fraction(wx * vy - wy * vx, den)
    s = Fraction(wx * uy - wy * ux, den)
    if t < 0 or t > 1 or s < 0 or s > 1:
        return None, 0.0
    kind = "proper" if (0 < t < 1 and 0 < s < 1) else "touching"
    th_e = math.atan2(uy, ux) % math.pi
    th_f = math.atan2(vy, vx) % math.pi
    diff = abs(th_e - th_f)
    return kind, min(diff, math.pi - diff)


def crossings(xy, edges, ideal):
    p = [(int(x), int(y)) for x, y in xy]
    E = [(int(a), int(b)) for a, b in edges]
    out = {"proper": 0, "touching": 0, "collinear": 0, "zero": 0, "dev": 0.0}
    out["zero"] = sum(1 for a, b in E if p[a] == p[b])
    devs = []
    for i in range(len(E)):
        for j in range(i + 1, len(E)):
            k, ang = classify(p, E[i], E[j])
            if k is None:
                continue
            out[k] += 1
            if k != "collinear":
                devs.append(abs(ideal - ang))
    out["dev"] = math.fsum(devs)
    return out


def min_angle_float_sort(xy, edges):
    """Algorithm 2 literally: per vertex, float angles in [0, 2 pi), sorted; the gaps
    a_i - a_{i-1} and 2 pi - a_n + a_1; d_v from the smallest gap.  Only valid when
    no two directions at a vertex are nearly equal."""
    inc = {}
    for a, b in edges:
        a, b = int(a), int(b)
        dx, dy = int(xy[b][0]) - int(xy[a][0]), int(xy[b][1]) - int(xy[a][1])
        if dx == 0 and dy == 0:
            continue
        inc.setdefault(a, []).append(math.atan2(dy, dx) % (2 * math.pi))
        inc.setdefault(b, []).append(math.atan2(-dy, -dx) % (2 * math.pi))
    ds = []
    for v, angs in inc.items():
        if len(angs) < 2:
            continue
        angs.sort()
        gaps = [2 * math.pi - angs[-1] + angs[0]] + [angs[i] - angs[i - 1] for i in range(1, len(angs))]
        ideal = 2 * math.pi / len(angs)
        ds.append((ideal - min(gaps)) / ideal)
    if not ds:
        return 1.0, 0.0, 0
    return 1.0 - math.fsum(ds) / len(ds), math.fsum(ds), len(ds)
