"""Seeded synthetic graph layouts shaped like the workloads of arXiv 2411.09809.

This module only draws inputs: vertex coordinates and edge lists.  It holds no
readability-metric arithmetic and is the one module that both the CUDA path's
tests and the CPU oracle's tests take inputs from.

The paper measures on SNAP graphs with random layouts (Sec. 4, Experiment 1:
vertices placed uniformly at random).  Those datasets are not used; these
generators stand in for them with the sizes, coordinate distributions and edge
structure stated for each configuration below.

Edge-list conventions
  * "k-NN" edges are rank-ordered and de-duplicated: every vertex's rank-1
    nearest-neighbour edge (vertex-id order), then every rank-2 edge, and so on;
    self and duplicate edges are dropped and the list is cut at the requested
    count.
  * Random edges are uniform vertex pairs that are neither self-loops nor
    already present (in either orientation).
Coordinates are int32 in [0, 65536) unless stated otherwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

COORD_LIMIT = 65536
BASE_SEED = 20241115


@dataclass
class Layout:
    xy: np.ndarray      # [V, 2] int32 (or float32 for the differentiable workload)
    edges: np.ndarray   # [E, 2] int32 vertex ids
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def V(self) -> int:
        return int(self.xy.shape[0])

    @property
    def E(self) -> int:
        return int(self.edges.shape[0])


def _knn_table(points: np.ndarray, k: int) -> np.ndarray:
    """[V, k] neighbour ids by rank (self removed), via a k-d tree."""
    from scipy.spatial import cKDTree

    V = points.shape[0]
    kk = min(k + 1, V)
    tree = cKDTree(points.astype(np.float64))
    _, idx = tree.query(points.astype(np.float64), k=kk)
    idx = idx.reshape(V, kk)
    not_self = idx != np.arange(V)[:, None]
    # keep the first k non-self entries of each row
    order = np.argsort(~not_self, axis=1, kind="stable")
    idx = np.take_along_axis(idx, order, axis=1)[:, : kk - 1]
    return idx[:, :k] if idx.shape[1] >= k else idx


def knn_edges(points: np.ndarray, ranks: int, count: int) -> np.ndarray:
    """Rank-ordered, de-duplicated nearest-neighbour edges, cut at `count`: the
    candidates (v, rank-r neighbour of v) in rank-major, vertex-id order, each
    unordered pair kept at its first occurrence."""
    V = points.shape[0]
    if V < 2 or count <= 0:
        return np.zeros((0, 2), np.int32)
    table = _knn_table(points, ranks)
    R = table.shape[1]
    a = np.tile(np.arange(V, dtype=np.int64), R)          # rank-major order
    b = table.T.reshape(-1).astype(np.int64)
    ok = a != b
    a, b = a[ok], b[ok]
    key = np.minimum(a, b) * V + np.maximum(a, b)
    _, first = np.unique(key, return_index=True)
    first.sort()
    first = first[:count]
    return np.stack([a[first], b[first]], axis=1).astype(np.int32)


def add_random_edges(rng: np.random.Generator, V: int, edges: np.ndarray, count: int) -> np.ndarray:
    """Appends `count` uniform random edges that are not self-loops and not present
    (in either orientation)."""
    edges = edges.astype(np.int32).reshape(-1, 2)
    if count <= 0:
        return edges
    seen = np.minimum(edges[:, 0], edges[:, 1]).astype(np.int64) * V + np.maximum(edges[:, 0], edges[:, 1])
    seen = np.unique(seen)
    out = []
    have = 0
    while have < count:
        need = count - have
        cand = rng.integers(0, V, size=(2 * need + 16, 2), dtype=np.int64)
        cand = cand[cand[:, 0] != cand[:, 1]]
        key = np.minimum(cand[:, 0], cand[:, 1]) * V + np.maximum(cand[:, 0], cand[:, 1])
        _, first = np.unique(key, return_index=True)
        first.sort()
        cand, key = cand[first], key[first]
        fresh = ~np.isin(key, seen)
        cand, key = cand[fresh][:need], key[fresh][:need]
        out.append(cand)
        seen = np.union1d(seen, key)
        have += len(cand)
    ex = np.concatenate(out).astype(np.int32)
    return np.concatenate([edges, ex], axis=0)


def uniform_points(rng: np.random.Generator, V: int) -> np.ndarray:
    return rng.integers(0, COORD_LIMIT, size=(V, 2), dtype=np.int64).astype(np.int32)


def gaussian_mixture_points(rng: np.random.Generator, V: int, components: int, sigma: float) -> np.ndarray:
    centres = rng.integers(0, COORD_LIMIT, size=(components, 2)).astype(np.float64)
    which = rng.integers(0, components, size=V)
    pts = centres[which] + rng.normal(0.0, sigma, size=(V, 2))
    return np.clip(np.rint(pts), 0, COORD_LIMIT - 1).astype(np.int32)


# ----------------------------------------------------------------- workloads

def plain_layout(V: int = 2000, knn_count: int = 4000, random_count: int = 1000,
                 seed: int = BASE_SEED + 0) -> Layout:
    """Plain single layout: V uniform int points, rank 1-4 k-NN edges plus random edges
    (|V| = 2,000, |E| = 5,000; occlusion diameter 256, ideal angle 70 degrees)."""
    rng = np.random.default_rng(seed)
    xy = uniform_points(rng, V)
    e = knn_edges(xy, 4, knn_count)
    e = add_random_edges(rng, V, e, random_count)
    return Layout(xy, e, "plain_v2000_e5000", {"d": 256, "ideal_deg": 70.0, "seed": seed})


def large_sparse_layout(V: int = 200_000, knn_count: int = 495_000, random_count: int = 5_000,
                        seed: int = BASE_SEED + 1) -> Layout:
    """Large sparse layout: 64-component Gaussian mixture (sigma 1,500, centres uniform,
    rounded and clipped), rank 1-5 k-NN edges plus 1 % uniform long edges; d = 64."""
    rng = np.random.default_rng(seed)
    xy = gaussian_mixture_points(rng, V, 64, 1500.0)
    e = knn_edges(xy, 5, knn_count)
    e = add_random_edges(rng, V, e, random_count)
    return Layout(xy, e, "large_sparse_v200k_e500k", {"d": 64, "ideal_deg": 70.0, "seed": seed})


def dense_long_edge_layout(V: int = 20_000, E: int = 200_000, seed: int = BASE_SEED + 2) -> Layout:
    """Dense long-edge layout: V uniform points, E uniform random edges (the paper's
    random-layout workload); d = 256."""
    rng = np.random.default_rng(seed)
    xy = uniform_points(rng, V)
    e = add_random_edges(rng, V, np.zeros((0, 2), np.int32), E)
    return Layout(xy, e, "dense_long_edge_v20k_e200k", {"d": 256, "ideal_deg": 70.0, "seed": seed})


def paper_sized_layout(V: int = 75_879, E: int = 508_837, seed: int = BASE_SEED + 6) -> Layout:
    """The random-layout workload at the size of the paper's largest graph
    (Table 1: 75,879 vertices, 508,837 edges): V uniform points, E uniform
    random edges; d = 256."""
    rng = np.random.default_rng(seed)
    xy = uniform_points(rng, V)
    e = add_random_edges(rng, V, np.zeros((0, 2), np.int32), E)
    return Layout(xy, e, "paper_sized_v75879_e508837", {"d": 256, "ideal_deg": 70.0, "seed": seed})


def batched_layouts(n_layouts: int = 4096, v_min: int = 50, v_max: int = 20_000,
                    seed: int = BASE_SEED + 3) -> list[Layout]:
    """Batched workload: V_i log-uniform in [v_min, v_max], E_i = round(2.5 V_i) of which
    round(2.0 V_i) rank-ordered k-NN edges and the rest uniform random (20 %)."""
    rng = np.random.default_rng(seed)
    out = []
    vs = np.rint(np.exp(rng.uniform(math.log(v_min), math.log(v_max), size=n_layouts))).astype(np.int64)
    for i, V in enumerate(vs):
        V = int(V)
        E = int(round(2.5 * V))
        k = int(round(2.0 * V))
        xy = uniform_points(rng, V)
        e = knn_edges(xy, 4, k)
        e = add_random_edges(rng, V, e, E - e.shape[0])
        out.append(Layout(xy, e, f"batch{i}", {"d": 256, "ideal_deg": 70.0}))
    return out


def pack_layouts(layouts: list[Layout]):
    """(v_off, e_off, xy, edges) of a list of layouts packed one after another;
    edges keep their layout-local vertex ids."""
    v_off = np.zeros(len(layouts) + 1, np.int64)
    e_off = np.zeros(len(layouts) + 1, np.int64)
    for i, L in enumerate(layouts):
        v_off[i + 1] = v_off[i] + L.V
        e_off[i + 1] = e_off[i] + L.E
    xy = np.concatenate([L.xy for L in layouts]).astype(np.int32) if layouts else np.zeros((0, 2), np.int32)
    edges = np.concatenate([L.edges for L in layouts]).astype(np.int32) if layouts else np.zeros((0, 2), np.int32)
    return v_off, e_off, np.ascontiguousarray(xy), np.ascontiguousarray(edges)


def differentiable_layout(V: int = 50_000, knn_count: int = 142_500, random_count: int = 7_500,
                          seed: int = BASE_SEED + 4) -> Layout:
    """Differentiable workload: float32 coordinates uniform in [0, 1)^2, rank 1-5 k-NN
    edges plus 5 % random edges."""
    rng = np.random.default_rng(seed)
    xy = rng.random((V, 2), dtype=np.float32)
    e = knn_edges(xy, 5, knn_count)
    e = add_random_edges(rng, V, e, random_count)
    return Layout(xy, e, "differentiable_v50k_e150k", {"ideal_deg": 70.0, "seed": seed})


def tiny_degenerate_layout(rng: np.random.Generator, V: int, E: int, span: int = 8,
                           offset: int = 0) -> Layout:
    """Small layouts with coordinates in [offset, offset + span)^2: collinear, touching,
    coincident and zero-length cases dominate.  Edges are random non-self pairs
    (duplicates allowed)."""
    xy = (offset + rng.integers(0, span, size=(V, 2))).astype(np.int32)
    a = rng.integers(0, V, size=E)
    b = (a + rng.integers(1, V, size=E)) % V
    return Layout(xy, np.stack([a, b], axis=1).astype(np.int32), "tiny_degenerate")
