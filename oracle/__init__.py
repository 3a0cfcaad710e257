"""CPU oracle for the readability metrics -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It wraps the plain C brute force in
`gr_oracle.c` (compiled here with gcc + OpenMP, no CUDA) through ctypes and
shares no code with the CUDA library.  Every function takes numpy arrays:
``xy`` int32 [V, 2], ``edges`` int32 [E, 2].

Each function follows a definition of arXiv 2411.09809:
  node_occlusion          -- Sec. 2.1, Algorithm 1
  crossings               -- Sec. 2.1, Algorithms 4 and 5
  crossings_of_edges      -- the same, restricted to sampled edges
  min_angle               -- Sec. 2.1, Algorithm 2
  edge_length_variation   -- Sec. 2.1, Algorithm 3
the paper's approximate strip algorithms (``strip_oracle.c``):
  strip_crossings         -- Sec. 3.2.2 (E_c estimate) and Sec. 3.2.3 with
      Eq. 1 (crossing-angle estimate), vertical or horizontal strips;
  strip_eq1, strip_category -- Eq. 1 and its 8 angle categories;
and, for FP32 coordinates (the differentiable form; ``xy`` float32 [V, 2]):
  orient_f32, crossings_f32, min_angle_f32, edge_length_variation_f32 -- the
      same definitions with exact orientation predicates on FP32 inputs;
  diff_terms_and_grads    -- E_ca, M_l, M_a and their FP64 gradients with the
      crossing set and every vertex's smallest gap held fixed.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gr_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "strip_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "libgr_oracle.so")
_lib = None

DEFAULT_IDEAL = 7.0 * math.pi / 18.0  # 70 degrees (Sec. 2.1)


def build(force: bool = False) -> str:
    """Compiles the oracle shared library with gcc (plain C, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
             *_SRCS, "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i64 = ctypes.c_int64
        lib.oracle_validate.argtypes = [i32p, i64, i32p, i64]
        lib.oracle_validate.restype = ctypes.c_int
        lib.oracle_node_occlusion.argtypes = [i32p, i64, i64]
        lib.oracle_node_occlusion.restype = i64
        lib.oracle_crossings.argtypes = [i32p, i64, i32p, i64, ctypes.c_double, i64p, f64p]
        lib.oracle_crossings.restype = ctypes.c_int
        lib.oracle_crossings_of_edges.argtypes = [i32p, i64, i32p, i64, ctypes.c_double,
                                                  i64p, i64, i64p, f64p]
        lib.oracle_crossings_of_edges.restype = ctypes.c_int
        lib.oracle_min_angle.argtypes = [i32p, i64, i32p, i64, f64p]
        lib.oracle_min_angle.restype = ctypes.c_int
        lib.oracle_edge_length_variation.argtypes = [i32p, i64, i32p, i64]
        lib.oracle_edge_length_variation.restype = ctypes.c_double
        lib.oracle_strip_crossings.argtypes = [i32p, i64, i32p, i64, i64, ctypes.c_int, ctypes.c_double, i64p,
                                               f64p, i64p]
        lib.oracle_strip_crossings.restype = ctypes.c_int
        lib.oracle_strip_eq1.argtypes = [ctypes.c_double, ctypes.c_double, i64p, f64p]
        lib.oracle_strip_eq1.restype = ctypes.c_double
        lib.oracle_strip_category.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_strip_category.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        fl = ctypes.c_float
        lib.oracle_orient_f32.argtypes = [fl, fl, fl, fl, fl, fl]
        lib.oracle_orient_f32.restype = ctypes.c_int
        lib.oracle_orient_f32_exact.argtypes = [fl, fl, fl, fl, fl, fl]
        lib.oracle_orient_f32_exact.restype = ctypes.c_int
        lib.oracle_crossings_f32.argtypes = [f32p, i64, i32p, i64, ctypes.c_double, i64p, f64p,
                                             ctypes.c_void_p, i64]
        lib.oracle_crossings_f32.restype = ctypes.c_int
        lib.oracle_min_angle_f32.argtypes = [f32p, i64, i32p, i64, f64p, ctypes.c_void_p]
        lib.oracle_min_angle_f32.restype = ctypes.c_int
        lib.oracle_edge_length_variation_f32.argtypes = [f32p, i64, i32p, i64]
        lib.oracle_edge_length_variation_f32.restype = ctypes.c_double
        lib.oracle_diff_terms_and_grads.argtypes = [f32p, i64, i32p, i64, ctypes.c_double, f64p, f64p, f64p, f64p,
                                                    i64p]
        lib.oracle_diff_terms_and_grads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _xy(xy) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    return a


def _edges(edges) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def validate(xy, edges) -> int:
    """0 = valid, 1 = bad vertex id or self-loop, 2 = coordinate outside [0, 65536)."""
    xy, edges = _xy(xy), _edges(edges)
    return int(_load().oracle_validate(xy, len(xy), edges, len(edges)))


def node_occlusion(xy, d: int) -> int:
    """N_c: unordered vertex pairs at squared distance < d^2 (d = 2r)."""
    xy = _xy(xy)
    r = int(_load().oracle_node_occlusion(xy, len(xy), int(d)))
    if r < 0:
        raise ValueError("d must be >= 0")
    return r


@dataclass
class Crossings:
    proper: int
    touching: int
    collinear: int
    zero_length_edges: int
    crossings: int          # E_c = proper + touching
    angle_dev_sum: float    # sum over E_c pairs of |ideal - a_c| (radians)
    E_ca: float


def crossings(xy, edges, ideal: float = DEFAULT_IDEAL) -> Crossings:
    xy, edges = _xy(xy), _edges(edges)
    counts = np.zeros(5, np.int64)
    fv = np.zeros(2, np.float64)
    if _load().oracle_crossings(xy, len(xy), edges, len(edges), float(ideal), counts, fv) != 0:
        raise ValueError("ideal angle must be in (0, pi/2]")
    return Crossings(int(counts[0]), int(counts[1]), int(counts[2]), int(counts[3]),
                     int(counts[4]), float(fv[0]), float(fv[1]))


def crossings_of_edges(xy, edges, sample, ideal: float = DEFAULT_IDEAL):
    """Per sampled edge: int64 [n, 3] (proper, touching, collinear) and float64 [n]
    sum of |ideal - a_c| over that edge's E_c partners."""
    xy, edges = _xy(xy), _edges(edges)
    sample = np.ascontiguousarray(np.asarray(sample, dtype=np.int64))
    out_c = np.zeros((len(sample), 3), np.int64)
    out_d = np.zeros(len(sample), np.float64)
    if _load().oracle_crossings_of_edges(xy, len(xy), edges, len(edges), float(ideal),
                                         sample, len(sample), out_c, out_d) != 0:
        raise ValueError("ideal angle must be in (0, pi/2]")
    return out_c, out_d


@dataclass
class MinAngle:
    M_a: float
    sum_d: float
    n_vertices: int


def min_angle(xy, edges) -> MinAngle:
    xy, edges = _xy(xy), _edges(edges)
    out = np.zeros(3, np.float64)
    _load().oracle_min_angle(xy, len(xy), edges, len(edges), out)
    return MinAngle(float(out[0]), float(out[1]), int(out[2]))


def edge_length_variation(xy, edges) -> float:
    xy, edges = _xy(xy), _edges(edges)
    return float(_load().oracle_edge_length_variation(xy, len(xy), edges, len(edges)))


# ---------------------------------------------------------------- FP32 form

def _xyf(xy) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(-1, 2))


def orient_f32(a, b, c) -> int:
    """Exact sign of (b - a) x (c - a) for FP32 points (FP64 error-bound filter,
    then expansion arithmetic)."""
    return int(_load().oracle_orient_f32(*(float(np.float32(v)) for v in (*a, *b, *c))))


def orient_f32_exact(a, b, c) -> int:
    """The same sign, always by expansion arithmetic."""
    return int(_load().oracle_orient_f32_exact(*(float(np.float32(v)) for v in (*a, *b, *c))))


def crossings_f32(xy, edges, ideal: float = DEFAULT_IDEAL, return_pairs: bool = False):
    """Crossings and crossing angle on FP32 coordinates (exact predicates)."""
    xy, edges = _xyf(xy), _edges(edges)
    counts = np.zeros(5, np.int64)
    fv = np.zeros(2, np.float64)
    lib = _load()
    if lib.oracle_crossings_f32(xy, len(xy), edges, len(edges), float(ideal), counts, fv, None, 0) != 0:
        raise ValueError("ideal angle must be in (0, pi/2]")
    res = Crossings(int(counts[0]), int(counts[1]), int(counts[2]), int(counts[3]), int(counts[4]),
                    float(fv[0]), float(fv[1]))
    if not return_pairs:
        return res
    pairs = np.zeros((max(res.crossings, 1), 2), np.int32)
    lib.oracle_crossings_f32(xy, len(xy), edges, len(edges), float(ideal), counts, fv,
                             pairs.ctypes.data, res.crossings)
    return res, pairs[: res.crossings]


def min_angle_f32(xy, edges, return_args: bool = False):
    xy, edges = _xyf(xy), _edges(edges)
    out = np.zeros(3, np.float64)
    args = np.zeros((max(len(xy), 1), 2), np.int32)
    _load().oracle_min_angle_f32(xy, len(xy), edges, len(edges), out, args.ctypes.data)
    r = MinAngle(float(out[0]), float(out[1]), int(out[2]))
    return (r, args[: len(xy)]) if return_args else r


def edge_length_variation_f32(xy, edges) -> float:
    xy, edges = _xyf(xy), _edges(edges)
    return float(_load().oracle_edge_length_variation_f32(xy, len(xy), edges, len(edges)))


def diff_terms_and_grads(xy, edges, ideal: float = DEFAULT_IDEAL, return_counts: bool = False):
    """(E_ca, M_l, M_a) and their FP64 gradients [V, 2] each, with the crossing set
    and the smallest gaps held fixed; with return_counts, also the crossing counts
    (proper, touching, collinear, zero-length edges, E_c) of the same pass."""
    xy, edges = _xyf(xy), _edges(edges)
    V = len(xy)
    terms = np.zeros(3, np.float64)
    counts = np.zeros(5, np.int64)
    g = [np.zeros((max(V, 1), 2), np.float64) for _ in range(3)]
    if _load().oracle_diff_terms_and_grads(xy, V, edges, len(edges), float(ideal), terms, *g, counts) != 0:
        raise ValueError("ideal angle must be in (0, pi/2]")
    out = (terms, g[0][:V], g[1][:V], g[2][:V])
    return out + (counts,) if return_counts else out


# ------------------------------------------------ approximate strip algorithm

@dataclass
class StripEstimate:
    crossings: int       # pairs whose key order reverses inside a strip both span (Sec. 3.2.2)
    term_sum: float      # sum over those pairs of |ideal - angle| / ideal (Sec. 3.2.3, Eq. 1)
    records: int         # (segment, strip) pairs
    E_ca: float          # 1 - term_sum / crossings (1 when there is none)
    orientation: int     # 0 vertical strips, 1 horizontal


def strip_crossings(xy, edges, l: int, orientation: int = 0, ideal: float = DEFAULT_IDEAL) -> StripEstimate:
    """The strip estimates of E_c and E_ca (Sec. 3.2.2-3.2.3) for strips of width l.
    orientation 0: vertical strips, 1: horizontal, 2: both (the larger count)."""
    if orientation == 2:
        a = strip_crossings(xy, edges, l, 0, ideal)
        b = strip_crossings(xy, edges, l, 1, ideal)
        return b if b.crossings > a.crossings else a
    xy, edges = _xy(xy), _edges(edges)
    c = np.zeros(1, np.int64)
    t = np.zeros(1, np.float64)
    r = np.zeros(1, np.int64)
    if _load().oracle_strip_crossings(xy, xy.shape[0], edges, edges.shape[0], int(l), int(orientation),
                                      float(ideal), c, t, r) != 0:
        raise ValueError("bad strip width, orientation or edge ids")
    n = int(c[0])
    return StripEstimate(n, float(t[0]), int(r[0]), 1.0 - float(t[0]) / n if n > 0 else 1.0, int(orientation))


def strip_eq1(theta_i: float, ideal: float, counts, sums) -> float:
    """Eq. 1: category counts and angle sums (LIL, LIG, LOG, LOL, RIL, RIG, ROG, ROL)
    -> sum of |ideal - angle| over the crossing segments."""
    return float(_load().oracle_strip_eq1(float(theta_i), float(ideal), np.ascontiguousarray(counts, np.int64),
                                          np.ascontiguousarray(sums, np.float64)))


def strip_category(theta_i: float, theta_j: float, ideal: float) -> int:
    """Angle category (0..7 = LIL, LIG, LOG, LOL, RIL, RIG, ROG, ROL) of theta_j relative to theta_i."""
    return int(_load().oracle_strip_category(float(theta_i), float(theta_j), float(ideal)))
