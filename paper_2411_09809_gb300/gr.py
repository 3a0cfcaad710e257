"""Thin ctypes binding of libgr (include/gr.h), with the C entry points' names.

Argument marshalling only: every step of every metric runs in the CUDA
library.  Inputs may be CUDA tensors (torch), CPU tensors or numpy arrays; the
library copies host inputs to the device itself.  If libgr.so has not been
built, loading raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import c_double, c_int32, c_int64, c_uint32, c_void_p

from . import build as _build

GR_OK, GR_EINVAL, GR_ERANGE, GR_ENOMEM, GR_ECUDA, GR_ETIMEOUT, GR_ENOTSUP = range(7)
GR_COORD_I32, GR_COORD_F32 = 0, 1
GR_LONG_AUTO, GR_LONG_ALLPAIRS, GR_LONG_GRID = 0, 1, 2
GR_METRIC_OCCLUSION, GR_METRIC_MIN_ANGLE, GR_METRIC_EDGE_LENGTH, GR_METRIC_CROSSINGS = 1, 2, 4, 8
GR_METRIC_ALL = 15
GR_PATH_AUTO, GR_PATH_GRID, GR_PATH_ALLPAIRS, GR_PATH_DELTA = 0, 1, 2, 3
DEFAULT_IDEAL = 7.0 * math.pi / 18.0

_STATUS_NAMES = ["GR_OK", "GR_EINVAL", "GR_ERANGE", "GR_ENOMEM", "GR_ECUDA", "GR_ETIMEOUT", "GR_ENOTSUP"]


class GrError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = _STATUS_NAMES[status] if 0 <= status < len(_STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class gr_options(ctypes.Structure):
    _fields_ = [("crossing_path", c_int32), ("cell_log2", c_int32),
                ("occlusion_path", c_int32), ("profile", c_int32), ("long_pairs", c_int32)]


class gr_partial(ctypes.Structure):
    """One part's tallies (gr_evaluate_part): every field an int64, summed over
    the parts by an integer all-reduce."""
    _fields_ = [(name, c_int64) for name in (
        "proper", "touching", "collinear_overlaps", "occlusion_pairs", "dev_hi32", "dev_lo32",
        "metrics", "crossing_path", "cell_log2", "occlusion_path", "zero_length_edges", "pairs_tested",
        "n_vertices_counted", "grid_records", "min_angle_sum_d_bits", "M_a_bits", "M_l_bits")]


class gr_params(ctypes.Structure):
    _fields_ = [("ideal_rad", c_double), ("occlusion_d", c_int64)]


class gr_crossing_counts(ctypes.Structure):
    _fields_ = [("crossings", c_int64), ("proper", c_int64), ("touching", c_int64),
                ("collinear_overlaps", c_int64), ("zero_length_edges", c_int64),
                ("pairs_tested", c_int64)]


class gr_crossing_angle_result(ctypes.Structure):
    _fields_ = [("c", gr_crossing_counts), ("angle_dev_sum", c_double), ("ideal_rad", c_double),
                ("E_ca", c_double)]


class gr_min_angle_result(ctypes.Structure):
    _fields_ = [("M_a", c_double), ("sum_d", c_double), ("n_vertices_counted", c_int64)]


class gr_result(ctypes.Structure):
    _fields_ = [("metrics", c_uint32), ("crossing_path", c_int32), ("cell_log2", c_int32),
                ("occlusion_path", c_int32), ("crossing", gr_crossing_angle_result),
                ("occlusion_pairs", c_int64), ("occlusion_d", c_int64),
                ("min_angle", gr_min_angle_result), ("M_l", c_double), ("grid_records", c_int64)]


GR_STRIP_VERTICAL, GR_STRIP_HORIZONTAL, GR_STRIP_BOTH = 0, 1, 2


class gr_strip_result(ctypes.Structure):
    _fields_ = [("crossings", c_int64), ("records", c_int64), ("strips", c_int64),
                ("angle_dev_sum", c_double), ("ideal_rad", c_double), ("E_ca", c_double),
                ("orientation", c_int32), ("strip_width", c_int32)]


GR_PHASE_NAMES = ["gather", "edge_length", "min_angle", "occl_bin", "occl_pairs", "cross_bin",
                  "cross_scatter", "cross_pairs", "finalize", "diff_backward", "strip_sort", "strip_count"]


class gr_profile(ctypes.Structure):
    _fields_ = [("ms", c_double * 16), ("calls", c_int64 * 16)]

    def as_dict(self) -> dict:
        return {n: (self.ms[i], self.calls[i]) for i, n in enumerate(GR_PHASE_NAMES)}


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Loads libgr.so (built by ``paper_2411_09809_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libgr.so is not built ({_build.LIB}); call build() first")
    lib = ctypes.CDLL(_build.LIB)
    P = c_void_p
    sigs = {
        "gr_layout_create": ([ctypes.POINTER(c_void_p), P, c_int32, c_int64, P, c_int64,
                              ctypes.POINTER(gr_options), P], c_int32),
        "gr_layout_update": ([P, P, P], c_int32),
        "gr_layout_destroy": ([P], c_int32),
        "gr_evaluate": ([P, c_uint32, ctypes.POINTER(gr_params), ctypes.POINTER(gr_result)], c_int32),
        "gr_node_occlusion": ([P, c_int64, ctypes.POINTER(c_int64)], c_int32),
        "gr_min_angle": ([P, ctypes.POINTER(gr_min_angle_result)], c_int32),
        "gr_edge_length_variation": ([P, ctypes.POINTER(c_double)], c_int32),
        "gr_edge_crossings": ([P, ctypes.POINTER(gr_crossing_counts)], c_int32),
        "gr_crossing_angle": ([P, c_double, ctypes.POINTER(gr_crossing_angle_result)], c_int32),
        "gr_crossings_per_edge": ([P, c_double, P, P], c_int32),
        "gr_profile_enable": ([P, c_int32], c_int32),
        "gr_profile_read": ([P, ctypes.POINTER(gr_profile), c_int32], c_int32),
        "gr_kernel_launches": ([], c_int64),
        "gr_io_bytes": ([P, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64)], c_int32),
        "gr_batch_tuning": ([P, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)], c_int32),
        "gr_evaluate_part": ([P, c_uint32, ctypes.POINTER(gr_params), c_int32, c_int32,
                              ctypes.POINTER(gr_partial)], c_int32),
        "gr_combine_parts": ([ctypes.POINTER(gr_partial), ctypes.POINTER(gr_params),
                              ctypes.POINTER(gr_result)], c_int32),
        "gr_crossing_angle_noalloc": ([P, c_int64, P, c_int64, c_double,
                                       ctypes.POINTER(gr_crossing_angle_result), P], c_int32),
        "gr_batch_create": ([ctypes.POINTER(c_void_p), c_int64, P, P, P, c_int32, P,
                             ctypes.POINTER(gr_options), P], c_int32),
        "gr_batch_update": ([P, P, P], c_int32),
        "gr_batch_evaluate": ([P, c_uint32, ctypes.POINTER(gr_params), P], c_int32),
        "gr_batch_destroy": ([P], c_int32),
        "gr_move_vertices": ([P, c_int64, P, P, c_uint32, ctypes.POINTER(gr_params), ctypes.POINTER(gr_result)],
                             c_int32),
        "gr_strip_crossings": ([P, c_int32, c_int32, c_double, ctypes.POINTER(gr_strip_result)], c_int32),
        "gr_evaluate_async": ([P, c_uint32, ctypes.POINTER(gr_params), P, P], c_int32),
        "gr_batch_evaluate_async": ([P, c_uint32, ctypes.POINTER(gr_params), P, P], c_int32),
        "gr_diff_forward": ([P, c_double, P, P], c_int32),
        "gr_diff_backward": ([P, P, P, P], c_int32),
        "gr_last_error": ([], ctypes.c_char_p),
        "gr_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(st: int) -> None:
    if st != GR_OK:
        raise GrError(st, load().gr_last_error().decode())


def _buffer(x, dtype: str):
    """(pointer, keepalive) for a torch tensor or numpy array of the given dtype."""
    if x is None:
        return None, None
    try:
        import torch  # noqa: F401
        if isinstance(x, torch.Tensor):
            want = {"int32": torch.int32, "float32": torch.float32, "int64": torch.int64,
                    "float64": torch.float64, "uint8": torch.uint8}[dtype]
            if x.dtype != want:
                raise TypeError(f"expected a {dtype} tensor, got {x.dtype}")
            if not x.is_contiguous():
                x = x.contiguous()
            return x.data_ptr(), x
    except ImportError:
        pass
    import numpy as np
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def _stream_of(*tensors):
    try:
        import torch
        for t in tensors:
            if isinstance(t, torch.Tensor) and t.is_cuda:
                return torch.cuda.current_stream(t.device).cuda_stream
    except ImportError:
        pass
    return None


def _count(x) -> int:
    return int(x.shape[0]) if hasattr(x, "shape") else len(x)


# ------------------------------------------------------------ C entry points

def gr_layout_create(xy, edges, coord_type: int = GR_COORD_I32, opt: gr_options | None = None,
                     stream=None) -> c_void_p:
    lib = load()
    xp, xk = _buffer(xy, "int32" if coord_type == GR_COORD_I32 else "float32")
    ep, ek = _buffer(edges, "int32")
    if stream is None:
        stream = _stream_of(xy, edges)
    h = c_void_p()
    st = lib.gr_layout_create(ctypes.byref(h), xp, coord_type, _count(xk), ep, _count(ek),
                              ctypes.byref(opt) if opt is not None else None, stream)
    _check(st)
    return h


def gr_layout_update(layout, xy, edges=None, coord_type: int = GR_COORD_I32) -> None:
    lib = load()
    xp, xk = _buffer(xy, "int32" if coord_type == GR_COORD_I32 else "float32")
    ep, ek = _buffer(edges, "int32")
    _check(lib.gr_layout_update(layout, xp, ep))


def gr_move_vertices(layout, ids, xy_new, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                     occlusion_d: int = 0) -> gr_result:
    """Moves vertices ids[i] to xy_new[i] and evaluates the moved layout
    (incrementally when the previous evaluation allows it)."""
    ip, ik = _buffer(ids, "int32")
    xp, xk = _buffer(xy_new, "int32")
    n = _count(ik)
    if tuple(xk.shape) != (n, 2):
        raise ValueError(f"xy_new must have shape ({n}, 2), got {tuple(xk.shape)}")
    r = gr_result()
    p = gr_params(float(ideal_rad), int(occlusion_d))
    _check(load().gr_move_vertices(layout, n, ip, xp, metrics, ctypes.byref(p), ctypes.byref(r)))
    return r


def gr_diff_forward(layout, ideal_rad: float = 0.0, out3=None, stream: int = 0):
    """{E_ca, M_l, M_a} of an FP32 layout into `out3` (a float32 [3] tensor or array;
    a new numpy array when None), keeping what gr_diff_backward needs; ordered
    after the work on `stream` (a cudaStream_t as int; 0: the layout's own)."""
    import numpy as np
    if out3 is None:
        out3 = np.zeros(3, np.float32)
    op, ok = _buffer(out3, "float32")
    _check(load().gr_diff_forward(layout, float(ideal_rad), op, ctypes.c_void_p(int(stream) or None)))
    if ok is not out3:  # a converted copy: hand back the values
        return ok
    return out3


def gr_diff_backward(layout, gout3, d_grad_xy, stream: int = 0) -> None:
    """Gradient of gout3 . (E_ca, M_l, M_a) w.r.t. the coordinates into d_grad_xy
    (float32 [V, 2] device tensor, overwritten), ordered on `stream` (a
    cudaStream_t as int; 0: the layout's own)."""
    gp, gk = _buffer(gout3, "float32")
    dp, dk = _buffer(d_grad_xy, "float32")
    if dk is not d_grad_xy:
        raise TypeError("d_grad_xy must be a contiguous float32 device tensor")
    _check(load().gr_diff_backward(layout, gp, dp, ctypes.c_void_p(int(stream) or None)))


def gr_layout_destroy(layout) -> None:
    _check(load().gr_layout_destroy(layout))


def gr_evaluate(layout, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                occlusion_d: int = 0) -> gr_result:
    r = gr_result()
    p = gr_params(float(ideal_rad), int(occlusion_d))
    _check(load().gr_evaluate(layout, metrics, ctypes.byref(p), ctypes.byref(r)))
    return r


def gr_evaluate_part(layout, part: int, n_parts: int, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                     occlusion_d: int = 0) -> gr_partial:
    """Part `part` of `n_parts` of the pair work of an evaluation (its tallies)."""
    out = gr_partial()
    p = gr_params(float(ideal_rad), int(occlusion_d))
    _check(load().gr_evaluate_part(layout, metrics, ctypes.byref(p), int(part), int(n_parts), ctypes.byref(out)))
    return out


def gr_batch_tuning(batch) -> tuple[int, int]:
    """(cell-size offset, tile height) that gr_batch_create settled on."""
    off, tile = c_int32(), c_int32()
    _check(load().gr_batch_tuning(batch, ctypes.byref(off), ctypes.byref(tile)))
    return off.value, tile.value


def gr_combine_parts(total: gr_partial, ideal_rad: float = 0.0, occlusion_d: int = 0) -> gr_result:
    """The gr_result of the summed tallies of all parts (host arithmetic)."""
    r = gr_result()
    p = gr_params(float(ideal_rad), int(occlusion_d))
    _check(load().gr_combine_parts(ctypes.byref(total), ctypes.byref(p), ctypes.byref(r)))
    return r


def partial_to_list(p: gr_partial) -> list[int]:
    return [getattr(p, name) for name, _ in gr_partial._fields_]


def partial_from_list(values) -> gr_partial:
    return gr_partial(*[int(v) for v in values])


def gr_node_occlusion(layout, d: int) -> int:
    out = c_int64()
    _check(load().gr_node_occlusion(layout, int(d), ctypes.byref(out)))
    return out.value


def gr_min_angle(layout) -> gr_min_angle_result:
    out = gr_min_angle_result()
    _check(load().gr_min_angle(layout, ctypes.byref(out)))
    return out


def gr_edge_length_variation(layout) -> float:
    out = c_double()
    _check(load().gr_edge_length_variation(layout, ctypes.byref(out)))
    return out.value


def gr_edge_crossings(layout) -> gr_crossing_counts:
    out = gr_crossing_counts()
    _check(load().gr_edge_crossings(layout, ctypes.byref(out)))
    return out


def gr_crossing_angle(layout, ideal_rad: float = 0.0) -> gr_crossing_angle_result:
    out = gr_crossing_angle_result()
    _check(load().gr_crossing_angle(layout, float(ideal_rad), ctypes.byref(out)))
    return out


def result_buffer(n: int = 1, device=None):
    """A CUDA byte tensor for n gr_result structs (the asynchronous evaluations' output)."""
    import torch
    return torch.empty(n * ctypes.sizeof(gr_result), dtype=torch.uint8, device=device or "cuda")


def results_from_device(buf, n: int = 1) -> list:
    """The gr_result structs of a result buffer (copies it to the host; synchronises)."""
    raw = bytes(buf.detach().cpu().numpy().tobytes())
    size = ctypes.sizeof(gr_result)
    return [gr_result.from_buffer_copy(raw[i * size:(i + 1) * size]) for i in range(n)]


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def gr_evaluate_async(layout, d_result, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                      occlusion_d: int = 0, stream=None) -> None:
    """Enqueues an evaluation writing its gr_result into d_result (see result_buffer)."""
    rp, rk = _buffer(d_result, "uint8")
    p = gr_params(float(ideal_rad), int(occlusion_d))
    _check(load().gr_evaluate_async(layout, metrics, ctypes.byref(p), rp, _stream_ptr(stream)))


def gr_batch_evaluate_async(batch, d_results, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                            occlusion_d: int = 0, stream=None) -> None:
    """Enqueues a batch evaluation writing its gr_result structs into d_results."""
    rp, rk = _buffer(d_results, "uint8")
    p = gr_params(float(ideal_rad), int(occlusion_d))
    _check(load().gr_batch_evaluate_async(batch, metrics, ctypes.byref(p), rp, _stream_ptr(stream)))


def gr_strip_crossings(layout, strip_width: int, orientation: int = GR_STRIP_VERTICAL,
                       ideal_rad: float = 0.0) -> gr_strip_result:
    """The paper's approximate strip estimates of E_c and E_ca (Sec. 3.2.2-3.2.3)."""
    out = gr_strip_result()
    _check(load().gr_strip_crossings(layout, int(strip_width), int(orientation), float(ideal_rad),
                                     ctypes.byref(out)))
    return out


def gr_crossings_per_edge(layout, ideal_rad: float, d_counts, d_dev) -> None:
    """d_counts: CUDA int64 tensor [E, 3]; d_dev: CUDA float64 tensor [E] (overwritten)."""
    cp, ck = _buffer(d_counts, "int64")
    dp, dk = _buffer(d_dev, "float64")
    _check(load().gr_crossings_per_edge(layout, float(ideal_rad), cp, dp))


GR_NOALLOC_MAX_EDGES = 32768


def gr_crossing_angle_noalloc(d_xy, d_edges, ideal_rad: float = 0.0, stream=None) -> gr_crossing_angle_result:
    """Crossings and crossing angle without any device allocation (CUDA int32
    tensors, at most GR_NOALLOC_MAX_EDGES edges); see include/gr.h."""
    xp, xk = _buffer(d_xy, "int32")
    ep, ek = _buffer(d_edges, "int32")
    if stream is None:
        stream = _stream_of(d_xy, d_edges)
    out = gr_crossing_angle_result()
    _check(load().gr_crossing_angle_noalloc(xp, _count(xk), ep, _count(ek), float(ideal_rad),
                                            ctypes.byref(out), stream))
    return out


def gr_profile_enable(layout, enable: bool = True) -> None:
    _check(load().gr_profile_enable(layout, 1 if enable else 0))


def gr_profile_read(layout, reset: bool = False) -> gr_profile:
    out = gr_profile()
    _check(load().gr_profile_read(layout, ctypes.byref(out), 1 if reset else 0))
    return out


def gr_io_bytes(layout) -> tuple[int, int]:
    h2d, d2h = c_int64(), c_int64()
    _check(load().gr_io_bytes(layout, ctypes.byref(h2d), ctypes.byref(d2h)))
    return h2d.value, d2h.value


def gr_kernel_launches() -> int:
    return int(load().gr_kernel_launches())


def gr_last_error() -> str:
    return load().gr_last_error().decode()


def gr_version() -> str:
    return load().gr_version().decode()


def gr_batch_create(n_layouts: int, v_off, e_off, xy, edges, opt: gr_options | None = None,
                    stream=None) -> c_void_p:
    vp, vk = _buffer(v_off, "int64")
    ep_, ek_ = _buffer(e_off, "int64")
    xp, xk = _buffer(xy, "int32")
    ep, ek = _buffer(edges, "int32")
    if stream is None:
        stream = _stream_of(xy, edges)
    h = c_void_p()
    _check(load().gr_batch_create(ctypes.byref(h), int(n_layouts), vp, ep_, xp, GR_COORD_I32, ep,
                                  ctypes.byref(opt) if opt is not None else None, stream))
    return h


def gr_batch_update(batch, xy, edges=None) -> None:
    xp, xk = _buffer(xy, "int32")
    ep, ek = _buffer(edges, "int32")
    _check(load().gr_batch_update(batch, xp, ep))


def gr_batch_evaluate(batch, n_layouts: int, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                      occlusion_d: int = 0, out=None):
    """Returns a ctypes array of n_layouts gr_result (or fills `out`, a CUDA
    buffer of n_layouts * sizeof(gr_result) bytes)."""
    p = gr_params(float(ideal_rad), int(occlusion_d))
    if out is None:
        res = (gr_result * int(n_layouts))()
        _check(load().gr_batch_evaluate(batch, metrics, ctypes.byref(p), ctypes.cast(res, c_void_p)))
        return res
    op, ok = _buffer(out, "int64") if not hasattr(out, "data_ptr") else (out.data_ptr(), out)
    _check(load().gr_batch_evaluate(batch, metrics, ctypes.byref(p), op))
    return out


def gr_batch_destroy(batch) -> None:
    _check(load().gr_batch_destroy(batch))


class Batch:
    """Owns a gr_batch handle over packed layouts (see include/gr.h)."""

    def __init__(self, v_off, e_off, xy, edges, opt: gr_options | None = None, stream=None):
        self.n = int(len(v_off) - 1)
        self.handle = gr_batch_create(self.n, v_off, e_off, xy, edges, opt, stream)

    def update(self, xy, edges=None) -> None:
        gr_batch_update(self.handle, xy, edges)

    def evaluate(self, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0, occlusion_d: int = 0):
        return gr_batch_evaluate(self.handle, self.n, metrics, ideal_rad, occlusion_d)

    def evaluate_async(self, d_results, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                       occlusion_d: int = 0, stream=None) -> None:
        gr_batch_evaluate_async(self.handle, d_results, metrics, ideal_rad, occlusion_d, stream)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            gr_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience

class Layout:
    """Owns a gr_layout handle: ``Layout(xy, edges).evaluate(...)``."""

    def __init__(self, xy, edges, opt: gr_options | None = None, stream=None,
                 coord_type: int = GR_COORD_I32):
        self.E = _count(edges)
        self.V = _count(xy)
        self.coord_type = coord_type
        self.handle = gr_layout_create(xy, edges, coord_type, opt, stream)

    def update(self, xy, edges=None) -> None:
        gr_layout_update(self.handle, xy, edges, self.coord_type)

    def evaluate(self, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0, occlusion_d: int = 0) -> gr_result:
        return gr_evaluate(self.handle, metrics, ideal_rad, occlusion_d)

    def move(self, ids, xy_new, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
             occlusion_d: int = 0) -> gr_result:
        return gr_move_vertices(self.handle, ids, xy_new, metrics, ideal_rad, occlusion_d)

    def evaluate_async(self, d_result, metrics: int = GR_METRIC_ALL, ideal_rad: float = 0.0,
                       occlusion_d: int = 0, stream=None) -> None:
        gr_evaluate_async(self.handle, d_result, metrics, ideal_rad, occlusion_d, stream)

    def strips(self, strip_width: int, orientation: int = GR_STRIP_VERTICAL,
               ideal_rad: float = 0.0) -> gr_strip_result:
        return gr_strip_crossings(self.handle, strip_width, orientation, ideal_rad)

    def profile(self, reset: bool = False) -> dict:
        return gr_profile_read(self.handle, reset).as_dict()

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            gr_layout_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
