"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point include/gr.h declares, its structs have the layout the binding
assumes, and argument checks that precede any CUDA call report GR_EINVAL."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2411_09809_gb300 import build, gr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gr.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["gr_layout_create", "gr_layout_update", "gr_layout_destroy", "gr_evaluate",
              "gr_node_occlusion", "gr_min_angle", "gr_edge_length_variation",
              "gr_edge_crossings", "gr_crossing_angle", "gr_crossings_per_edge",
              "gr_last_error", "gr_version", "gr_profile_enable", "gr_profile_read",
              "gr_kernel_launches", "gr_io_bytes", "gr_crossing_angle_noalloc",
              "gr_batch_create", "gr_batch_update", "gr_batch_evaluate", "gr_batch_destroy",
              "gr_diff_forward", "gr_diff_backward", "gr_move_vertices", "gr_strip_crossings",
              "gr_evaluate_async", "gr_batch_evaluate_async", "gr_evaluate_part", "gr_combine_parts"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gr.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gr_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gr_options), sizeof(gr_params),
         sizeof(gr_crossing_counts), sizeof(gr_crossing_angle_result),
         sizeof(gr_min_angle_result), sizeof(gr_result), sizeof(gr_profile));
  printf("%zu %zu %zu %zu\\n", offsetof(gr_result, crossing), offsetof(gr_result, occlusion_pairs),
         offsetof(gr_result, min_angle), offsetof(gr_result, grid_records));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    offs = [int(v) for v in lines[1].split()]
    assert sizes == [ctypes.sizeof(t) for t in (gr.gr_options, gr.gr_params, gr.gr_crossing_counts,
                                                gr.gr_crossing_angle_result, gr.gr_min_angle_result,
                                                gr.gr_result, gr.gr_profile)]
    assert offs == [gr.gr_result.crossing.offset, gr.gr_result.occlusion_pairs.offset,
                    gr.gr_result.min_angle.offset, gr.gr_result.grid_records.offset]


def test_argument_errors_need_no_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.gr_layout_create(None, None, 0, 0, None, 0, None, None) == gr.GR_EINVAL
    assert lib.gr_layout_create(ctypes.byref(h), None, 0, -1, None, 0, None, None) == gr.GR_EINVAL
    assert lib.gr_layout_create(ctypes.byref(h), None, 0, 10, None, 0, None, None) == gr.GR_EINVAL
    assert "NULL" in gr.gr_last_error()
    assert lib.gr_layout_create(ctypes.byref(h), None, 7, 0, None, 0, None, None) == gr.GR_ENOTSUP
    assert lib.gr_evaluate(None, 15, None, None) == gr.GR_EINVAL
    assert lib.gr_layout_destroy(None) == gr.GR_OK
    out = gr.gr_crossing_angle_result()
    assert lib.gr_crossing_angle_noalloc(None, 0, None, gr.GR_NOALLOC_MAX_EDGES + 1, 0.0,
                                         ctypes.byref(out), None) == gr.GR_EINVAL
    assert "limit" in gr.gr_last_error()
    assert gr.gr_version().startswith("gr ")
    assert gr.gr_kernel_launches() == 0  # nothing launched in a process without a GPU call


def test_partial_struct_is_seventeen_int64(tmp_path):
    src = tmp_path / "partial.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gr.h"
int main(void) { printf("%zu %zu\\n", sizeof(gr_partial), offsetof(gr_partial, M_l_bits)); return 0; }
""")
    exe = tmp_path / "partial"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include", str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [17 * 8, 16 * 8] == [ctypes.sizeof(gr.gr_partial), gr.gr_partial.M_l_bits.offset]
