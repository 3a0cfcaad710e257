"""Benchmark: exact readability metrics of one synthetic layout per step on GB300.

One step = one pass of the whole hot path over one layout: gather + validation
of the inputs (gr_layout_update), then all five metrics (gr_evaluate: edge
length variation, minimum angle, occlusion binning + pairs, crossing binning +
scatter + pair kernel, final reduction).  The default workload is the large
sparse layout (200,000 vertices from a 64-component Gaussian mixture, 500,000
edges: rank 1-5 nearest-neighbour edges plus 1 % uniform long edges, d = 64,
ideal angle 70 deg).

metric  edge-pair tests/s, resolved: |E| (|E| - 1) / 2 pairs per step (the
        all-pairs-equivalent rate, which credits the pairs the grid never
        has to test); `issued_pairs_per_s` reports the pairs actually tested.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the layout's stream, with a 256 MiB L2 flush between steps (outside the
events; the inputs are smaller than L2).  Barrier + synchronize around the
timed region; the max over ranks is reported.  With --gpus N > 1 (torchrun),
every rank evaluates its own replica of the layout (no collective on the data
path; weak scaling).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

IDEAL = 7.0 * math.pi / 18.0
L2_FLUSH_BYTES = 256 << 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")

LONG_PAIRS = {"auto": 0, "allpairs": 1, "grid": 2}

WORKLOADS = {
    "large_sparse": ("large_sparse_layout", 64),
    "dense_long_edge": ("dense_long_edge_layout", 256),
    "plain": ("plain_layout", 256),
    "batched": ("batched_layouts", 256),
    "differentiable": ("differentiable_layout", 0),
    "moves": ("large_sparse_layout", 64),
    "strips": ("dense_long_edge_layout", 0),
    "per_edge": ("large_sparse_layout", 0),
    "paper_sized": ("paper_sized_layout", 256),
}
MOVES_PER_STEP = 16
STRIP_WIDTH = 64          # vertical strips of the approximate algorithm (Sec. 3.2.2)
OPS_PER_STRIP_PAIR = 10   # per counted pair: direction load, wrapped difference, acute fold, |ideal - a|, add
OPS_PER_MERGE_STEP = 6    # per binary-search step of a merge level: load, 64-bit compare, select


def max_over_ranks(values, world: int, device) -> list[float]:
    """The element-wise maximum of per-rank timings over all ranks (one
    all-reduce); the values themselves on a single rank."""
    vals = [float(v) for v in values]
    if world <= 1:
        return vals
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def make_workload(name):
    from paper_2411_09809_gb300 import synth
    fn, d = WORKLOADS[name]
    return getattr(synth, fn)(), d


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # wait for the sampler's first line, so that short timed regions still see a live sampler
        # (the last sample before a region of a few milliseconds is then the one reported)
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- roofline

def load_peaks() -> tuple[dict, str]:
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def load_capture(kernel: str, workload: str, src_hash: str) -> dict:
    """The committed ncu summary's figures for `kernel` (DRAM bytes per launch,
    issue-slot utilisation), or {} if the kernel source changed since the capture."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            t = json.load(f)
    except OSError:
        return {}
    e = t.get(f"{kernel}/{workload}")
    if not e or e.get("source_sha256") != src_hash:
        return {}
    return e


def load_traffic(kernel: str, workload: str, src_hash: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None if
    the kernel source changed since the capture."""
    return load_capture(kernel, workload, src_hash).get("dram_bytes_per_launch")


# The sources each captured kernel is built from: its own file and every
# header it includes, so an edit anywhere in them retires the capture.
KERNEL_SOURCES = {
    "k_cell_pairs": ["k_grid.cu", "grid_common.cuh", "pair_math.cuh", "gr_internal.cuh"],
    "k_grid_pairs": ["k_grid.cu", "grid_common.cuh", "pair_math.cuh", "gr_internal.cuh"],
    "k_grid_fill": ["k_grid.cu", "grid_common.cuh", "pair_math.cuh", "gr_internal.cuh"],
    "k_cross_allpairs_agg": ["k_crossings.cu", "allpairs_common.cuh", "pair_math.cuh", "gr_internal.cuh"],
    "crossing_phase_f32": ["k_diff.cu", "gr_internal.cuh"],
}


def kernel_source_hash(files: list[str]) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2411_09809_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


# Algorithmic work per unit, the figures the roofline divides by time:
#   grid pair kernel (a6): per candidate pair 25 integer ops for the shared-id
#     skip, four orientations and the sign tests; per E_c pair 60 more for the
#     angle (cross/dot, conversion, atan2, fixed-point add) and the owner test.
#   all-pairs kernel (a7): the same per pair, without the owner test (45 more
#     per E_c pair).
#   scatter (a4): per record a 16-byte segment + 4-byte edge id write and per
#     segment a 16 + 4 byte read.
OPS_PER_PAIR = 25
OPS_PER_CROSSING_GRID = 60
OPS_PER_CROSSING_ALLPAIRS = 45
#   FP32 all-pairs kernel of the differentiable form: per pair 4 id compares,
#     four filtered FP32 orientations (differences, two products, the
#     difference, the error bound and its tests: 11 each) and the sign tests;
#     per E_c pair 20 more (the angle term and the pair record).
OPS_PER_PAIR_F32 = 52
OPS_PER_CROSSING_F32 = 20
SM_COUNT = 152
LANES_PER_SM_PER_CLK = 128  # 4 SM sub-partitions x 32 lanes, one warp instruction per clock each


_PIPES = None


def measured_pipes() -> dict | None:
    """Thread-operations per second (T/s) of the instruction classes the pair
    kernels use, measured on this GPU by the pipe microbenchmarks
    (paper_2411_09809_gb300/peaks/pipe_peaks.cu); cached per process."""
    global _PIPES
    if _PIPES is None:
        import ctypes
        try:
            from paper_2411_09809_gb300 import build as gb
            lib = ctypes.CDLL(gb.build_peaks())
            out = (ctypes.c_double * 7)()
            n = lib.gr_peaks_measure(out, 7)
            names = ["iadd3", "lop3", "imnmx_plus_iadd", "imad", "ffma", "mufu_rsqrt", "dfma"]
            _PIPES = {names[i]: round(out[i] / 1e12, 3) for i in range(n)} if n > 0 else {}
        except (OSError, RuntimeError):
            _PIPES = {}
    return _PIPES or None


def roofline(res, prof: dict, n_seg: int, peaks: dict, peak_kind: str, workload: str) -> dict:
    pairs_ms, pairs_calls = prof["cross_pairs"]
    scat_ms, scat_calls = prof["cross_scatter"]
    grid = res.crossing_path == 1
    ec = res.crossing.c.crossings
    if pairs_calls and (not scat_calls or pairs_ms >= scat_ms):
        t = pairs_ms / pairs_calls / 1e3
        pairs = res.crossing.c.pairs_tested
        ops = pairs * OPS_PER_PAIR + ec * (OPS_PER_CROSSING_GRID if grid else OPS_PER_CROSSING_ALLPAIRS)
        peak = SM_COUNT * LANES_PER_SM_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        # the grid path runs the rotation kernel unless the planner sends pairs of two long
        # segments to the all-pairs tiles (then the tile kernel k_grid_pairs); the bench
        # workloads keep them in the grid
        kernel = "k_cell_pairs" if grid else "k_cross_allpairs_agg"
        achieved = ops / t / 1e12
        cap = load_capture(kernel, workload, kernel_source_hash(KERNEL_SOURCES[kernel]))
        return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tops/s (int32-equivalent lane ops)", "frac": achieved / peak,
                "peak_source": f"{SM_COUNT} SMs x {LANES_PER_SM_PER_CLK} lanes x "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_kind} max clock)",
                "traffic": cap.get("dram_bytes_per_launch"),
                # issued instructions against the issue-rate peak (smsp__issue_active, ncu), the
                # pair kernels' target measure; null once the kernel changed since the capture
                "issue_slot_frac": cap.get("issue_active_frac"),
                "launch_ms": t * 1e3}
    t = scat_ms / scat_calls / 1e3
    nbytes = res.grid_records * 20 + n_seg * 20
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = nbytes / t / 1e9
    return {"kernel": "k_grid_fill", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"hbm_gbs ({peak_kind})",
            "traffic": load_traffic("k_grid_fill", workload, kernel_source_hash(KERNEL_SOURCES["k_grid_fill"])),
            "launch_ms": t * 1e3}


# ------------------------------------------------------------- CPU baseline

def cpu_oracle_diff_step(L, budget_s: float) -> dict:
    """Times the oracle's FP32 forward + FP64 gradients on the first E_s edges of
    the layout (all vertices), E_s sized to about budget_s seconds, and scales the
    time by the number of edge pairs to the full edge list."""
    import oracle
    E = L.E
    Es = max(256, E // 32)
    t0 = time.perf_counter()
    oracle.diff_terms_and_grads(L.xy, L.edges[:Es])
    t = time.perf_counter() - t0
    Es2 = int(min(E, Es * math.sqrt(max(1.0, budget_s / max(t, 1e-3)))))
    t0 = time.perf_counter()
    oracle.diff_terms_and_grads(L.xy, L.edges[:Es2])
    t2 = time.perf_counter() - t0
    step_s = t2 * (E * (E - 1)) / max(1, Es2 * (Es2 - 1))
    return {"step_s": step_s, "cores": oracle.num_threads(),
            "sample": f"terms and FP64 gradients of the first {Es2} of {E} edges (all {L.V} vertices, "
                      f"{Es2 * (Es2 - 1) / 2:.3g} edge pairs, {t2:.1f} s), scaled by edge pairs to one full "
                      f"step ({step_s:.1f} s)"}


def cpu_oracle_step(L, d, budget_s: float, rng_seed: int = 0, crossings_only: bool = False) -> dict:
    """Times the oracle on a bounded sample of one step and scales it to the full
    step: crossings of S sampled edges against all edges, occlusion on the first
    V_s vertices, minimum angle and edge length variation in full."""
    import numpy as np

    import oracle
    E, V = L.E, L.V
    rng = np.random.default_rng(rng_seed)
    t0 = time.perf_counter()
    if not crossings_only:
        oracle.edge_length_variation(L.xy, L.edges)
        oracle.min_angle(L.xy, L.edges)
    t_lin = time.perf_counter() - t0
    # calibrate crossings on growing samples, then take one of ~budget/2 seconds
    S, t_small = 16, 0.0
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.crossings_of_edges(L.xy, L.edges, rng.choice(E, size=S, replace=False))
        t_small = time.perf_counter() - t0
        if t_small > 0.5 or S >= E:
            break
        S = int(min(E, S * 1.0 / max(t_small, 1e-4)))
    S2 = int(max(16, min(E, S * (0.5 * budget_s) / max(t_small, 1e-6))))
    sample = rng.choice(E, size=S2, replace=False)
    t0 = time.perf_counter()
    oracle.crossings_of_edges(L.xy, L.edges, sample)
    t_cross = time.perf_counter() - t0
    cross_full = t_cross * (E * (E - 1) / 2) / (S2 * (E - 1))
    Vs = 0 if crossings_only else min(V, 20000)
    t0 = time.perf_counter()
    if Vs:
        oracle.node_occlusion(L.xy[:Vs], d)
    t_occ = time.perf_counter() - t0
    occ_full = t_occ * (V * (V - 1) / 2) / max(1, Vs * (Vs - 1) / 2) if Vs else 0.0
    step_s = cross_full + occ_full + t_lin
    if crossings_only:
        return {"step_s": step_s, "cores": oracle.num_threads(),
                "sample": f"per-edge crossings (oracle.crossings_of_edges) of {S2} sampled edges against all "
                          f"{E} edges ({S2 * (E - 1):.3g} pair tests, {t_cross:.1f} s), scaled to all edges "
                          f"({step_s:.1f} s)",
                "measured_s": t_small + t_cross}
    return {"step_s": step_s, "cores": oracle.num_threads(),
            "sample": f"crossings of {S2} sampled edges against all {E} edges "
                      f"({S2 * (E - 1):.3g} pair tests, {t_cross:.1f} s), occlusion of the first {Vs} "
                      f"vertices ({t_occ:.1f} s), minimum angle and edge length variation in full "
                      f"({t_lin:.2f} s); scaled to one full step ({step_s:.1f} s)",
            "measured_s": t_lin + t_small + t_cross + t_occ}


def batched_workload():
    """The 4,096-layout batch, packed; cached in the temp directory (generation
    takes about a minute)."""
    import tempfile

    import numpy as np

    from paper_2411_09809_gb300 import synth
    path = os.path.join(tempfile.gettempdir(), f"gr_batched_{synth.BASE_SEED + 3}_v2.npz")
    if os.path.exists(path):
        z = np.load(path)
        return z["v_off"], z["e_off"], z["xy"], z["edges"]
    v_off, e_off, xy, edges = synth.pack_layouts(synth.batched_layouts())
    tmp = path + f".{os.getpid()}.npz"
    np.savez(tmp, v_off=v_off, e_off=e_off, xy=xy, edges=edges)
    os.replace(tmp, path)
    return v_off, e_off, xy, edges


def run_batched(args, rank, world, local_rank):
    """Batched workload: one step = gr_batch_update + gr_batch_evaluate (all five
    metrics of every layout, one CUDA-graph replay).  Reported beside the same
    layouts evaluated one by one through the single-layout entry points."""
    import torch
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build as gr_build, gr

    torch.cuda.set_device(local_rank)
    if world > 1:
        if rank == 0:
            gr_build.build()
        dist.barrier()
    else:
        gr_build.build()
    gr.load()
    v_off, e_off, xy, edges = batched_workload()
    n = len(v_off) - 1
    d = WORKLOADS["batched"][1]
    dev = torch.device("cuda", local_rank)
    dxy = torch.from_numpy(xy).to(dev)
    ded = torch.from_numpy(edges).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    B = gr.Batch(v_off, e_off, dxy, ded, gr.gr_options(0, 0, 0, 0, LONG_PAIRS[args.long_pairs]),
                 stream=stream.cuda_stream)
    create_s = time.perf_counter() - t0

    def step():
        B.update(dxy)
        return B.evaluate(gr.GR_METRIC_ALL, IDEAL, d)

    for _ in range(args.warmup):
        res = step()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = gr.gr_kernel_launches()
    for i in range(args.steps):
        flush.fill_(i)
        starts[i].record(stream)
        res = step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    launches = gr.gr_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))
    (ms,) = max_over_ranks([ms], world, dev)
    # the same layouts one by one (a fixed sample, scaled to the batch)
    sample = [] if args.no_single_loop else list(range(0, n, max(1, n // 256)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        with gr.Layout(dxy[v_off[i]:v_off[i + 1]], ded[e_off[i]:e_off[i + 1]]) as one:
            one.evaluate(gr.GR_METRIC_ALL, IDEAL, d)
    single_s = (time.perf_counter() - t0) * n / max(1, len(sample))
    # end to end through the C ABI: coordinates and edges from pinned host memory, results to the host
    hxy = torch.from_numpy(xy).pin_memory()
    hed = torch.from_numpy(edges).pin_memory()
    e2e_s = []
    for i in range(0 if args.no_e2e else args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr.gr_batch_update(B.handle, hxy, hed)
        gr.gr_batch_evaluate(B.handle, n, gr.GR_METRIC_ALL, IDEAL, d)
        e2e_s.append(time.perf_counter() - t0)
    e2e_ms = statistics.mean(e2e_s) * 1e3 if e2e_s else float("nan")
    tuned_offset, tuned_tile = gr.gr_batch_tuning(B.handle)
    B.close()
    if rank != 0:
        return
    pairs = float(sum((e_off[i + 1] - e_off[i]) * (e_off[i + 1] - e_off[i] - 1) / 2 for i in range(n)))
    value = world * n / (ms / 1e3)
    # roofline over the whole step: the pair tests of every layout (grid candidates and long-long
    # tile pairs) and their crossings, against the issue-rate peak
    peaks, peak_kind = load_peaks()
    tested = float(sum(r.crossing.c.pairs_tested for r in res))
    crossings = float(sum(r.crossing.c.crossings for r in res))
    ops = tested * OPS_PER_PAIR + crossings * OPS_PER_CROSSING_GRID
    peak = SM_COUNT * LANES_PER_SM_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = ops / (ms / 1e3) / 1e12
    line = {
        "metric": "layouts/s", "value": value, "unit": "layouts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batched_{n}_layouts", "layouts": n, "V": int(v_off[-1]), "E": int(e_off[-1]),
                   "occlusion_d": d, "ideal_deg": 70.0,
                   "metrics": "all five per layout", "inputs": "seeded synthetic (paper_2411_09809_gb300.synth)",
                   "l2": "256 MiB write between timed steps",
                   "autotuned": {"cell_offset": tuned_offset, "tile": tuned_tile},
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "resolved_pairs_per_s": world * pairs / (ms / 1e3),
        "single_layout_loop": {"layouts_per_s": n / single_s, "sample_layouts": len(sample),
                               "speedup_of_batch": (n / (ms / 1e3)) / (n / single_s)} if sample else None,
        "create_s": create_s,
        "roofline": {"kernel": "the whole step (k_batch_long_pairs and k_batch_grid_pairs take three quarters)",
                     "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (int32-equivalent lane ops)", "frac": achieved / peak,
                     "peak_source": f"{SM_COUNT} SMs x {LANES_PER_SM_PER_CLK} lanes x "
                                    f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_kind} max clock)",
                     "work": f"{OPS_PER_PAIR} ops per pair tested, {OPS_PER_CROSSING_GRID} per crossing",
                     "traffic": None, "pipe_peaks_tops": measured_pipes()},
        "e2e": {"value": world * n / (e2e_ms / 1e3), "unit": "layouts/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(xy.nbytes + edges.nbytes),
                "d2h_bytes_per_step": n * ctypes.sizeof(gr.gr_result)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb_s, n_sample = batch_oracle_step(v_off, e_off, xy, edges, d)
        import oracle
        line["cpu_baseline"] = {"value": n / cb_s, "unit": "layouts/s", "cores": oracle.num_threads(),
                                "kind": "oracle",
                                "sample": f"{n_sample} layouts stratified by size, all five metrics, scaled to {n}"}
    return line


def batch_oracle_step(v_off, e_off, xy, edges, d) -> tuple[float, int]:
    """The oracle's time for all five metrics of a size-stratified sample of the
    layouts (every 64th by size), scaled to the whole batch; and the sample size."""
    import oracle
    n = len(v_off) - 1
    order = sorted(range(n), key=lambda i: v_off[i + 1] - v_off[i])
    sample = order[:: max(1, n // 64)]
    t0 = time.perf_counter()
    for i in sample:
        lxy = xy[v_off[i]:v_off[i + 1]]
        led = edges[e_off[i]:e_off[i + 1]]
        oracle.crossings(lxy, led)
        oracle.node_occlusion(lxy, d)
        oracle.min_angle(lxy, led)
        oracle.edge_length_variation(lxy, led)
    return (time.perf_counter() - t0) * n / len(sample), len(sample)


def run_reference_batched(args):
    """Reference arm of the batched workload: the oracle evaluates all five
    metrics of a size-stratified sample of the layouts, scaled to the batch."""
    import oracle
    v_off, e_off, xy, edges = batched_workload()
    n = len(v_off) - 1
    d = WORKLOADS["batched"][1]
    secs = []
    for _ in range(args.warmup + args.steps):
        t, n_sample = batch_oracle_step(v_off, e_off, xy, edges, d)
        secs.append(t)
    sample = range(n_sample)
    step_s = statistics.mean(secs[args.warmup:])
    value = n / step_s
    line = {
        "impl": "reference", "metric": "layouts/s", "value": value, "unit": "layouts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batched_{n}_layouts", "layouts": n, "occlusion_d": d},
        "cpu_baseline": {"value": value, "unit": "layouts/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{len(sample)} layouts stratified by size, all five metrics, scaled to {n}"},
        "e2e": {"value": value, "unit": "layouts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_differentiable(args):
    """Reference arm of the differentiable workload: the oracle's FP32 forward and
    FP64 gradients on a bounded edge sample per step, scaled to the full layout."""
    L, _ = make_workload("differentiable")
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_diff_step(L, budget / 4)
    steps = [cpu_oracle_diff_step(L, budget) for _ in range(args.steps)]
    step_s = statistics.mean(s["step_s"] for s in steps)
    value = 1.0 / step_s
    line = {
        "impl": "reference", "metric": "fwd+bwd steps/s", "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": diff_config(L),
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": steps[0]["cores"], "kind": "oracle",
                         "sample": steps[0]["sample"]},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def diff_config(L):
    return {"workload": L.name, "V": L.V, "E": L.E, "ideal_deg": 70.0,
            "step": "gr_layout_update + gr_diff_forward (E_ca, M_l, M_a) + gr_diff_backward (d/dxy)",
            "inputs": "seeded synthetic (paper_2411_09809_gb300.synth), FP32 coordinates in [0, 1)^2",
            "l2": "256 MiB write between timed steps (inputs are smaller than L2)"}


def run_differentiable(args, rank, world, local_rank):
    """Differentiable workload: one step = gr_layout_update + gr_diff_forward +
    gr_diff_backward (the gradient of (1 - E_ca) + M_l + (1 - M_a)).  The plain
    forward (update + gr_diff_forward) is timed beside it."""
    import torch
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build as gr_build, gr

    torch.cuda.set_device(local_rank)
    if world > 1:
        if rank == 0:
            gr_build.build()
        dist.barrier()
    else:
        gr_build.build()
    gr.load()
    L, _ = make_workload("differentiable")
    dev = torch.device("cuda", local_rank)
    xy = torch.from_numpy(L.xy).to(dev)
    edges = torch.from_numpy(L.edges).to(dev)
    out3 = torch.empty(3, dtype=torch.float32, device=dev)
    gout = torch.tensor([-1.0, 1.0, -1.0], dtype=torch.float32, device=dev)
    grad = torch.empty_like(xy)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lay = gr.Layout(xy, edges, gr.gr_options(0, 0, 0, 1), stream=stream.cuda_stream, coord_type=gr.GR_COORD_F32)

    def fwd():
        lay.update(xy)
        gr.gr_diff_forward(lay.handle, IDEAL, out3)

    def fwd_bwd():
        fwd()
        gr.gr_diff_backward(lay.handle, gout, grad)

    def timed(fn, n):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for i in range(n):
            flush.fill_(i)
            starts[i].record(stream)
            fn()
            ends[i].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))

    for _ in range(args.warmup):
        fwd_bwd()
    lay.profile(reset=True)
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = gr.gr_kernel_launches()
    ms = timed(fwd_bwd, args.steps)
    launches = gr.gr_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = lay.profile()
    fwd_ms = timed(fwd, args.steps)
    ms, fwd_ms = max_over_ranks([ms, fwd_ms], world, dev)
    res = lay.evaluate(gr.GR_METRIC_CROSSINGS, IDEAL)

    # end to end through the C ABI with host buffers (pinned): coordinates in,
    # the three terms out, the upstream gradient in; the gradient stays on the device
    hxy = torch.from_numpy(L.xy).pin_memory()
    hout = torch.empty(3, dtype=torch.float32).pin_memory()
    hg = torch.tensor([-1.0, 1.0, -1.0], dtype=torch.float32).pin_memory()
    io0 = gr.gr_io_bytes(lay.handle)
    e2e_s = []
    for i in range(0 if args.no_e2e else args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr.gr_layout_update(lay.handle, hxy, None, gr.GR_COORD_F32)
        gr.gr_diff_forward(lay.handle, IDEAL, hout)
        gr.gr_diff_backward(lay.handle, hg, grad)
        e2e_s.append(time.perf_counter() - t0)
    io1 = gr.gr_io_bytes(lay.handle)
    e2e_ms = statistics.mean(e2e_s) * 1e3 if e2e_s else float("nan")
    lay.close()
    if rank != 0:
        return
    E = L.E
    pairs_ms, pairs_calls = prof["cross_pairs"]
    t = pairs_ms / max(1, pairs_calls) / 1e3
    ec = res.crossing.c.crossings
    grid = res.crossing_path == 1
    # pair tests actually made: the grid's candidate pairs plus the long-long tiles
    ops = res.crossing.c.pairs_tested * OPS_PER_PAIR_F32 + ec * OPS_PER_CROSSING_F32
    peaks, peak_kind = load_peaks()
    peak = SM_COUNT * LANES_PER_SM_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    kernel = "crossing phase: k_f32_grid_ss + k_f32_grid_ls + k_cross_f32 (long x long)" if grid else "k_cross_f32"
    rf = {"kernel": kernel, "bound": "alu", "achieved": ops / t / 1e12 if t > 0 else None, "peak": peak,
          "unit": "Tops/s (int32-equivalent lane ops)", "frac": ops / t / 1e12 / peak if t > 0 else None,
          "peak_source": f"{SM_COUNT} SMs x {LANES_PER_SM_PER_CLK} lanes x "
                         f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_kind} max clock)",
          "traffic": load_traffic("crossing_phase_f32" if grid else "k_cross_f32", "differentiable",
                                  kernel_source_hash(KERNEL_SOURCES["crossing_phase_f32"])),
          "launch_ms": t * 1e3, "pairs_tested": res.crossing.c.pairs_tested}
    line = {
        "metric": "fwd+bwd steps/s", "value": world * 1e3 / ms, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(diff_config(L), parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "fwd_ms": fwd_ms, "fwd_bwd_ms": ms, "fwd_bwd_over_fwd": ms / fwd_ms,
        "results": {"E_ca": float(out3[0]), "M_l": float(out3[1]), "M_a": float(out3[2]), "E_c": ec},
        "crossing_path": {1: "grid", 2: "all-pairs"}.get(res.crossing_path, "none"),
        "phase_ms": {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]},
        "roofline": rf,
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "steps/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": (io1[0] - io0[0]) // max(1, len(e2e_s)),
                "d2h_bytes_per_step": (io1[1] - io0[1]) // max(1, len(e2e_s))},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_diff_step(L, args.cpu_budget)
        line["cpu_baseline"] = {"value": 1.0 / cb["step_s"], "unit": "steps/s", "cores": cb["cores"],
                                "kind": "oracle", "sample": cb["sample"]}
    return line


def move_roofline(L, ms: float) -> dict:
    """A move against HBM: its algorithmic bytes are dominated by the O(E) passes (the regather:
    8 B of ids, 16 B of coordinates, 16 + 4 + 4 B of segment, id and direction, 8 B of squared length
    per edge, and 8 B of coordinates per vertex for the range check; the edge length variation: the
    squared length read, the length written and read back, 3 x 8 B per edge; the affected-edge scan:
    8 B of ids and 8 B of moved flags per edge).  The step is latency-bound: the fraction is small by
    construction."""
    peaks, peak_kind = load_peaks()
    nbytes = L.E * (56 + 24 + 16) + L.V * 8
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = nbytes / (ms / 1e3) / 1e9
    return {"kernel": "the whole move (the O(E) regather, edge length variation and affected-edge scan)",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": f"hbm_gbs ({peak_kind})", "work": "96 B per edge + 8 B per vertex",
            "traffic": None}


def run_moves(args, rank, world, local_rank):
    """Incremental workload: on the large sparse layout, one step = gr_move_vertices
    of 16 random vertices to random positions (all five metrics of the moved
    layout, the crossing and occlusion counts updated from the previous
    evaluation).  A full evaluation of the same layout is timed beside it."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build as gr_build, gr

    torch.cuda.set_device(local_rank)
    if world > 1:
        if rank == 0:
            gr_build.build()
        dist.barrier()
    else:
        gr_build.build()
    gr.load()
    L, d = make_workload("moves")
    dev = torch.device("cuda", local_rank)
    xy = torch.from_numpy(L.xy).to(dev)
    edges = torch.from_numpy(L.edges).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lay = gr.Layout(xy, edges, stream=stream.cuda_stream)
    rng = np.random.default_rng(20241115 + 5)
    n_steps = args.warmup + 2 * args.steps
    ids = [torch.from_numpy(rng.choice(L.V, size=MOVES_PER_STEP, replace=False).astype(np.int32)).to(dev)
           for _ in range(n_steps)]
    new = [torch.from_numpy(rng.integers(0, 65536, size=(MOVES_PER_STEP, 2)).astype(np.int32)).to(dev)
           for _ in range(n_steps)]
    res = lay.evaluate(gr.GR_METRIC_ALL, IDEAL, d)

    def timed(fn, k, off):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        out = None
        for i in range(k):
            flush.fill_(i)
            starts[i].record(stream)
            out = fn(off + i)
            ends[i].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends)), out

    move = lambda i: lay.move(ids[i], new[i], gr.GR_METRIC_ALL, IDEAL, d)
    timed(move, args.warmup, 0)
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = gr.gr_kernel_launches()
    ms, res = timed(move, args.steps, args.warmup)
    launches = gr.gr_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    full_ms, _ = timed(lambda i: lay.evaluate(gr.GR_METRIC_ALL, IDEAL, d), args.steps, 0)
    # end to end through the C ABI: the moved ids and coordinates from pinned host memory, the result
    # read back (gr_move_vertices returns it on the host)
    h_ids = [ids[i].cpu().pin_memory() for i in range(args.warmup, args.warmup + args.steps)]
    h_new = [new[i].cpu().pin_memory() for i in range(args.warmup, args.warmup + args.steps)]
    io0 = gr.gr_io_bytes(lay.handle)
    e2e_s = []
    for i in range(args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr.gr_move_vertices(lay.handle, h_ids[i], h_new[i], gr.GR_METRIC_ALL, IDEAL, d)
        e2e_s.append(time.perf_counter() - t0)
    io1 = gr.gr_io_bytes(lay.handle)
    e2e_ms = statistics.mean(e2e_s) * 1e3
    ms, full_ms = max_over_ranks([ms, full_ms], world, dev)
    lay.close()
    if rank != 0:
        return
    line = {
        "metric": "incremental evaluations/s", "value": world * 1e3 / ms, "unit": "evaluations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(workload_config(L, d, "moves"), workload=f"moves_{MOVES_PER_STEP}_of_{L.name}",
                       step=f"gr_move_vertices of {MOVES_PER_STEP} random vertices, all five metrics",
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "full_evaluation_ms": full_ms, "speedup_over_full": full_ms / ms,
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": "evaluations/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": (io1[0] - io0[0]) // args.steps,
                "d2h_bytes_per_step": (io1[1] - io0[1]) // args.steps},
        "roofline": move_roofline(L, ms),
        "pairs_tested_per_step": res.crossing.c.pairs_tested,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_move_steps(L, 3)
        line["cpu_baseline"] = {"value": 1.0 / cb["step_s"], "unit": "evaluations/s", "cores": cb["cores"],
                                "kind": "oracle", "sample": cb["sample"]}
    print(json.dumps(line), flush=True)


def strip_oracle_sample(L, l, budget_s: float, seed: int = 0) -> dict:
    """The strip oracle on the first E' edges, E' grown until one run takes about
    budget_s / 4; the rate in resolved pairs/s (the oracle's work and the metric
    both scale as E'^2)."""
    import oracle
    E = min(L.E, 2000)
    while True:
        t0 = time.perf_counter()
        oracle.strip_crossings(L.xy, L.edges[:E], l, 0)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or E >= L.E:
            break
        E = min(L.E, int(E * max(1.3, min(4.0, math.sqrt(budget_s / 4 / max(dt, 1e-3))))))
    return {"rate": E * (E - 1) / 2 / dt, "step_s": dt, "edges": E, "cores": oracle.num_threads(),
            "sample": f"the strip oracle (vertical strips of width {l}) on the first {E} of {L.E} edges, "
                      f"rate = E'(E'-1)/2 / time (its work grows as E'^2)"}


def run_strips(args, rank, world, local_rank):
    """Approximate-strip workload (Sec. 3.2.2-3.2.3): on the dense long-edge
    layout (random segments, the paper's setting for Table 3), one step =
    gr_strip_crossings with vertical strips of width STRIP_WIDTH (the E_c
    estimate and the crossing-angle estimate).  The exact count is taken once,
    untimed, for the errors."""
    import torch
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build as gr_build, gr

    torch.cuda.set_device(local_rank)
    if world > 1:
        if rank == 0:
            gr_build.build()
        dist.barrier()
    else:
        gr_build.build()
    gr.load()
    L, _ = make_workload("strips")
    l = args.strip_width
    dev = torch.device("cuda", local_rank)
    xy = torch.from_numpy(L.xy).to(dev)
    edges = torch.from_numpy(L.edges).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lay = gr.Layout(xy, edges, gr.gr_options(0, 0, 0, 1, 0), stream=stream.cuda_stream)
    exact = lay.evaluate(gr.GR_METRIC_CROSSINGS, IDEAL, 0).crossing

    def step():
        lay.update(xy)
        return lay.strips(l, gr.GR_STRIP_VERTICAL, IDEAL)

    for _ in range(args.warmup):
        res = step()
    lay.profile(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = gr.gr_kernel_launches()
    for i in range(args.steps):
        flush.fill_(i)
        starts[i].record(stream)
        res = step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    launches = gr.gr_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))
    (ms,) = max_over_ranks([ms], world, dev)
    prof = lay.profile()
    # end to end through the C ABI from pinned host coordinates
    hxy = torch.from_numpy(L.xy).pin_memory()
    io0 = gr.gr_io_bytes(lay.handle)
    e2e_s = []
    for i in range(0 if args.no_e2e else args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr.gr_layout_update(lay.handle, hxy, None)
        gr.gr_strip_crossings(lay.handle, l, gr.GR_STRIP_VERTICAL, IDEAL)
        e2e_s.append(time.perf_counter() - t0)
    io1 = gr.gr_io_bytes(lay.handle)
    e2e_ms = statistics.mean(e2e_s) * 1e3 if e2e_s else float("nan")
    lay.close()
    if rank != 0:
        return
    E = L.E
    pairs = E * (E - 1) / 2
    # roofline of the counting phase (merge by r with the inverted pairs)
    peaks, peak_kind = load_peaks()
    R = res.records
    levels = max(1, math.ceil(math.log2(max(2, R / max(1, res.strips)))))
    merge_ops = R * sum(OPS_PER_MERGE_STEP * (k + 2) for k in range(levels))
    count_ops = merge_ops + res.crossings * OPS_PER_STRIP_PAIR
    cnt_ms = prof["strip_count"][0] / max(1, prof["strip_count"][1])
    peak = SM_COUNT * LANES_PER_SM_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = count_ops / (cnt_ms / 1e3) / 1e12
    line = {
        "metric": "edge-pair tests/s", "value": world * pairs / (ms / 1e3), "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"strips_{l}_of_{L.name}", "V": L.V, "E": E, "strip_width": l,
                   "orientation": "vertical", "ideal_deg": 70.0,
                   "step": "gr_layout_update + gr_strip_crossings (E_c and E_ca estimates, Sec. 3.2.2-3.2.3)",
                   "inputs": "seeded synthetic (paper_2411_09809_gb300.synth)",
                   "l2": "256 MiB write between timed steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "results": {"E_c_estimate": res.crossings, "E_c_exact": exact.c.crossings,
                    "E_c_error": 1.0 - res.crossings / max(1, exact.c.crossings),
                    "E_ca_estimate": res.E_ca, "E_ca_exact": exact.E_ca,
                    "E_ca_error": abs(res.E_ca - exact.E_ca) / exact.E_ca,
                    "records": R, "strips": res.strips},
        "phase_ms": {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]},
        "roofline": {"kernel": "k_strip_tile<true> + k_strip_level<true> (the counting phase)", "bound": "alu",
                     "achieved": achieved, "peak": peak, "unit": "Tops/s (int32-equivalent lane ops)",
                     "frac": achieved / peak,
                     "peak_source": f"{SM_COUNT} SMs x {LANES_PER_SM_PER_CLK} lanes x "
                                    f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_kind} max clock)",
                     "work": f"{OPS_PER_MERGE_STEP} ops per binary-search step of each merge level and record, "
                             f"{OPS_PER_STRIP_PAIR} per counted pair",
                     "traffic": None, "launch_ms": cnt_ms, "pipe_peaks_tops": measured_pipes()},
        "e2e": {"value": world * pairs / (e2e_ms / 1e3), "unit": "pairs/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": (io1[0] - io0[0]) // max(1, len(e2e_s)),
                "d2h_bytes_per_step": (io1[1] - io0[1]) // max(1, len(e2e_s))},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = strip_oracle_sample(L, l, args.cpu_budget)
        line["cpu_baseline"] = {"value": cb["rate"], "unit": "pairs/s", "cores": cb["cores"], "kind": "oracle",
                                "sample": cb["sample"]}
    print(json.dumps(line), flush=True)


def run_per_edge(args, rank, world, local_rank):
    """Per-edge workload (the per-segment quantities of Sec. 3.2.3 / Eq. 1, NEXT-2):
    on the large sparse layout, one step = gr_layout_update + gr_crossings_per_edge
    (every edge's proper, touching and collinear counts and its sum of
    |ideal - a_c|, into device arrays).  The crossing-only evaluation of the same
    layout is timed beside it."""
    import torch
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build as gr_build, gr

    torch.cuda.set_device(local_rank)
    if world > 1:
        if rank == 0:
            gr_build.build()
        dist.barrier()
    else:
        gr_build.build()
    gr.load()
    L, _ = make_workload("per_edge")
    dev = torch.device("cuda", local_rank)
    xy = torch.from_numpy(L.xy).to(dev)
    edges = torch.from_numpy(L.edges).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lay = gr.Layout(xy, edges, gr.gr_options(0, 0, 0, 1, 0), stream=stream.cuda_stream)
    counts = torch.zeros((L.E, 3), dtype=torch.int64, device=dev)
    devsum = torch.zeros(L.E, dtype=torch.float64, device=dev)
    res = lay.evaluate(gr.GR_METRIC_CROSSINGS, IDEAL, 0)

    def timed(fn, k):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for i in range(k):
            flush.fill_(i)
            starts[i].record(stream)
            fn()
            ends[i].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends))

    def step():
        lay.update(xy)
        gr.gr_crossings_per_edge(lay.handle, IDEAL, counts, devsum)

    timed(step, args.warmup)
    lay.profile(reset=True)
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = gr.gr_kernel_launches()
    ms = timed(step, args.steps)
    launches = gr.gr_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = lay.profile()

    def plain():
        lay.update(xy)
        lay.evaluate(gr.GR_METRIC_CROSSINGS, IDEAL, 0)

    timed(plain, 3)
    plain_ms = timed(plain, args.steps)
    ms, plain_ms = max_over_ranks([ms, plain_ms], world, dev)
    # end to end: coordinates from pinned host memory, the per-edge arrays read back
    hxy = torch.from_numpy(L.xy).pin_memory()
    hc = torch.empty((L.E, 3), dtype=torch.int64).pin_memory()
    hd = torch.empty(L.E, dtype=torch.float64).pin_memory()
    e2e_s = []
    for i in range(0 if args.no_e2e else args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr.gr_layout_update(lay.handle, hxy, None)
        gr.gr_crossings_per_edge(lay.handle, IDEAL, counts, devsum)
        hc.copy_(counts, non_blocking=True)
        hd.copy_(devsum, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s.append(time.perf_counter() - t0)
    e2e_ms = statistics.mean(e2e_s) * 1e3 if e2e_s else float("nan")
    tot = counts.sum(dim=0).tolist()
    lay.close()
    if rank != 0:
        return
    E = L.E
    pairs = E * (E - 1) / 2
    peaks, peak_kind = load_peaks()
    rf = roofline(res, prof, E - res.crossing.c.zero_length_edges, peaks, peak_kind, "per_edge")
    rf["traffic"] = None  # the per-edge form of the kernel has no committed capture
    rf["pipe_peaks_tops"] = measured_pipes()
    rf["kernel"] += " (per-edge form: + 4 atomics per E_c pair)"
    line = {
        "metric": "edge-pair tests/s", "value": world * pairs / (ms / 1e3), "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"per_edge_of_{L.name}", "V": L.V, "E": E, "ideal_deg": 70.0,
                   "step": "gr_layout_update + gr_crossings_per_edge (per-edge counts and angle sums, device arrays)",
                   "inputs": "seeded synthetic (paper_2411_09809_gb300.synth)",
                   "l2": "256 MiB write between timed steps (inputs are smaller than L2)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "crossings_only_evaluation_ms": plain_ms, "per_edge_over_plain": ms / plain_ms,
        "results": {"sum_proper": tot[0] // 2, "sum_touching": tot[1] // 2, "E_c": res.crossing.c.crossings},
        "phase_ms": {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]},
        "roofline": rf,
        "e2e": {"value": world * pairs / (e2e_ms / 1e3), "unit": "pairs/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": L.V * 8, "d2h_bytes_per_step": E * 32},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_step(L, 0, args.cpu_budget, crossings_only=True)
        line["cpu_baseline"] = {"value": pairs / cb["step_s"], "unit": "pairs/s", "cores": cb["cores"],
                                "kind": "oracle", "sample": cb["sample"]}
    print(json.dumps(line), flush=True)


def run_reference_strips(args):
    L, _ = make_workload("strips")
    l = args.strip_width
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        strip_oracle_sample(L, l, budget / 2)
    runs = [strip_oracle_sample(L, l, budget) for _ in range(args.steps)]
    rate = statistics.mean(r["rate"] for r in runs)
    E = L.E
    line = {
        "impl": "reference", "metric": "edge-pair tests/s", "value": rate, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": E * (E - 1) / 2 / rate * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"strips_{l}_of_{L.name}", "V": L.V, "E": E, "strip_width": l,
                   "orientation": "vertical", "ideal_deg": 70.0},
        "cpu_baseline": {"value": rate, "unit": "pairs/s", "cores": runs[0]["cores"], "kind": "oracle",
                         "sample": runs[0]["sample"]},
        "e2e": {"value": rate, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_move_steps(L, n: int, warmup: int = 1) -> dict:
    """The oracle's form of a move, timed n times: the crossings of the
    affected edges (a moved endpoint) against all edges before and after the
    move, plus the minimum angle and edge length variation in full
    (occlusion left out)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(20241115 + 5)
    xy = L.xy.copy()

    def one():
        ids = rng.choice(L.V, size=MOVES_PER_STEP, replace=False)
        aff = np.nonzero(np.isin(L.edges[:, 0], ids) | np.isin(L.edges[:, 1], ids))[0]
        t0 = time.perf_counter()
        oracle.crossings_of_edges(xy, L.edges, aff)
        xy[ids] = rng.integers(0, 65536, size=(len(ids), 2)).astype(np.int32)
        oracle.crossings_of_edges(xy, L.edges, aff)
        oracle.min_angle(xy, L.edges)
        oracle.edge_length_variation(xy, L.edges)
        return time.perf_counter() - t0, len(aff)

    for _ in range(warmup):
        one()
    runs = [one() for _ in range(n)]
    return {"step_s": statistics.mean(r[0] for r in runs), "cores": oracle.num_threads(),
            "sample": f"the oracle's incremental form of a move, {n} moves: crossings of the ~{runs[0][1]} "
                      f"affected edges against all {L.E} edges before and after, minimum angle and edge "
                      f"length variation in full (occlusion left out)"}


def run_reference_moves(args):
    L, d = make_workload("moves")
    cb = oracle_move_steps(L, args.steps, args.warmup)
    step_s = cb["step_s"]
    line = {
        "impl": "reference", "metric": "incremental evaluations/s", "value": 1.0 / step_s, "unit": "evaluations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(workload_config(L, d, "moves"), workload=f"moves_{MOVES_PER_STEP}_of_{L.name}"),
        "cpu_baseline": {"value": 1.0 / step_s, "unit": "evaluations/s", "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"]},
        "e2e": {"value": 1.0 / step_s, "unit": "evaluations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle (plain C brute force) on the host cores."""
    if rank != 0:
        return
    if args.workload == "batched":
        run_reference_batched(args)
        return
    if args.workload == "differentiable":
        run_reference_differentiable(args)
        return
    if args.workload == "strips":
        run_reference_strips(args)
        return
    if args.workload == "moves":
        run_reference_moves(args)
        return
    L, d = make_workload(args.workload)
    E = L.E
    pairs = E * (E - 1) / 2
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    xo = args.workload == "per_edge"  # the per-edge crossing tallies only
    for _ in range(args.warmup):
        cpu_oracle_step(L, d, budget / 4, crossings_only=xo)
    steps = [cpu_oracle_step(L, d, budget, rng_seed=i + 1, crossings_only=xo) for i in range(args.steps)]
    step_s = statistics.mean(s["step_s"] for s in steps)
    value = pairs / step_s
    line = {
        "impl": "reference", "metric": "edge-pair tests/s", "value": value, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": workload_config(L, d, args.workload),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": steps[0]["cores"], "kind": "oracle",
                         "sample": steps[0]["sample"]},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        # ms_per_step is a full step scaled from the sample; this is the oracle time each step ran
        "measured_s_per_step": statistics.mean(s["measured_s"] for s in steps),
    }
    print(json.dumps(line), flush=True)


def workload_config(L, d, name):
    return {"workload": L.name, "V": L.V, "E": L.E, "occlusion_d": d, "ideal_deg": 70.0,
            "metrics": "all five (crossings, crossing angle, occlusion, minimum angle, edge length variation)",
            "inputs": "seeded synthetic (paper_2411_09809_gb300.synth)",
            "l2": "256 MiB write between timed steps (inputs are smaller than L2)"}


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2411_09809_gb300 import build as gr_build, gr

    torch.cuda.set_device(local_rank)
    if world > 1:
        if rank == 0:
            gr_build.build()
        dist.barrier()
    else:
        gr_build.build()
    gr.load()
    L, d = make_workload(args.workload)
    dev = torch.device("cuda", local_rank)
    xy = torch.from_numpy(L.xy).to(dev)
    edges = torch.from_numpy(L.edges).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lay = gr.Layout(xy, edges, gr.gr_options(0, args.cell_log2, 0, 1, LONG_PAIRS[args.long_pairs]),
                    stream=stream.cuda_stream)

    shard = args.shard and world > 1
    if shard:
        from paper_2411_09809_gb300 import shard as gr_shard

    def step():
        lay.update(xy)
        if shard:  # this rank's part of the one layout, then one all-reduce of the parts' tallies
            return gr_shard.evaluate_sharded(lay, gr.GR_METRIC_ALL, IDEAL, d)
        return lay.evaluate(gr.GR_METRIC_ALL, IDEAL, d)

    for _ in range(args.warmup):
        res = step()
    lay.profile(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = gr.gr_kernel_launches()
    for i in range(args.steps):
        flush.fill_(i)
        starts[i].record(stream)
        res = step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    launches = gr.gr_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = statistics.mean(step_ms)
    (ms,) = max_over_ranks([ms], world, dev)
    prof = lay.profile()

    # end to end through the C ABI with host buffers (pinned), copies inside
    hxy = torch.from_numpy(L.xy).pin_memory()
    hed = torch.from_numpy(L.edges).pin_memory()
    io0 = gr.gr_io_bytes(lay.handle)
    e2e_s = []
    for i in range(0 if args.no_e2e else args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr.gr_layout_update(lay.handle, hxy, hed)
        if shard:
            gr_shard.evaluate_sharded(lay, gr.GR_METRIC_ALL, IDEAL, d)
        else:
            gr.gr_evaluate(lay.handle, gr.GR_METRIC_ALL, IDEAL, d)
        e2e_s.append(time.perf_counter() - t0)
    io1 = gr.gr_io_bytes(lay.handle)
    e2e_ms = statistics.mean(e2e_s) * 1e3 if e2e_s else float("nan")
    (e2e_ms,) = max_over_ranks([e2e_ms], world, dev)

    n_seg = L.E - res.crossing.c.zero_length_edges
    peaks, peak_kind = load_peaks()
    rf = roofline(res, prof, n_seg, peaks, peak_kind, args.workload)
    rf["pipe_peaks_tops"] = measured_pipes()
    lay.close()
    if rank != 0:
        return
    E = L.E
    pairs = E * (E - 1) / 2
    copies = 1 if shard else world  # sharded: the ranks share one layout
    value = copies * pairs / (ms / 1e3)
    line = {
        "metric": "edge-pair tests/s", "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(workload_config(L, d, args.workload),
                       parallelism=(f"one layout in {world} parts" if shard else f"replicas x{world}")
                       if world > 1 else "single GPU",
                       crossing_path={1: "grid", 2: "all-pairs"}.get(res.crossing_path, "none"),
                       cell_log2=res.cell_log2, grid_records=res.grid_records,
                       occlusion_path={1: "grid", 2: "all-pairs"}.get(res.occlusion_path, "none")),
        "issued_pairs_per_s": copies * res.crossing.c.pairs_tested / (ms / 1e3),
        "results": {"E_c": res.crossing.c.crossings, "E_ca": res.crossing.E_ca,
                    "N_c": res.occlusion_pairs, "M_a": res.min_angle.M_a, "M_l": res.M_l},
        "phase_ms": {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]},
        "roofline": rf,
        "e2e": {"value": copies * pairs / (e2e_ms / 1e3), "unit": "pairs/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": (io1[0] - io0[0]) // max(1, len(e2e_s)),
                "d2h_bytes_per_step": (io1[1] - io0[1]) // max(1, len(e2e_s))},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_step(L, d, args.cpu_budget)
        line["cpu_baseline"] = {"value": pairs / cb["step_s"], "unit": "pairs/s", "cores": cb["cores"],
                                "kind": "oracle", "sample": cb["sample"]}
    return line


# The other workloads the headline metric names, measured in the default run
# beside the large sparse layout: the dense long-edge layout (edge-pair
# tests/s on the all-pairs tiles), the batch of 4,096 layouts (layouts/s) and
# the differentiable form (fwd+bwd steps/s and fwd+bwd / fwd).  Each is its
# own bounded run (its own warm-up, timed steps, clocks, roofline, e2e and
# oracle baseline).
SUB_WORKLOADS = ("dense_long_edge", "batched", "differentiable")
SUB_STEPS = 10
SUB_CPU_BUDGET = 8.0


def run_sub_workloads(args, rank, world, local_rank) -> dict:
    out = {}
    for name in SUB_WORKLOADS:
        sub = argparse.Namespace(**vars(args))
        sub.workload = name
        sub.steps = min(args.steps, SUB_STEPS)
        sub.cpu_budget = min(args.cpu_budget, SUB_CPU_BUDGET)
        sub.cell_log2 = 0
        sub.long_pairs = "auto"
        if name == "batched":
            r = run_batched(sub, rank, world, local_rank)
        elif name == "differentiable":
            r = run_differentiable(sub, rank, world, local_rank)
        else:
            r = run_ours(sub, rank, world, local_rank)
        if r is not None:
            out[name] = r
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large_sparse")
    ap.add_argument("--cell-log2", type=int, default=0)
    ap.add_argument("--long-pairs", choices=sorted(LONG_PAIRS), default="auto",
                    help="where pairs of two long segments are tested (default: the cost model decides)")
    ap.add_argument("--strip-width", type=int, default=STRIP_WIDTH, help="strips workload: strip width")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (for profiler runs)")
    ap.add_argument("--shard", action="store_true",
                    help="single layouts under torchrun: every rank evaluates its part of the one layout "
                         "(gr_evaluate_part) and one all-reduce combines them (strong scaling)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default workload: skip the dense, batched and differentiable runs reported beside it")
    ap.add_argument("--no-single-loop", action="store_true",
                    help="batched workload: skip the one-layout-at-a-time comparison (for profiler runs)")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)  # rank 0 only; no process group needed
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        line = None
        if args.workload == "batched":
            line = run_batched(args, rank, world, local_rank)
        elif args.workload == "differentiable":
            line = run_differentiable(args, rank, world, local_rank)
        elif args.workload == "moves":
            run_moves(args, rank, world, local_rank)
        elif args.workload == "strips":
            run_strips(args, rank, world, local_rank)
        elif args.workload == "per_edge":
            run_per_edge(args, rank, world, local_rank)
        else:
            line = run_ours(args, rank, world, local_rank)
            if args.workload == "large_sparse" and world == 1 and not args.no_workloads and line is not None:
                line["workloads"] = run_sub_workloads(args, rank, world, local_rank)
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
