"""One large layout evaluated by several ranks, one part of the pair work each.

The paper scales its readability metrics across machines by partitioning the
plane (Sec. 3.2.1-3.2.2: the grid and strip divisions behind its strong
scaling experiment).  Here each rank evaluates one part of the same layout
(gr_evaluate_part: a disjoint share of the crossing grid's work items, the
all-pairs tiles and the occlusion points; binning, minimum angle and edge
length variation repeated), and one all-reduce of the parts' integer tallies
(gr_partial, 17 int64) followed by gr_combine_parts gives every rank the
result of evaluating the whole layout, bit for bit.  This module only moves
those integers through torch.distributed; the arithmetic is libgr's.
"""
from __future__ import annotations

from . import gr


def reduce_partials(partial: gr.gr_partial, group=None) -> gr.gr_partial:
    """Sums a gr_partial over the ranks of `group` (one integer all-reduce).
    The tensor lives on the current CUDA device for NCCL, on the host otherwise."""
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(gr.partial_to_list(partial), dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return gr.partial_from_list(t.cpu().tolist())


def evaluate_sharded(layout, metrics: int = gr.GR_METRIC_ALL, ideal_rad: float = 0.0, occlusion_d: int = 0,
                     group=None) -> gr.gr_result:
    """The gr_result of `layout` (a gr.Layout or its handle) evaluated by all
    ranks of `group` together, rank r taking part r of world_size."""
    import torch.distributed as dist

    handle = getattr(layout, "handle", layout)
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    part = gr.gr_evaluate_part(handle, rank, world, metrics, ideal_rad, occlusion_d)
    return gr.gr_combine_parts(reduce_partials(part, group), ideal_rad, occlusion_d)
