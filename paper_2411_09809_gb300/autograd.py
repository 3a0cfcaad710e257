"""PyTorch autograd over the differentiable readability terms.

``ReadabilityTerms(edges)(xy)`` returns the float32 tensor (E_ca, M_l, M_a) of
an FP32 layout (arXiv 2411.09809, Sec. 2.1: Algorithms 5, 3 and 2) and, on
backward, the gradient of any function of it with respect to ``xy``.  Both
directions run in libgr's kernels (gr_diff_forward / gr_diff_backward); this
module only moves tensors across the C boundary.

The crossing set and every vertex's smallest gap are held fixed by the
gradient: the metrics are piecewise smooth in the coordinates and the gradient
is the one of the piece the forward found.  ``readability_loss`` combines the
terms as (1 - E_ca) + M_l + (1 - M_a), which is zero for a layout whose
crossings are all at the ideal angle, whose edges are equally long and whose
vertices have evenly spread edges.
"""
from __future__ import annotations

import math

import torch

from . import gr


class _Terms(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xy, module):
        layout = module._layout_for(xy)
        out = torch.empty(3, dtype=torch.float32, device=xy.device)
        gr.gr_diff_forward(layout.handle, module.ideal_rad, out, torch.cuda.current_stream(xy.device).cuda_stream)
        module._generation += 1
        ctx.module = module
        ctx.generation = module._generation
        ctx.shape = xy.shape
        return out

    @staticmethod
    def backward(ctx, gout):
        module = ctx.module
        if module._generation != ctx.generation:
            raise RuntimeError("ReadabilityTerms: backward must follow its own forward "
                               "(the module ran another forward in between)")
        grad = torch.empty(ctx.shape, dtype=torch.float32, device=gout.device)
        gr.gr_diff_backward(module._layout.handle, gout.detach().to(torch.float32).contiguous(), grad,
                            torch.cuda.current_stream(gout.device).cuda_stream)
        return grad, None


class ReadabilityTerms(torch.nn.Module):
    """Differentiable (E_ca, M_l, M_a) of layouts of one graph.

    ``edges`` is an int32 [E, 2] tensor on the device; ``xy`` passed to
    ``forward`` a float32 [V, 2] tensor on the same device.  The library
    layout is created at the first call and updated in place afterwards; one
    backward may follow each forward.
    """

    def __init__(self, edges: torch.Tensor, ideal_rad: float = 7.0 * math.pi / 18.0):
        super().__init__()
        if edges.dtype != torch.int32 or not edges.is_cuda:
            raise TypeError("edges must be an int32 CUDA tensor")
        self.edges = edges.contiguous()
        self.ideal_rad = float(ideal_rad)
        self._layout = None
        self._generation = 0

    def _layout_for(self, xy: torch.Tensor) -> gr.Layout:
        if xy.dtype != torch.float32 or not xy.is_cuda or xy.dim() != 2 or xy.shape[1] != 2:
            raise TypeError("xy must be a float32 CUDA tensor of shape [V, 2]")
        xy = xy.detach().contiguous()
        stream = torch.cuda.current_stream(xy.device).cuda_stream
        if self._layout is None or self._layout.V != xy.shape[0] or self._stream != stream:
            if self._layout is not None:
                self._layout.close()
            self._layout = gr.Layout(xy, self.edges, stream=stream, coord_type=gr.GR_COORD_F32)
            self._stream = stream
        else:
            self._layout.update(xy)
        return self._layout

    def forward(self, xy: torch.Tensor) -> torch.Tensor:
        return _Terms.apply(xy, self)

    def close(self) -> None:
        if self._layout is not None:
            self._layout.close()
            self._layout = None


def readability_loss(terms: torch.Tensor) -> torch.Tensor:
    """(1 - E_ca) + M_l + (1 - M_a) of a (E_ca, M_l, M_a) tensor."""
    return (1.0 - terms[0]) + terms[1] + (1.0 - terms[2])
