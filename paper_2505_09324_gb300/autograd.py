"""torch.autograd integration of the rasterizer.

``rasterize(params, rast)`` renders Eq. 2 (accumulated-sum blending, Sec. 3.1)
for a ``[9, n]`` parameter tensor and returns a ``[3, H, W]`` image whose
backward pass runs the library's backward kernels.  The forward pass saves no
per-pixel state: the workspace keeps the sorted per-tile Gaussian lists and
their ranges, and the backward pass recomputes each pair's contribution from
them.  If the workspace has been re-binned since (another forward on the same
rasterizer), the backward pass re-projects and re-bins from the saved
parameters first.
"""

from __future__ import annotations

import torch

from .raster import GaussianRasterizer


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, rast: GaussianRasterizer):
        p = params.detach().contiguous()
        rast.prepare(p)
        ctx.rast = rast
        ctx.version = rast.version
        ctx.save_for_backward(p)
        return rast.render_fwd()

    @staticmethod
    def backward(ctx, dimg: torch.Tensor):
        (p,) = ctx.saved_tensors
        rast: GaussianRasterizer = ctx.rast
        if rast.version != ctx.version:
            rast.prepare(p)
        grads = rast.render_bwd(p, dimg.detach().contiguous().float())
        return grads, None


def rasterize(params: torch.Tensor, rast: GaussianRasterizer) -> torch.Tensor:
    """Differentiable render of ``params`` ([9, n] float32 CUDA) with ``rast``."""
    return _Rasterize.apply(params, rast)
