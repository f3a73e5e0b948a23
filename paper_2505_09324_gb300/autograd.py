"""torch.autograd integration of the rasterizer.

``rasterize(params, rast)`` renders Eq. 2 (accumulated-sum blending, Sec. 3.1)
for a ``[9, n]`` parameter tensor and returns a ``[3, H, W]`` image whose
backward pass runs the library's backward kernels.  The forward pass saves no
per-pixel state: the workspace keeps the sorted per-tile Gaussian lists and
their ranges, and the backward pass recomputes each pair's contribution from
them.  If the workspace has been re-binned since (another forward on the same
rasterizer, or a fit on it), the backward pass re-projects and re-bins from
the saved parameters first.

Capacity: when the Gaussians' tile entries exceed the plan's ``max_entries``
the kernels record GS2D_ERR_CAPACITY in the workspace and render zeros (the
gradients are zero too).  That status is device-side and reading it costs a
stream synchronisation, so it is not read by default: pass
``check_status=True`` to ``rasterize`` to read it after binning and raise, or
call ``rast.status()`` yourself.
"""

from __future__ import annotations

import torch

from . import _native as nat
from .raster import GaussianRasterizer


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, rast: GaussianRasterizer, check_status: bool):
        p = params.detach().contiguous()
        rast.prepare(p)
        if check_status:
            _raise_on_status(rast)
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
        return grads, None, None


def _raise_on_status(rast: GaussianRasterizer):
    st = rast.status()
    if st != nat.GS2D_OK:
        raise nat.Gs2dError(st, "device status after binning (GS2D_ERR_CAPACITY: the tile "
                                "entries exceed max_entries; the render would be zero)")


def rasterize(params: torch.Tensor, rast: GaussianRasterizer,
              check_status: bool = False) -> torch.Tensor:
    """Differentiable render of ``params`` ([9, n] float32 CUDA) with ``rast``.

    With ``check_status`` the workspace status is read after binning (one
    stream synchronisation) and a capacity overflow raises ``Gs2dError``
    instead of returning a zero image."""
    return _Rasterize.apply(params, rast, check_status)
