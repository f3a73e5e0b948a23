"""GB300-native (sm_103a) 2D Gaussian-splatting frame encoder: the hot path of
"Neural Video Compression using 2D Gaussian Splatting" (arXiv 2505.09324).

The differentiable tile rasterizer (projection, tile binning + per-tile index sort,
accumulated-sum blending of Eq. 2, backward pass), the Adam fitting step and
the frame-fitting loop are hand-written CUDA kernels in ``libgs2d.so`` behind
the C ABI of ``include/gs2d.h``; this package is a thin binding over it.
"""

from .quant import Quantizer  # noqa: F401
from .raster import (BatchRasterizer, GaussianRasterizer, RasterConfig, adam_step,  # noqa: F401
                     autotune, encode_sequence, frame_from_rgb8, roi_init,
                     roi_init_trace)

__all__ = ["BatchRasterizer", "GaussianRasterizer", "Quantizer", "RasterConfig", "adam_step",
           "autotune", "encode_sequence", "frame_from_rgb8", "roi_init", "roi_init_trace"]
