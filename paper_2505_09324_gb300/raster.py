"""Torch-facing wrapper of libgs2d: PyTorch provides device memory and streams,
the library's kernels do all the work.

``GaussianRasterizer`` owns one workspace (a plan for a W x H frame and n
Gaussians).  Parameters are float32 CUDA tensors of shape ``[9, n]`` with rows
``mu_x, mu_y, l1, l2, l3, c_r, c_g, c_b, w`` (Sec. 3.1: mean, Cholesky vector of
Eq. 1, colour; w weights the colour, c' = w c in Eq. 2).  Images are float32
``[3, H, W]``.
"""

from __future__ import annotations

import dataclasses
import math

import torch

from . import _native as nat


@dataclasses.dataclass
class RasterConfig:
    """Constants of the rasterizer and the optimiser (project readings; the paper
    fixes none): tile 16, stage 64, sigma <= 4.5, |alpha| >= 1/255,
    det Sigma > 1e-8, Adam lr 1e-2, betas (0.9, 0.999), eps 1e-8.  tile (8, 16,
    32), stage (32, 64, 128, 256 Gaussians per shared-memory batch) and launch
    (persistent queue or one block per tile) choose the render schedule only."""

    tile: int = 16
    sigma_cut: float = 4.5
    alpha_min: float = 1.0 / 255.0
    det_eps: float = 1e-8
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    stage: int = 64
    launch: int = nat.LAUNCH_GRID
    # fit-loop learning-rate scales per parameter group and decay per step
    lr_mu: float = 1.0
    lr_shape: float = 1.0
    lr_color: float = 1.0
    lr_weight: float = 1.0
    lr_decay: float = 1.0
    # fit-loop tile lists: boxes widened by this many pixels, rebuilt only when
    # a Gaussian leaves its listed tiles (negative: every iteration)
    bin_margin: float = 4.0
    # backward reduction: REDUCE_SLOTS (fixed order, bit-reproducible) or
    # REDUCE_ATOMIC (float atomics; order of additions varies run to run)
    reduce: int = nat.REDUCE_SLOTS

    @classmethod
    def fast_fit(cls, **overrides):
        """The FAST_FIT schedule (plus any other field overrides)."""
        return cls(**{**FAST_FIT, **overrides})

    def to_c(self) -> nat.Config:
        return nat.Config(self.tile, self.sigma_cut, self.alpha_min, self.det_eps, self.lr,
                          self.beta1, self.beta2, self.eps, self.stage, self.launch, self.lr_mu,
                          self.lr_shape, self.lr_color, self.lr_weight, self.lr_decay,
                          self.bin_margin, self.reduce)


# Learning-rate schedule for fitting a frame from an initialiser (the
# "dynamic learning rate scheduler" the paper credits without specifying it;
# tuned on the 1080p conferencing workload: 35 dB in about 35 iterations from
# the ROI initialisation instead of about 230, monotone PSNR over long fits).
# Warm starts (P-frames) keep the plain rate: with fresh Adam moments every
# parameter's first step is a full learning rate.
FAST_FIT = {"lr_mu": 50.0, "lr_shape": 30.0, "lr_color": 10.0, "lr_weight": 3.0,
            "lr_decay": 0.995}


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check(t: torch.Tensor, name: str, shape=None, dtype=torch.float32):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


class GaussianRasterizer:
    """One plan + workspace: project -> bin_sort -> render_fwd / render_bwd /
    render_l2 on a W x H frame with n Gaussians."""

    def __init__(self, width: int, height: int, n: int, max_entries: int = 0,
                 config: RasterConfig | None = None, device=None):
        self.config = config or RasterConfig()
        self.plan = nat.plan_init(width, height, n, max_entries, self.config.to_c())
        self.width, self.height, self.n = width, height, n
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        # zero-filled: the workspace status word must start at GS2D_OK
        self.ws = torch.zeros(int(self.plan.ws_bytes), dtype=torch.uint8, device=self.device)
        if self.ws.data_ptr() % 256:
            raise RuntimeError("workspace allocation is not 256-byte aligned")
        self.version = 0  # bumped whenever the binned lists in the workspace change

    @property
    def ws_ptr(self) -> int:
        return self.ws.data_ptr()

    def image_shape(self):
        return (3, self.height, self.width)

    def project(self, params: torch.Tensor, stream=None):
        p = _check(params, "params", (9, self.n))
        nat.project(self.plan, self.ws_ptr, p, _stream(stream))
        self.version += 1

    def bin_sort(self, stream=None):
        nat.bin_sort(self.plan, self.ws_ptr, _stream(stream))
        self.version += 1

    def prepare(self, params: torch.Tensor, stream=None):
        """project + bin_sort (fused into one launch where the device allows)."""
        p = _check(params, "params", (9, self.n))
        nat.prepare(self.plan, self.ws_ptr, p, _stream(stream))
        self.version += 1

    def render_fwd(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        img = out if out is not None else torch.empty(self.image_shape(), device=self.device)
        nat.render_fwd(self.plan, self.ws_ptr, _check(img, "img", self.image_shape()),
                       _stream(stream))
        return img

    def render_bwd(self, params: torch.Tensor, dimg: torch.Tensor, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        grads = out if out is not None else torch.empty((9, self.n), device=self.device)
        nat.render_bwd(self.plan, self.ws_ptr, _check(params, "params", (9, self.n)),
                       _check(dimg, "dimg", self.image_shape()),
                       _check(grads, "grads", (9, self.n)), _stream(stream))
        return grads

    def render_l2(self, params: torch.Tensor, target: torch.Tensor, want_image: bool = False,
                  stream=None):
        """Fused forward + L2 loss + backward.  Returns (grads, loss[2], img|None)
        where loss = (mean squared error, mean squared error of the clamped image)."""
        grads = torch.empty((9, self.n), device=self.device)
        loss = torch.empty(2, device=self.device)
        img = torch.empty(self.image_shape(), device=self.device) if want_image else None
        nat.render_l2(self.plan, self.ws_ptr, _check(params, "params", (9, self.n)),
                      _check(target, "target", self.image_shape()),
                      _check(grads, "grads", (9, self.n)),
                      0 if img is None else img.data_ptr(), loss.data_ptr(), _stream(stream))
        return grads, loss, img

    def read_bins(self, stream=None, max_keys: int = -1):
        return nat.read_bins(self.plan, self.ws_ptr, _stream(stream), max_keys)

    def count_pairs(self, stream=None):
        """(listed pairs, contributing pairs) of the current sorted list."""
        return nat.count_pairs(self.plan, self.ws_ptr, _stream(stream))

    def rebins(self, stream=None) -> int:
        """How often the fit loop rebuilt its tile lists in this workspace
        (since the last fit reset); see RasterConfig.bin_margin."""
        return nat.fit_rebins(self.plan, self.ws_ptr, _stream(stream))

    def status(self, reset: bool = False, stream=None) -> int:
        return nat.ws_status(self.plan, self.ws_ptr, reset, _stream(stream))

    def select_changed(self, reference: torch.Tensor, frame: torch.Tensor, threshold: float,
                       stream=None):
        """P-frame selection (gs2d_select_changed) on the current binning (of
        the reference Gaussians): (uint8 [n] flags, count)."""
        sel = torch.empty(self.n, dtype=torch.uint8, device=self.device)
        cnt = nat.select_changed(self.plan, self.ws_ptr,
                                 _check(reference, "reference", self.image_shape()),
                                 _check(frame, "frame", self.image_shape()), float(threshold),
                                 sel.data_ptr(), _stream(stream))
        return sel, cnt

    def encode_pframe(self, target: torch.Tensor, params: torch.Tensor,
                      selected: torch.Tensor, iters: int, adam_state=None, stream=None) -> float:
        """Fits only the selected Gaussians (params in place) for `iters`
        iterations over the tiles they cover; returns the full-frame PSNR."""
        if adam_state is None:
            adam_state = (torch.empty_like(params), torch.empty_like(params))
        m, v = adam_state
        shape = (9, self.n)
        # the P-frame loop re-bins the workspace every iteration
        self.version += 1
        return nat.encode_pframe(self.plan, self.ws_ptr,
                                 _check(target, "target", self.image_shape()),
                                 _check(params, "params", shape), _check(m, "adam_m", shape),
                                 _check(v, "adam_v", shape),
                                 _check(selected, "selected", (self.n,), dtype=torch.uint8),
                                 iters, _stream(stream))

    def encode_frame(self, target: torch.Tensor, params: torch.Tensor, iters: int,
                     target_psnr: float = 0.0, check_every: int = 50, adam_state=None,
                     stream=None):
        """Fits ``params`` (in place) to ``target``; see gs2d_encode_frame."""
        if adam_state is None:
            adam_state = (torch.empty_like(params), torch.empty_like(params))
        m, v = adam_state
        # the fit loop re-bins the workspace (lists of other parameters)
        self.version += 1
        st, done, final, trace = nat.encode_frame(
            self.plan, self.ws_ptr, _check(target, "target", self.image_shape()),
            _check(params, "params", (9, self.n)), _check(m, "adam_m", (9, self.n)),
            _check(v, "adam_v", (9, self.n)), iters, float(target_psnr), check_every,
            _stream(stream))
        if st not in (nat.GS2D_OK, nat.GS2D_ERR_CAPACITY):
            nat.check(st, "gs2d_encode_frame")
        return {"status": st, "iters": done, "psnr": final, "trace": trace}

    def encode_frame_qat(self, target: torch.Tensor, params: torch.Tensor, iters: int,
                         quantizer, adam_state=None, stream=None):
        """Quantisation-aware fit (Sec. 3.3 A, QAT): ``iters`` iterations of
        gs2d_fit_step_qat from fresh Adam moments, each rendering the Gaussians
        as ``quantizer`` codes them (straight-through gradient to the float
        ``params``, updated in place).  Returns the PSNR of the float and of
        the quantised fit, and the quantiser's output for the final params."""
        if adam_state is None:
            adam_state = (torch.empty_like(params), torch.empty_like(params))
        m, v = adam_state
        shape = (9, self.n)
        t = _check(target, "target", self.image_shape())
        p = _check(params, "params", shape)
        mp, vp = _check(m, "adam_m", shape), _check(v, "adam_v", shape)
        s = _stream(stream)
        nat.fit_reset(self.plan, self.ws_ptr, mp, vp, s)
        for _ in range(iters):
            nat.fit_step_qat(self.plan, self.ws_ptr, t, p, mp, vp, quantizer.c, s)
        self.version += 1
        codes, values, ranges = quantizer.quantize(params, stream=stream)
        return {"psnr": self.psnr(target, params, stream), "psnr_q": self.psnr(target, values,
                                                                               stream),
                "codes": codes, "values": values, "ranges": ranges}

    def fit_step(self, target: torch.Tensor, params: torch.Tensor, adam_state, stream=None):
        """One fit iteration (gs2d_fit_step) on params and the Adam moments
        (m, v) in place; the step counter lives in the workspace."""
        m, v = adam_state
        shape = (9, self.n)
        nat.fit_step(self.plan, self.ws_ptr, _check(target, "target", self.image_shape()),
                     _check(params, "params", shape), _check(m, "adam_m", shape),
                     _check(v, "adam_v", shape), _stream(stream))
        self.version += 1

    def fit_reset(self, adam_state, stream=None):
        """Restarts the fit's optimiser (gs2d_fit_reset)."""
        m, v = adam_state
        nat.fit_reset(self.plan, self.ws_ptr, _check(m, "adam_m", (9, self.n)),
                      _check(v, "adam_v", (9, self.n)), _stream(stream))

    def fit_checkpoint(self, params: torch.Tensor, adam_state, stream=None) -> dict:
        """A checkpoint of a fit in progress: host copies of params and the
        Adam moments and the optimiser state of the workspace
        (gs2d_fit_state_get; synchronises the stream)."""
        st = nat.fit_state_get(self.plan, self.ws_ptr, _stream(stream))
        m, v = adam_state
        return {"params": params.detach().cpu().clone(), "m": m.cpu().clone(),
                "v": v.cpu().clone(), "step": int(st.step), "beta1_pow": st.beta1_pow,
                "beta2_pow": st.beta2_pow, "decay_pow": st.decay_pow}

    def fit_restore(self, ckpt: dict, params: torch.Tensor, adam_state, stream=None):
        """Resumes from fit_checkpoint's output: copies params and the moments
        back into the given device tensors and sets the workspace's optimiser
        state (gs2d_fit_state_set); the next fit_step continues the fit."""
        m, v = adam_state
        params.copy_(ckpt["params"])
        m.copy_(ckpt["m"])
        v.copy_(ckpt["v"])
        st = nat.FitState(int(ckpt["step"]), 0, float(ckpt["beta1_pow"]),
                          float(ckpt["beta2_pow"]), float(ckpt["decay_pow"]))
        nat.fit_state_set(self.plan, self.ws_ptr, st, _stream(stream))
        self.version += 1

    def psnr(self, target: torch.Tensor, params: torch.Tensor, stream=None) -> float:
        """PSNR of the clamped render of ``params`` against ``target``
        (re-bins the workspace)."""
        self.prepare(params, stream=stream)
        _, loss, _ = self.render_l2(params, target, stream=stream)
        mse = float(loss[1].item())
        return 10.0 * math.log10(1.0 / max(mse, 1e-30))


def encode_sequence(rast: GaussianRasterizer, frames, params: torch.Tensor, iters_first: int,
                    iters_next: int, stream=None, selective_threshold: float | None = None,
                    gop: int | None = None, on_frame=None):
    """Fits a frame sequence with inter-frame reuse (Sec. 3.2: P-frames start
    from the previous frame's optimised Gaussians): frame 0 for ``iters_first``
    iterations from ``params`` (an initialiser's output), every later frame
    for ``iters_next`` iterations from the previous frame's fit; the Adam
    moments restart per frame.  With ``selective_threshold`` the later frames
    are P-frames (Sec. 3.2 C): only the Gaussians contributing to pixels whose
    residual against the previous fit's render exceeds the threshold are
    fitted (gs2d_select_changed, gs2d_encode_pframe).  ``frames`` yields
    [3, H, W] float32 CUDA tensors.  ``params`` is updated in place (ends as
    the last frame's fit).  With ``gop`` every frame k with k % gop == 0 is an
    I-frame (all Gaussians fitted and coded); otherwise only frame 0 is.
    ``on_frame(k, params, selected)`` runs after each frame, outside its
    timing (selected: the P-frame's uint8 mask, None on an I-frame).
    Returns one {"iters", "psnr", "seconds", "coded"[, "selected"]} record
    per frame (wall clock around the frame's calls, which synchronise the
    stream; coded = Gaussians the frame transmits)."""
    import time
    out = []
    adam = (torch.empty_like(params), torch.empty_like(params))
    ref = None
    for k, frame in enumerate(frames):
        iters = iters_first if k == 0 else iters_next
        t0 = time.perf_counter()
        if k == 0 or selective_threshold is None or (gop and k % gop == 0):
            r = rast.encode_frame(frame, params, iters, target_psnr=0.0, check_every=iters,
                                  adam_state=adam, stream=stream)
            out.append({"iters": r["iters"], "psnr": r["psnr"],
                        "seconds": time.perf_counter() - t0, "coded": rast.n})
            if on_frame is not None:
                on_frame(k, params, None)
            continue
        rast.prepare(params, stream=stream)
        ref = rast.render_fwd(out=ref, stream=stream)
        sel, cnt = rast.select_changed(ref, frame, selective_threshold, stream=stream)
        psnr = rast.encode_pframe(frame, params, sel, iters, adam_state=adam, stream=stream)
        out.append({"iters": iters, "psnr": psnr, "seconds": time.perf_counter() - t0,
                    "selected": cnt, "coded": cnt})
        if on_frame is not None:
            on_frame(k, params, sel)
    return out


def frame_from_rgb8(rgb: torch.Tensor, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """gs2d_frame_from_rgb8: an 8-bit [H, W, 3] RGB frame on the device to the
    planar float32 [3, H, W] frame (c / 255) the fit loop targets."""
    if not (isinstance(rgb, torch.Tensor) and rgb.is_cuda and rgb.dtype == torch.uint8
            and rgb.dim() == 3 and rgb.shape[2] == 3 and rgb.stride(2) == 1
            and rgb.stride(1) == 3):
        raise ValueError("rgb must be a uint8 CUDA tensor [H, W, 3] with packed pixels")
    h, w = rgb.shape[0], rgb.shape[1]
    if out is None:
        out = torch.empty((3, h, w), device=rgb.device)
    nat.frame_from_rgb8(rgb.data_ptr(), w, h, rgb.stride(0), _check(out, "out", (3, h, w)),
                        _stream(stream))
    return out


def roi_init(frame: torch.Tensor, mask: torch.Tensor, n: int, roi_frac: float,
             bg_xy: torch.Tensor, stream=None):
    """Region-of-interest superpixel initialiser (gs2d_roi_init).  frame:
    [3, H, W] float32, mask: [H, W] uint8/bool, bg_xy: [2, n] float32 random
    background positions.  Returns (params [9, n], n_roi)."""
    return _roi_init(frame, mask, n, roi_frac, bg_xy, stream, trace=False)[:2]


def roi_init_trace(frame: torch.Tensor, mask: torch.Tensor, n: int, roi_frac: float,
                   bg_xy: torch.Tensor, stream=None):
    """roi_init with the K-means iterations written out
    (gs2d_roi_init_trace): (params [9, n], n_roi, centres [10, 5, n] (r, g,
    b, x, y rows; the first n_roi columns used) each assignment used,
    labels [10, H, W] int32 each assignment made)."""
    return _roi_init(frame, mask, n, roi_frac, bg_xy, stream, trace=True)


def _roi_init(frame, mask, n, roi_frac, bg_xy, stream, trace):
    _, h, w = frame.shape
    f = _check(frame, "frame", (3, h, w))
    if mask.dtype == torch.bool:
        mask = mask.to(torch.uint8)
    mk = _check(mask.contiguous(), "mask", (h, w), dtype=torch.uint8)
    bg = _check(bg_xy, "bg_xy", (2, n))
    params = torch.empty((9, n), device=frame.device)
    nbytes = int(nat.load().gs2d_roi_init_scratch_bytes(w, h, n))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=frame.device)
    n_roi = nat.ctypes.c_int32(0)
    args = (nat._p(f), nat._p(mk), w, h, n, float(roi_frac), nat._p(bg),
            nat._p(params.data_ptr()), nat.ctypes.byref(n_roi), nat._p(scratch.data_ptr()),
            nbytes)
    if not trace:
        nat.check(nat.load().gs2d_roi_init(*args, nat._p(_stream(stream))), "gs2d_roi_init")
        return params, int(n_roi.value), None, None
    cen = torch.empty((10, 5, n), device=frame.device)
    lab = torch.empty((10, h, w), dtype=torch.int32, device=frame.device)
    nat.check(nat.load().gs2d_roi_init_trace(*args, nat._p(cen.data_ptr()),
                                             nat._p(lab.data_ptr()), nat._p(_stream(stream))),
              "gs2d_roi_init_trace")
    return params, int(n_roi.value), cen, lab


def adam_step(params: torch.Tensor, grads: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
              step: int, mask: torch.Tensor | None = None, config: RasterConfig | None = None,
              stream=None):
    """One Adam step in place over equally shaped float32 CUDA tensors."""
    shape = tuple(params.shape)
    ptrs = [_check(t, n, shape) for t, n in ((params, "params"), (grads, "grads"), (m, "m"),
                                              (v, "v"))]
    mp = 0
    if mask is not None:
        if params.numel() % 9:
            raise ValueError("mask needs params with 9 rows")
        mp = _check(mask, "mask", (params.numel() // 9,), dtype=torch.uint8)
    cfg = (config or RasterConfig()).to_c()
    nat.adam_step(*ptrs, params.numel(), step, mp, cfg, _stream(stream))


class BatchRasterizer(GaussianRasterizer):
    """One plan + workspace for a batch of independent clips of different sizes
    (gs2d_plan_init_batch): ``sizes`` = [(width, height, n), ...].  Parameters
    are one ``[9, n_total]`` tensor (clip c owns columns ``offsets[c]`` ...);
    images are one flat float32 tensor of ``pixels * 3`` values, clip c's
    ``[3, H, W]`` image at ``pix_off[c]`` (see ``clip_view``).  Every step runs
    once over all clips; each clip keeps its own loss."""

    def __init__(self, sizes, max_entries: int = 0, config: RasterConfig | None = None,
                 device=None):
        self.config = config or RasterConfig()
        self.sizes = [(int(w), int(h), int(n)) for (w, h, n) in sizes]
        self.plan, self.clips = nat.plan_init_batch(self.sizes, max_entries, self.config.to_c())
        self.width, self.height, self.n = 0, 0, int(self.plan.n)
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        self.ws = torch.zeros(int(self.plan.ws_bytes), dtype=torch.uint8, device=self.device)
        if self.ws.data_ptr() % 256:
            raise RuntimeError("workspace allocation is not 256-byte aligned")
        nat.ws_set_clips(self.plan, self.ws_ptr, self.clips, _stream(None))
        self.version = 0
        self.offsets = [int(c.g_off) for c in self.clips]
        self.pix_off = [int(c.pix_off) for c in self.clips]

    def image_shape(self):
        return (3 * int(self.plan.pixels),)

    def clip_view(self, flat: torch.Tensor, c: int) -> torch.Tensor:
        """Clip c's [3, H, W] view of a batch image buffer."""
        w, h, _ = self.sizes[c]
        o = self.pix_off[c]
        return flat[o:o + 3 * w * h].view(3, h, w)

    def pack_images(self, images) -> torch.Tensor:
        """Concatenates per-clip [3, H, W] tensors into the batch layout."""
        return torch.cat([im.reshape(-1) for im in images]).contiguous()

    def pack_params(self, params) -> torch.Tensor:
        """Concatenates per-clip [9, n_c] tensors into one [9, n_total]."""
        return torch.cat(list(params), dim=1).contiguous()

    def clip_losses(self, stream=None):
        """[(mse, clamped mse)] per clip of the last render_l2."""
        return nat.clip_losses(self.plan, self.ws_ptr, _stream(stream))

    def encode_frame(self, *args, **kwargs):
        raise TypeError("a batch plan is fitted with encode_batch")

    def encode_batch(self, targets: torch.Tensor, params: torch.Tensor, iters: int,
                     adam_state=None, stream=None):
        """Fits every clip (params in place) for ``iters`` iterations; returns the
        per-clip PSNR of the fitted Gaussians (gs2d_encode_batch)."""
        if adam_state is None:
            adam_state = (torch.empty_like(params), torch.empty_like(params))
        m, v = adam_state
        shape = (9, self.n)
        self.version += 1  # the fit loop re-bins the workspace
        return nat.encode_batch(self.plan, self.ws_ptr, _check(targets, "targets",
                                                                self.image_shape()),
                                _check(params, "params", shape), _check(m, "adam_m", shape),
                                _check(v, "adam_v", shape), iters, _stream(stream))


_TUNED = {}


def autotune(sizes, params: torch.Tensor, targets: torch.Tensor, tiles=(8, 16, 32),
             stages=(32, 64, 128, 256), launches=(nat.LAUNCH_PERSISTENT, nat.LAUNCH_GRID),
             reps: int = 5, config: RasterConfig | None = None, max_entries: int = 0,
             stream=None, cache: bool = True, reduces=(nat.REDUCE_SLOTS,)):
    """Picks the render schedule (tile, stage, launch) for a batch
    (gs2d_autotune), and the backward reduction among ``reduces``
    (REDUCE_SLOTS only by default: the bit-reproducible one).  ``params`` /
    ``targets`` in the batch layout of ``BatchRasterizer(sizes)``.  Returns
    {"tile", "stage", "launch", "reduce", "config", "ms": {(tile, stage,
    launch): ms per fit iteration}} -- keys (tile, stage, launch, reduce)
    when several reductions are candidates; the result is cached per (sizes,
    candidates) unless ``cache`` is False."""
    sizes = [(int(w), int(h), int(n)) for (w, h, n) in sizes]
    reduces = tuple(int(r) for r in reduces)
    key = (tuple(sizes), tuple(tiles), tuple(stages), tuple(launches), max_entries, reduces)
    if cache and key in _TUNED:
        return _TUNED[key]
    base_cfg = config or RasterConfig()
    nbytes = nat.autotune_ws_bytes(sizes, list(tiles), max_entries, base_cfg.to_c())
    if nbytes == 0 or not reduces:
        raise ValueError("invalid batch or candidate lists")
    n_total = sum(n for (_, _, n) in sizes)
    pixels = sum(w * h for (w, h, _) in sizes)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=params.device)
    table, best = {}, None
    for r in reduces:
        base = dataclasses.replace(base_cfg, reduce=r).to_c()
        t, bt, bs, bl = nat.autotune(sizes, _check(params, "params", (9, n_total)),
                                     _check(targets, "targets", (3 * pixels,)), ws.data_ptr(),
                                     nbytes, list(tiles), list(stages), list(launches), reps,
                                     _stream(stream), max_entries, base)
        for k, v in t.items():
            table[k if len(reduces) == 1 else (*k, r)] = v
        ms = t[(bt, bs, bl)]
        if ms >= 0 and (best is None or ms < best[0]):
            best = (ms, bt, bs, bl, r)
    if best is None:
        raise RuntimeError("every autotuner candidate overflowed max_entries")
    _, bt, bs, bl, br = best
    cfg = dataclasses.replace(base_cfg, tile=bt, stage=bs, launch=bl, reduce=br)
    res = {"tile": bt, "stage": bs, "launch": bl, "reduce": br, "config": cfg, "ms": table}
    if cache:
        _TUNED[key] = res
    return res
