"""Learned initialiser (Sec. 3.2 B: a regressor from the frame to the N
Gaussians' parameters, trained with a Chamfer loss on the means).

Network: the frame (r, g, b) and its region-of-interest mask, NHWC BF16 with 8
channels, through five 3 x 3 stride-2 convolutions with ReLU (8 -> 32 -> 64 ->
128 -> 256 -> 384 channels by default) to a stride-32 grid of cells, then a 1 x 1
convolution to `slots` groups of nine numbers per cell that the head decodes
into cell-anchored Gaussians; each frame keeps the n with the largest |w|.
About 1.3 M parameters; BF16 weights and activations, FP32 accumulation and
FP32 master weights.

In training every convolution is im2col + one BF16 tensor-core GEMM
(gs2d_gemm_bf16, the bias a weight column against a column of ones); at
inference the convolutions run as implicit GEMMs that read their operands
straight from the activations (gs2d_conv_bf16, gs2d_conv_frame_bf16), with
the same sums in the same order.  The backward pass is one
weight-gradient GEMM (dZ^T . col, split over pixels) and one input-gradient
GEMM (dZ . W) + col2im with the ReLU mask per layer.  The optimiser is the
library's Adam on the FP32 master weights.  Training minimises the L2 render
loss of the decoded Gaussians through the rasterizer (the colour and shape
signal the paper's regressor lacked) plus lambda times the Chamfer distance
between the predicted means and those of Gaussians the encoder fitted to the
same frame.  torch only provides device memory and streams.
"""

from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _native as nat
from .raster import BatchRasterizer, RasterConfig, adam_step


def _ceil8(x: int) -> int:
    return -(-x // 8) * 8


def _out(n: int) -> int:
    return (n + 2 - 3) // 2 + 1  # 3 x 3, stride 2, pad 1


@dataclasses.dataclass
class NetConfig:
    channels: tuple = (8, 32, 64, 128, 256, 384)
    slots: int = 10
    scale: float = 6.0          # px; Cholesky diagonal at o = 0
    lr: float = 1e-3
    chamfer_lambda: float = 1e-5
    wgrad_split_pixels: int = 4096  # pixels per split of the weight-gradient GEMMs


class LearnedInitializer:
    """Maps B frames of W x H to B sets of n Gaussians ([9, B n] batch layout)."""

    def __init__(self, width: int, height: int, n: int, batch: int,
                 config: NetConfig | None = None, seed: int = 0, device=None):
        self.cfg = config or NetConfig()
        self.W, self.H, self.n, self.B = width, height, n, batch
        self.dev = torch.device(device) if device is not None else torch.device("cuda")
        ch = self.cfg.channels
        if ch[0] != 8 or any(c % 8 for c in ch):
            raise ValueError("channels must be multiples of 8, starting at 8")
        self.L = len(ch) - 1
        self.sizes = [(height, width)]
        for _ in range(self.L):
            h, w = self.sizes[-1]
            self.sizes.append((_out(h), _out(w)))
        self.gh, self.gw = self.sizes[-1]
        self.cell = 2 ** self.L
        if self.gh * self.gw * self.cfg.slots < n:
            raise ValueError("fewer slots than Gaussians")
        self.ldo = _ceil8(9 * self.cfg.slots)
        # layers: (ci, co, ks, ldk); the head is a 1 x 1 convolution
        self.layers = [(ch[i], ch[i + 1], 3, _ceil8(9 * ch[i] + 1)) for i in range(self.L)]
        self.layers.append((ch[-1], self.ldo, 1, _ceil8(ch[-1] + 1)))
        g = np.random.Generator(np.random.PCG64(seed))
        self.w32, self.m, self.v, self.wb, self.wt, self.dw = [], [], [], [], [], []
        for li, (ci, co, ks, ldk) in enumerate(self.layers):
            w = np.zeros((co, ldk), np.float32)
            fan = ks * ks * ci
            if li < self.L:
                w[:, :fan] = g.normal(0.0, np.sqrt(2.0 / fan), (co, fan))  # He init for ReLU
            else:
                w[:9 * self.cfg.slots, :fan] = g.normal(0.0, 1e-3, (9 * self.cfg.slots, fan))
            t = torch.from_numpy(w).to(self.dev)
            self.w32.append(t)
            self.m.append(torch.zeros_like(t))
            self.v.append(torch.zeros_like(t))
            self.dw.append(torch.zeros_like(t))
            self.wb.append(torch.empty((co, ldk), dtype=torch.bfloat16, device=self.dev))
            self.wt.append(torch.empty((ldk, co), dtype=torch.bfloat16, device=self.dev))
        self.step_count = 0
        self._alloc()
        self._cast()

    # ------------------------------------------------------------------
    def _alloc(self):
        B, dev, bf = self.B, self.dev, torch.bfloat16
        self.x = [torch.empty((B * self.H * self.W, 8), dtype=bf, device=dev)]
        self.col, self.colT, self.dz, self.dzT, self.dcol = [], [], [], [], []
        for li, (ci, co, ks, ldk) in enumerate(self.layers):
            h, w = self.sizes[li + 1] if li < self.L else self.sizes[-1]
            P = B * h * w
            self.col.append(torch.empty((P, ldk), dtype=bf, device=dev))
            self.colT.append(torch.empty((ldk, _ceil8(P)), dtype=bf, device=dev))
            self.dz.append(torch.empty((P, co), dtype=bf, device=dev))
            self.dzT.append(torch.empty((co, _ceil8(P)), dtype=bf, device=dev))
            self.dcol.append(torch.empty((P, ldk), device=dev) if li > 0 else None)
            if li < self.L:
                self.x.append(torch.empty((P, co), dtype=bf, device=dev))
        self.out = torch.empty((B * self.gh * self.gw, self.ldo), device=dev)
        self.params = torch.empty((9, B * self.n), device=dev)
        self.sel = torch.empty((B, self.n), dtype=torch.int32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        most = 0
        for li, (ci, co, ks, ldk) in enumerate(self.layers):
            h, w = self.sizes[li + 1] if li < self.L else self.sizes[-1]
            P = B * h * w
            most = max(most, nat.load().gs2d_gemm_partial_bytes(co, ldk, ldk, P,
                                                                 self._splits(P)))
        self.partial = torch.empty(max(most // 4, 1), device=dev)

    def _splits(self, pixels: int) -> int:
        return max(1, min(512, pixels // self.cfg.wgrad_split_pixels))

    def _cast(self):
        s = self._s()
        for li, (ci, co, ks, ldk) in enumerate(self.layers):
            nat.call("gs2d_cast_weights", self.w32[li].data_ptr(), co, ldk,
                     self.wb[li].data_ptr(), self.wt[li].data_ptr(), s)

    @staticmethod
    def _s() -> int:
        return int(torch.cuda.current_stream().cuda_stream)

    def num_params(self) -> int:
        return sum(co * (ks * ks * ci + 1) for (ci, co, ks, ldk) in self.layers[:-1]) + \
            9 * self.cfg.slots * (self.layers[-1][0] + 1)

    # ------------------------------------------------------------------
    def forward(self, frames: torch.Tensor, masks: torch.Tensor | None,
                keep_col: bool = True) -> torch.Tensor:
        """frames: [B, 3, H, W] float32 CUDA; masks: [B, H, W] uint8 or None.
        Returns the Gaussians, [9, B n] float32 (frame b in columns b n ...).
        keep_col=False (inference) runs the convolutions as implicit GEMMs
        (gs2d_conv_bf16; the first one, gs2d_conv_frame_bf16, straight from
        the frames when W is a multiple of 16; the same result bit for bit)
        and keeps neither the im2col operands nor the 8-channel input, which
        backward() needs."""
        B, s = self.B, self._s()
        if tuple(frames.shape) != (B, 3, self.H, self.W) or frames.dtype != torch.float32:
            raise ValueError("frames must be [B, 3, H, W] float32")
        frames = frames.contiguous()
        mptr = 0
        if masks is not None:
            masks = masks.to(torch.uint8).contiguous()
            mptr = masks.data_ptr()
        st = self.status.data_ptr()
        ci0, co0, ks0, ldk0 = self.layers[0]
        first = 0
        if not keep_col and self.W % 16 == 0 and ks0 == 3 and co0 <= 128 and self.L > 0:
            # the first convolution straight from the frames and masks (the
            # 8-channel input never written; the same result bit for bit)
            nat.call("gs2d_conv_frame_bf16", frames.data_ptr(), mptr, B, self.H, self.W, 3, 2,
                     1, self.wb[0].data_ptr(), ldk0, co0, 1, 0, self.x[1].data_ptr(), co0, st, s)
            first = 1
        else:
            nat.call("gs2d_cnn_input", frames.data_ptr(), mptr, B, self.H, self.W,
                     self.x[0].data_ptr(), s)
        for li, (ci, co, ks, ldk) in enumerate(self.layers):
            if li < first:
                continue
            src = self.x[li]
            hi, wi = self.sizes[li] if li < self.L else self.sizes[-1]
            stride, pad = (2, 1) if ks == 3 else (1, 0)
            # implicit GEMM unless K is very deep (the last 3 x 3 layer: 37
            # k-tiles over 32 tiles, where the TMA-fed GEMM over an im2col
            # operand is faster); the results are identical either way
            if not keep_col and (ldk + 63) // 64 <= 32:
                last = li == self.L
                nat.call("gs2d_conv_bf16", src.data_ptr(), B, hi, wi, ci, ks, stride, pad,
                         self.wb[li].data_ptr(), ldk, co, 0 if last else 1,
                         self.out.data_ptr() if last else 0,
                         0 if last else self.x[li + 1].data_ptr(), co, st, s)
                continue
            nat.call("gs2d_im2col", src.data_ptr(), B, hi, wi, ci, ks, stride, pad,
                     self.col[li].data_ptr(), ldk, s)
            P = self.col[li].shape[0]
            if li < self.L:
                nat.gemm_bf16(self.col[li].data_ptr(), ldk, self.wb[li].data_ptr(), ldk, P, co,
                              ldk, 0, True, 0, self.x[li + 1].data_ptr(), co, 1, 0, st, s)
            else:
                nat.gemm_bf16(self.col[li].data_ptr(), ldk, self.wb[li].data_ptr(), ldk, P, co,
                              ldk, 0, False, self.out.data_ptr(), 0, co, 1, 0, st, s)
        c = self.cfg
        nat.call("gs2d_head_decode", self.out.data_ptr(), self.ldo, B, self.gh, self.gw, c.slots,
                 self.cell, c.scale, self.n, self.params.data_ptr(), B * self.n,
                 self.sel.data_ptr(), s)
        return self.params

    def capture(self, frames: torch.Tensor, masks: torch.Tensor | None = None):
        """Records forward() on these input tensors as one CUDA graph; replay()
        then re-runs the whole network (every launch of it) on whatever the
        same tensors hold, with no per-launch host work."""
        side = torch.cuda.Stream(self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            # one-time setup (kernel attributes) outside the graph
            self.forward(frames, masks, keep_col=False)
        side.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            self.forward(frames, masks, keep_col=False)
        self._graph = graph
        return graph

    def replay(self) -> torch.Tensor:
        """Runs the captured forward on the current stream's timeline;
        returns the Gaussians ([9, B n], the same tensor as forward's)."""
        if getattr(self, "_graph", None) is None:
            raise RuntimeError("capture() first")
        self._graph.replay()
        return self.params

    def backward(self, dparams: torch.Tensor):
        """Weight gradients (into self.dw) for dL/dparams ([9, B n] float32) of
        the last forward."""
        B, s, c = self.B, self._s(), self.cfg
        st = self.status.data_ptr()
        nat.call("gs2d_head_decode_bwd", self.out.data_ptr(), self.ldo, B, self.gh, self.gw,
                 c.slots, self.cell, c.scale, self.n, self.sel.data_ptr(),
                 dparams.contiguous().data_ptr(), B * self.n, self.dz[self.L].data_ptr(), s)
        for li in range(self.L, -1, -1):
            ci, co, ks, ldk = self.layers[li]
            P = self.col[li].shape[0]
            ldp = self.dzT[li].shape[1]
            # weight gradient: dW[co][k] = sum_p dZ[p][co] col[p][k]
            nat.call("gs2d_transpose_bf16", self.dz[li].data_ptr(), P, co, co,
                     self.dzT[li].data_ptr(), ldp, s)
            nat.call("gs2d_transpose_bf16", self.col[li].data_ptr(), P, ldk, ldk,
                     self.colT[li].data_ptr(), ldp, s)
            nat.gemm_bf16(self.dzT[li].data_ptr(), ldp, self.colT[li].data_ptr(), ldp, co, ldk, P,
                          0, False, self.dw[li].data_ptr(), 0, ldk, self._splits(P),
                          self.partial.data_ptr(), st, s)
            if li == 0:
                break
            # input gradient: dcol[p][k] = sum_co dZ[p][co] W[co][k], then the
            # taps back onto the input, times the ReLU mask of that input
            nat.gemm_bf16(self.dz[li].data_ptr(), co, self.wt[li].data_ptr(), co, P, ldk, co, 0,
                          False, self.dcol[li].data_ptr(), 0, ldk, 1, 0, st, s)
            hi, wi = self.sizes[li] if li < self.L else self.sizes[-1]
            stride, pad = (2, 1) if ks == 3 else (1, 0)
            nat.call("gs2d_col2im", self.dcol[li].data_ptr(), ldk, B, hi, wi, ci, ks, stride,
                     pad, self.x[li].data_ptr(), self.dz[li - 1].data_ptr(), s)

    def step(self):
        """One Adam step of every weight (the library's Adam), then the BF16 copies."""
        self.step_count += 1
        cfg = RasterConfig(lr=self.cfg.lr)
        for li in range(len(self.layers)):
            adam_step(self.w32[li], self.dw[li], self.m[li], self.v[li], self.step_count,
                      config=cfg)
        self._cast()

    def check_status(self):
        if int(self.status.item()) != 0:
            raise RuntimeError(f"tensor-core GEMM status {int(self.status.item())}")

    # ------------------------------------------------------------------
    def state(self) -> dict:
        return {f"w{i}": w.cpu().numpy() for i, w in enumerate(self.w32)}

    def load_state(self, st: dict):
        """Weights from state(), or BF16 bit patterns (uint16) of them."""
        for i, w in enumerate(self.w32):
            a = np.asarray(st[f"w{i}"])
            if a.dtype == np.uint16:
                a = (a.astype(np.uint32) << 16).view(np.float32)
            w.copy_(torch.from_numpy(np.ascontiguousarray(a, np.float32)))
        self._cast()


PACKAGED = "data/learned_init_1920x1080_20k.npz"


def packaged(width: int, height: int, n: int, batch: int = 1, device=None):
    """The initialiser trained by `python -m paper_2505_09324_gb300.learned`
    on 5000 synthetic 1920 x 1080 conferencing frames (seeds 10000 ... 14999,
    Gaussians fitted to 35 dB by the ROI-initialised encoder), shipped with the
    package as BF16 weights; None for other sizes."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), PACKAGED)
    if not os.path.exists(path):
        return None
    st = dict(np.load(path))
    meta = json.loads(bytes(st.pop("meta")).decode())
    if (meta["width"], meta["height"], meta["n"]) != (width, height, n):
        return None
    net = LearnedInitializer(width, height, n, batch,
                             NetConfig(channels=tuple(meta["channels"]), slots=meta["slots"],
                                       scale=meta["scale"]), device=device)
    net.load_state(st)
    return net


class Trainer:
    """Fits the initialiser to (frame, mask, encoder-fitted Gaussians) triples
    with the render loss through the rasterizer plus the Chamfer term."""

    def __init__(self, net: LearnedInitializer, raster_config: RasterConfig | None = None):
        self.net = net
        B, n = net.B, net.n
        self.rast = BatchRasterizer([(net.W, net.H, n)] * B, config=raster_config,
                                    device=net.dev)
        self.chamfer_scratch = torch.empty(
            nat.load().gs2d_chamfer_scratch_bytes(n, n, B), dtype=torch.uint8, device=net.dev)
        self.chamfer_loss = torch.empty(B, device=net.dev)

    def step(self, frames: torch.Tensor, masks, targets: torch.Tensor):
        """frames [B, 3, H, W]; targets: encoder-fitted Gaussians [9, B n].
        Returns (render loss = sum over frames of MSE, mean Chamfer)."""
        net = self.net
        params = net.forward(frames, masks)
        flat = frames.reshape(-1)
        self.rast.prepare(params)
        grads, loss, _ = self.rast.render_l2(params, flat)
        s = int(torch.cuda.current_stream().cuda_stream)
        nat.call("gs2d_chamfer", params.data_ptr(), net.n, net.B * net.n, targets.data_ptr(),
                 net.n, net.B * net.n, net.B, net.cfg.chamfer_lambda, grads.data_ptr(),
                 self.chamfer_loss.data_ptr(), self.chamfer_scratch.data_ptr(), s)
        net.backward(grads)
        net.step()
        return loss, self.chamfer_loss


# ---------------------------------------------------------------------------
# Data, training and evaluation (the learned-initialiser workload: frames of
# the synthetic conferencing scene, Gaussians fitted by the encoder to 35 dB)

def _frame_job(args):
    """Synthetic frame and mask (runs in a spawned worker process)."""
    from gs2d_inputs import conferencing_frame
    W, H, seed = args
    f, m = conferencing_frame(W, H, seed=seed)
    return f.astype(np.float16), m


class FrameSource:
    """Frames of the given seeds from a pool of spawned workers, in order."""

    def __init__(self, W: int, H: int, seeds, workers: int = 0):
        import multiprocessing as mp
        import os
        self.W, self.H, self.seeds = W, H, list(seeds)
        self.workers = workers or max(1, min(14, (os.cpu_count() or 2) - 2))
        self.pool = mp.get_context("spawn").Pool(self.workers)

    def __iter__(self):
        jobs = [(self.W, self.H, s) for s in self.seeds]
        yield from self.pool.imap(_frame_job, jobs, chunksize=2)

    def close(self):
        self.pool.close()
        self.pool.join()


@dataclasses.dataclass
class Dataset:
    frames: torch.Tensor    # [F, 3, H, W] float16
    masks: torch.Tensor     # [F, H, W] uint8
    targets: torch.Tensor   # [F, 9, n] float32, encoder-fitted Gaussians
    iters: list             # encoder iterations per frame
    seconds: float


def make_dataset(W: int, H: int, n: int, seeds, target_psnr: float = 35.0, cap: int = 2000,
                 roi_frac: float = 0.7, device=None, log=None) -> Dataset:
    """(frame, mask, fitted Gaussians) for every seed: ROI initialisation then
    the encoder to `target_psnr` (at most `cap` iterations)."""
    import time
    from gs2d_inputs import background_positions
    from .raster import GaussianRasterizer, roi_init
    dev = torch.device(device) if device is not None else torch.device("cuda")
    F = len(seeds)
    frames = torch.empty((F, 3, H, W), dtype=torch.float16, device=dev)
    masks = torch.empty((F, H, W), dtype=torch.uint8, device=dev)
    targets = torch.empty((F, 9, n), device=dev)
    rast = GaussianRasterizer(W, H, n, device=dev)
    side = torch.cuda.Stream(dev)
    iters = []
    src = FrameSource(W, H, seeds)
    t0 = time.perf_counter()
    try:
        for i, (f16, m) in enumerate(src):
            fr = torch.from_numpy(f16).to(dev).float()
            mk = torch.from_numpy(m.astype(np.uint8)).to(dev)
            bg = torch.from_numpy(background_positions(m, n, seed=seeds[i] + 10)).to(dev)
            p, _ = roi_init(fr, mk, n, roi_frac, bg)
            with torch.cuda.stream(side):
                r = rast.encode_frame(fr, p, cap, target_psnr=target_psnr, check_every=25,
                                      stream=side)
            side.synchronize()
            frames[i] = fr.half()
            masks[i] = mk
            targets[i] = p
            iters.append(r["iters"])
            if log and (i + 1) % 250 == 0:
                log(f"dataset {i + 1}/{F} frames, {time.perf_counter() - t0:.0f} s")
    finally:
        src.close()
    return Dataset(frames, masks, targets, iters, time.perf_counter() - t0)


def batch_targets(t: torch.Tensor) -> torch.Tensor:
    """[B, 9, n] -> [9, B n] (the batch layout)."""
    return t.permute(1, 0, 2).reshape(9, -1).contiguous()


def train(net: LearnedInitializer, data: Dataset, epochs: int, seed: int = 0, log=None):
    import time
    trainer = Trainer(net)
    g = np.random.Generator(np.random.PCG64(seed))
    F, B = data.frames.shape[0], net.B
    hist = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = g.permutation(F)
        rl, cl, k = 0.0, 0.0, 0
        for j in range(0, F - B + 1, B):
            idx = torch.from_numpy(order[j:j + B]).to(data.frames.device)
            loss, ch = trainer.step(data.frames[idx].float(), data.masks[idx],
                                    batch_targets(data.targets[idx]))
            rl += float(loss[0])
            cl += float(ch.mean())
            k += 1
        net.check_status()
        hist.append({"epoch": ep, "render_mse_per_frame": rl / max(k, 1) / B,
                     "chamfer": cl / max(k, 1), "seconds": time.perf_counter() - t0})
        if log:
            log(f"epoch {ep}: {hist[-1]}")
    return hist


def evaluate(net: LearnedInitializer, seeds, target_psnr: float = 35.0, cap: int = 2000,
             roi_frac: float = 0.7, log=None) -> dict:
    """Iterations and seconds to target_psnr from the learned initialiser and
    from the ROI initialiser on held-out frames, and PSNR after 0, 100, 500
    iterations, at equal Gaussian count."""
    import time
    from gs2d_inputs import background_positions
    from .raster import GaussianRasterizer, roi_init
    dev, B, n, W, H = net.dev, net.B, net.n, net.W, net.H
    rast = GaussianRasterizer(W, H, n, device=dev)
    side = torch.cuda.Stream(dev)
    rec = {"learned": [], "roi": []}
    src = FrameSource(W, H, seeds)
    buf_f, buf_m = [], []

    def fit(frame, p0, init_s):
        out = {"init_s": init_s}
        p = p0.clone()
        rast.prepare(p)
        _, l0, _ = rast.render_l2(p, frame)
        mse0 = float(l0[1])
        out["psnr0"] = 10 * np.log10(1 / mse0) if mse0 > 0 else float("inf")
        if out["psnr0"] >= target_psnr:  # the initialiser alone reaches the target
            out.update(iters=0, psnr=out["psnr0"], reached=True, fit_s=0.0)
        else:
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            with torch.cuda.stream(side):
                r = rast.encode_frame(frame, p, cap, target_psnr=target_psnr, check_every=25,
                                      stream=side)
            side.synchronize()
            out.update(iters=r["iters"], psnr=r["psnr"], reached=r["psnr"] >= target_psnr,
                       fit_s=time.perf_counter() - t0)
        q = p0.clone()
        with torch.cuda.stream(side):
            r2 = rast.encode_frame(frame, q, 500, target_psnr=0.0, check_every=100, stream=side)
        side.synchronize()
        out["psnr100"], out["psnr500"] = r2["trace"][0], r2["trace"][4]
        return out

    try:
        for f16, m in src:
            buf_f.append(torch.from_numpy(f16).to(dev).float())
            buf_m.append(torch.from_numpy(m.astype(np.uint8)).to(dev))
            if len(buf_f) < B:
                continue
            frames = torch.stack(buf_f)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            P = net.forward(frames, torch.stack(buf_m), keep_col=False).clone()
            torch.cuda.synchronize(dev)
            per = (time.perf_counter() - t0) / B
            for b in range(B):
                rec["learned"].append(fit(buf_f[b], P[:, b * n:(b + 1) * n].contiguous(), per))
                mnp = buf_m[b].cpu().numpy().astype(bool)
                bg = torch.from_numpy(
                    background_positions(mnp, n, seed=len(rec["roi"]) + 7)).to(dev)
                torch.cuda.synchronize(dev)
                t1 = time.perf_counter()
                q, _ = roi_init(buf_f[b], buf_m[b], n, roi_frac, bg)
                torch.cuda.synchronize(dev)
                rec["roi"].append(fit(buf_f[b], q, time.perf_counter() - t1))
            buf_f, buf_m = [], []
            if log:
                log(f"evaluated {len(rec['roi'])} frames")
    finally:
        src.close()

    def summary(rs):
        it = np.array([r["iters"] for r in rs], float)
        tot = np.array([r["init_s"] + r["fit_s"] for r in rs])
        return {"frames": len(rs), "reached": int(sum(r["reached"] for r in rs)),
                "iters_mean": float(it.mean()), "iters_median": float(np.median(it)),
                "s_per_frame_mean": float(tot.mean()),
                "init_ms_mean": 1e3 * float(np.mean([r["init_s"] for r in rs])),
                "psnr0_mean": float(np.mean([r["psnr0"] for r in rs])),
                "psnr100_mean": float(np.mean([r["psnr100"] for r in rs])),
                "psnr500_mean": float(np.mean([r["psnr500"] for r in rs]))}

    return {"learned": summary(rec["learned"]), "roi": summary(rec["roi"]),
            "target_psnr": target_psnr, "cap": cap}


def main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="train and evaluate the learned initialiser")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--train-frames", type=int, default=5000)
    ap.add_argument("--eval-frames", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--chamfer-lambda", type=float, default=1e-5)
    ap.add_argument("--out", default="learned_init.json")
    ap.add_argument("--weights", default="", help="write the trained weights (.npz)")
    ap.add_argument("--load", default="", help="start from these weights (.npz)")
    ap.add_argument("--eval-only", action="store_true")
    ap.add_argument("--time-forward", action="store_true",
                    help="time the shipped network's forward (with and without im2col "
                         "operands: 3 warm-up + 20 timed calls each) and exit")
    a = ap.parse_args(argv)

    def log(msg):
        print(msg, flush=True)

    from . import build
    build.build()
    nat.load()
    if a.time_forward:
        from gs2d_inputs import conferencing_frame
        net = packaged(a.width, a.height, a.n, a.batch) or \
            LearnedInitializer(a.width, a.height, a.n, a.batch)
        fr = [conferencing_frame(a.width, a.height, seed=1 + b) for b in range(a.batch)]
        frames = torch.from_numpy(np.stack([f for f, _ in fr])).cuda()
        masks = torch.from_numpy(np.stack([m for _, m in fr]).astype(np.uint8)).cuda()
        out = {}
        for keep in (True, False):
            for _ in range(3):
                net.forward(frames, masks, keep_col=keep)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                net.forward(frames, masks, keep_col=keep)
            e1.record()
            torch.cuda.synchronize()
            out["ms_im2col" if keep else "ms_implicit"] = e0.elapsed_time(e1) / 20
        net.check_status()
        print(json.dumps({"batch": a.batch, **out}))
        return 0
    t0 = time.perf_counter()
    train_seeds = [10000 + i for i in range(a.train_frames)]
    eval_seeds = [20000 + i for i in range(a.eval_frames)]
    net = LearnedInitializer(a.width, a.height, a.n, a.batch,
                             NetConfig(lr=a.lr, chamfer_lambda=a.chamfer_lambda))
    if a.load:
        net.load_state(dict(np.load(a.load)))
    hist = []
    if not a.eval_only:
        data = make_dataset(a.width, a.height, a.n, train_seeds, log=log)
        log(f"dataset: {len(train_seeds)} frames in {data.seconds:.0f} s, encoder iterations "
            f"mean {np.mean(data.iters):.0f}")
        hist = train(net, data, a.epochs, log=log)
        del data
        torch.cuda.empty_cache()
    res = evaluate(net, eval_seeds, log=log)
    res.update(params=net.num_params(), history=hist, train_frames=len(train_seeds),
               eval_frames=len(eval_seeds), batch=a.batch, total_s=time.perf_counter() - t0)
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    if a.weights:
        np.savez(a.weights, **net.state())
    log(json.dumps({k: res[k] for k in ("learned", "roi")}))


if __name__ == "__main__":
    main()
