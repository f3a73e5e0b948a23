"""CPU oracle for the 2D Gaussian rasterizer -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The product path (``paper_2505_09324_gb300``) never
imports it and shares no code with it; the only module both sides use is
``gs2d_inputs`` (seeded input generation, no method arithmetic).

Contents (each function cites the passage of arXiv 2505.09324 it follows):

* ``render`` / ``render_pixels`` -- brute-force Eq. 2 in double precision
  (``gs2d_oracle.c``).
* ``render_grad`` -- analytic gradients of a loss through Eq. 2 with respect
  to the factorised parameters of Sec. 3.1 (Eq. 1), double precision.
* ``l2_loss`` / ``psnr`` -- the L2 fitting loss and the PSNR used to judge the
  fit (Sec. 4 reports PSNR targets).
* ``tile_rects`` / ``sorted_keys`` -- the tile binning of the tile-based
  rasterizer (Sec. 3: "differentiable tile-based rasterization"), single
  precision, and the sorted (tile, index) list with per-tile ranges.
* ``adam_step`` -- one Adam step (the paper's "optimization steps", Sec. 4.1;
  the optimiser is a project reading: Adam with bias correction, constant lr).

Parity pins for each function live in ``tests/test_oracle_*.py``.  Functions
without such a pin are marked "parity unpinned" in their docstring.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs2d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgs2d_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (``-ffp-contract=off``: no FMA contraction,
    so single-precision binning is reproducible on x86-64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.orc_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int,
                                       P, P, P]
            lib.orc_render_pixels.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P, P]
            lib.orc_render_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P,
                                            ctypes.c_int, P, P, P, ctypes.c_int, P, P]
            lib.orc_tile_rects.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           P, ctypes.c_float, ctypes.c_float, ctypes.c_float, P,
                                           P, P]
            lib.orc_sorted_keys.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            P, i64, P, P]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            for f in (lib.orc_render, lib.orc_render_pixels, lib.orc_render_grad,
                      lib.orc_tile_rects, lib.orc_sorted_keys, lib.orc_set_threads):
                f.restype = ctypes.c_int
            del i32
            _lib = lib
    return _lib


@dataclasses.dataclass(frozen=True)
class Config:
    """Contribution predicate constants (project readings; the paper gives none).

    sigma_cut: the 3-sigma ellipse (sigma <= 4.5); alpha_min: |alpha| >= 1/255;
    det_eps: minimum det Sigma; amb_tol: half-width of the band around tau in
    which a single-precision predicate may legitimately differ.
    """

    sigma_cut: float = 4.5
    alpha_min: float = 1.0 / 255.0
    det_eps: float = 1e-8
    amb_tol: float = 1e-4
    tile: int = 16


class _CCfg(ctypes.Structure):
    _fields_ = [("sigma_cut", ctypes.c_double), ("alpha_min", ctypes.c_double),
                ("det_eps", ctypes.c_double), ("amb_tol", ctypes.c_double)]


def _ccfg(cfg: Config) -> _CCfg:
    return _CCfg(cfg.sigma_cut, cfg.alpha_min, cfg.det_eps, cfg.amb_tol)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _params64(params) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if p.ndim != 2 or p.shape[0] != 9:
        raise ValueError("params must have shape [9, n]")
    return p


def set_threads(k: int = 0) -> int:
    """Set the OpenMP thread count (k <= 0 leaves it); returns the count in use."""
    return int(_load().orc_set_threads(int(k)))


def render(params, width: int, height: int, cfg: Config = Config(), fast: bool = False,
           ambiguity: bool = False):
    """Eq. 2 (Sec. 3.1) by brute force: every pixel against every Gaussian in
    ascending index order, double precision, no tiling.

    Returns ``img[3, H, W]`` (float64) or, with ``ambiguity``, ``(img, lo, hi)``
    where ``img + lo <= C_true <= img + hi`` covers every pair whose predicate a
    single-precision evaluation could decide either way.  ``fast`` restricts each
    Gaussian to its ellipse bounding box (exact by the ellipse bound).
    """
    p = _params64(params)
    n = p.shape[1]
    img = np.zeros((3, height, width), np.float64)
    lo = np.zeros_like(img) if ambiguity else None
    hi = np.zeros_like(img) if ambiguity else None
    c = _ccfg(cfg)
    rc = _load().orc_render(width, height, n, _ptr(p), ctypes.byref(c), int(fast), _ptr(img),
                            _ptr(lo), _ptr(hi))
    if rc != 0:
        raise RuntimeError(f"orc_render failed ({rc})")
    return (img, lo, hi) if ambiguity else img


def render_pixels(params, xy, cfg: Config = Config(), ambiguity: bool = False):
    """Eq. 2 at the listed integer pixels ``xy[k] = (x, y)``; returns ``[3, k]``."""
    p = _params64(params)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    k = xy.shape[0]
    out = np.zeros((3, k), np.float64)
    lo = np.zeros_like(out) if ambiguity else None
    hi = np.zeros_like(out) if ambiguity else None
    c = _ccfg(cfg)
    rc = _load().orc_render_pixels(p.shape[1], _ptr(p), ctypes.byref(c), k, _ptr(xy), _ptr(out),
                                   _ptr(lo), _ptr(hi))
    if rc != 0:
        raise RuntimeError(f"orc_render_pixels failed ({rc})")
    return (out, lo, hi) if ambiguity else out


def render_grad(params, width: int, height: int, dimg, cfg: Config = Config(), fast: bool = False,
                dimg_unc=None, which=None, uncertainty: bool = False):
    """Gradient of a loss with respect to the ``[9, n]`` parameters given
    ``dimg = dL/dC`` (``[3, H, W]``), through Eq. 2 and Eq. 1 (Sec. 3.1).

    With ``uncertainty`` also returns a bound on how far a correct FP32
    implementation may deviate (ambiguous pairs, plus ``dimg_unc`` propagated to
    first order).  ``which`` restricts the computation to a subset of Gaussians.
    """
    p = _params64(params)
    n = p.shape[1]
    g = np.ascontiguousarray(np.asarray(dimg, dtype=np.float64))
    if g.shape != (3, height, width):
        raise ValueError("dimg must have shape [3, H, W]")
    gu = None if dimg_unc is None else np.ascontiguousarray(np.asarray(dimg_unc, np.float64))
    wh = None if which is None else np.ascontiguousarray(np.asarray(which, dtype=np.int32))
    grad = np.zeros((9, n), np.float64)
    unc = np.zeros((9, n), np.float64) if uncertainty else None
    c = _ccfg(cfg)
    rc = _load().orc_render_grad(width, height, n, _ptr(p), ctypes.byref(c), int(fast), _ptr(g),
                                 _ptr(gu), _ptr(wh), 0 if wh is None else len(wh), _ptr(grad),
                                 _ptr(unc))
    if rc != 0:
        raise RuntimeError(f"orc_render_grad failed ({rc})")
    return (grad, unc) if uncertainty else grad


def l2_loss(img, target):
    """L2 fitting loss L = mean over 3HW of (C - T)^2 and dL/dC = 2 (C - T)/(3HW)
    (project reading: the paper fits with an L2 objective and reports PSNR)."""
    d = np.asarray(img, np.float64) - np.asarray(target, np.float64)
    m = d.size
    return float(np.sum(d * d) / m), 2.0 * d / m


def loss_and_grad(params, target, cfg: Config = Config(), fast: bool = False, which=None):
    """L2 loss of the oracle render against ``target`` and its parameter
    gradient, with the FP32 uncertainty bound (ambiguous pairs change C, which
    changes dL/dC, which is propagated into the gradient bound)."""
    target = np.asarray(target, np.float64)
    _, h, w = target.shape
    img, lo, hi = render(params, w, h, cfg, fast=fast, ambiguity=True)
    loss, g = l2_loss(img, target)
    m = img.size
    g_unc = 2.0 * np.maximum(-lo, hi) / m
    grad, unc = render_grad(params, w, h, g, cfg, fast=fast, dimg_unc=g_unc, which=which,
                            uncertainty=True)
    return {"loss": loss, "img": img, "amb_lo": lo, "amb_hi": hi, "dimg": g, "grad": grad,
            "grad_unc": unc}


def psnr(img, target) -> float:
    """PSNR in dB of an image clamped to [0, 1] against a target with peak 1."""
    c = np.clip(np.asarray(img, np.float64), 0.0, 1.0)
    mse = float(np.mean((c - np.asarray(target, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


def tile_rects(params, width: int, height: int, cfg: Config = Config()):
    """Single-precision tile rectangle ``[tx0, ty0, tx1, ty1)`` and tile count of
    every Gaussian (the binning step of tile-based rasterization, Sec. 3)."""
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    n = p.shape[1]
    rect = np.zeros((n, 4), np.int32)
    count = np.zeros(n, np.int32)
    total = ctypes.c_int64(0)
    rc = _load().orc_tile_rects(width, height, cfg.tile, n, _ptr(p), np.float32(cfg.sigma_cut),
                                np.float32(cfg.alpha_min), np.float32(cfg.det_eps), _ptr(rect),
                                _ptr(count), ctypes.byref(total))
    if rc != 0:
        raise RuntimeError(f"orc_tile_rects failed ({rc})")
    return rect, count, int(total.value)


def sorted_keys(params, width: int, height: int, cfg: Config = Config()):
    """All (tile, index) pairs as ``key = tile << 32 | index`` sorted ascending,
    plus per-tile ``[start, end)`` ranges into that list (shape ``[tiles, 2]``)."""
    rect, count, total = tile_rects(params, width, height, cfg)
    t = cfg.tile
    tiles = ((width + t - 1) // t) * ((height + t - 1) // t)
    keys = np.zeros(max(total, 1), np.uint64)
    ranges = np.zeros((tiles, 2), np.int32)
    rc = _load().orc_sorted_keys(width, height, t, rect.shape[0], _ptr(rect), total, _ptr(keys),
                                 _ptr(ranges))
    if rc != 0:
        raise RuntimeError(f"orc_sorted_keys failed ({rc})")
    return keys[:total], ranges


def adam_step(p, g, m, v, step: int, lr: float = 1e-2, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step with bias correction (Kingma & Ba 2015, Algorithm 1), in
    double precision.  ``step`` is 1-based.  Returns new ``(p, m, v)``.
    The paper names no optimiser; Adam with a constant learning rate is the
    project reading of its "optimization steps" (Sec. 4.1)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def contributes(params, xy, cfg: Config = Config()):
    """Which Gaussians contribute to Eq. 2 at the integer pixels ``xy[k] = (x, y)``
    (the cut-off predicate of the notation above, double precision, pixel
    centres at +0.5): ``(definite [k, n], ambiguous [k, n])`` boolean arrays,
    ambiguous where sigma lies within amb_tol max(1, tau) of tau (a single
    precision evaluation may decide those either way)."""
    p = _params64(params)
    mx, my, l1, l2, l3 = p[0], p[1], p[2], p[3], p[4]
    w = p[8]
    sxx, sxy, syy = l1 * l1, l1 * l2, l2 * l2 + l3 * l3
    det = sxx * syy - sxy * sxy
    finite = np.all(np.isfinite(p), axis=0)
    ok = finite & (det > cfg.det_eps) & (np.abs(w) >= cfg.alpha_min)
    with np.errstate(divide="ignore", invalid="ignore"):
        tau = np.minimum(cfg.sigma_cut, np.log(np.abs(w) / cfg.alpha_min))
        a, b, c = syy / det, -sxy / det, sxx / det
    xy = np.asarray(xy, np.float64).reshape(-1, 2)
    dx = (xy[:, 0:1] + 0.5) - mx[None, :]
    dy = (xy[:, 1:2] + 0.5) - my[None, :]
    with np.errstate(invalid="ignore"):
        sig = 0.5 * (a * dx * dx + c * dy * dy) + b * dx * dy
    band = cfg.amb_tol * np.maximum(1.0, tau)
    definite = ok[None, :] & (sig <= tau - band)
    ambiguous = ok[None, :] & (np.abs(sig - tau) < band)
    return definite, ambiguous
