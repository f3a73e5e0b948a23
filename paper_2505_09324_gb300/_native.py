"""ctypes binding of libgs2d (include/gs2d.h).  Argument marshalling only: every
step of the rasterizer runs in the library's CUDA kernels.  Importing this
module does not touch the GPU; the first call loads the library and raises if
it is missing (there is no fallback implementation)."""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

GS2D_OK = 0
GS2D_ERR_INVALID_ARG = 1
GS2D_ERR_CUDA = 2
GS2D_ERR_CAPACITY = 3
GS2D_ERR_TIMEOUT = 4
GS2D_ERR_BOUNDS = 5
STATUS_NAMES = {0: "GS2D_OK", 1: "GS2D_ERR_INVALID_ARG", 2: "GS2D_ERR_CUDA",
                3: "GS2D_ERR_CAPACITY", 4: "GS2D_ERR_TIMEOUT", 5: "GS2D_ERR_BOUNDS"}

# every function declared in include/gs2d.h
EXPORTS = (
    "gs2d_config_default", "gs2d_sizeof_plan", "gs2d_sizeof_config", "gs2d_plan_init",
    "gs2d_plan_init_batch", "gs2d_ws_set_clips",
    "gs2d_project", "gs2d_bin_sort", "gs2d_prepare", "gs2d_render_fwd", "gs2d_render_fwd_noalloc",
    "gs2d_render_bwd", "gs2d_render_l2",
    "gs2d_adam_step", "gs2d_fit_step", "gs2d_fit_reset", "gs2d_encode_frame", "gs2d_clip_losses",
    "gs2d_select_changed", "gs2d_pframe_step", "gs2d_encode_pframe", "gs2d_quantize",
    "gs2d_fit_step_qat", "gs2d_code_entropy_scratch_bytes", "gs2d_code_entropy",
    "gs2d_sequence_bits", "gs2d_frame_from_rgb8", "gs2d_conv_bf16", "gs2d_fit_step_rgb8",
    "gs2d_fit_rebins", "gs2d_fit_state_get", "gs2d_fit_state_set",
    "gs2d_encode_batch",
    "gs2d_autotune_ws_bytes", "gs2d_autotune",
    "gs2d_gemm_bf16", "gs2d_gemm_partial_bytes", "gs2d_cnn_input", "gs2d_conv_frame_bf16",
    "gs2d_conv_wait_check", "gs2d_im2col", "gs2d_col2im",
    "gs2d_transpose_bf16", "gs2d_relu_bwd", "gs2d_cast_weights", "gs2d_head_decode",
    "gs2d_head_smem_bytes", "gs2d_head_decode_bwd", "gs2d_chamfer", "gs2d_chamfer_scratch_bytes",
    "gs2d_read_bins", "gs2d_count_pairs", "gs2d_ws_status",
    "gs2d_roi_init_scratch_bytes", "gs2d_roi_init", "gs2d_roi_init_trace",
    "gs2d_probe_ops", "gs2d_probe_peak", "gs2d_gemm_wait_check",
    "gs2d_quant_calibrate_scratch_bytes", "gs2d_quant_calibrate",
    "gs2d_frame_bits_scratch_bytes", "gs2d_frame_bits",
    "gs2d_last_error",
)


class Gs2dError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("sigma_cut", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("det_eps", ctypes.c_float),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("stage", ctypes.c_int32), ("launch", ctypes.c_int32),
                ("lr_mu", ctypes.c_float), ("lr_shape", ctypes.c_float),
                ("lr_color", ctypes.c_float), ("lr_weight", ctypes.c_float),
                ("lr_decay", ctypes.c_float), ("bin_margin", ctypes.c_float),
                ("reduce", ctypes.c_int32)]


LAUNCH_PERSISTENT = 0
LAUNCH_GRID = 1
REDUCE_SLOTS = 0
REDUCE_ATOMIC = 1


class Clip(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n", ctypes.c_int32),
                ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
                ("g_off", ctypes.c_int32), ("tile_off", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("pix_off", ctypes.c_int64)]


class FitState(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("beta1_pow", ctypes.c_double), ("beta2_pow", ctypes.c_double),
                ("decay_pow", ctypes.c_double)]


class Quant(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_int32 * 9), ("refine", ctypes.c_int32),
                ("lo", ctypes.c_float * 9),
                ("hi", ctypes.c_float * 9), ("scale", ctypes.c_float * 9),
                ("step", ctypes.c_float * 9)]


class SeqBits(ctypes.Structure):
    _fields_ = [("i_bits", ctypes.c_double), ("p_bits", ctypes.c_double),
                ("savings", ctypes.c_double), ("total_bits", ctypes.c_double),
                ("i_frames", ctypes.c_int32), ("p_frames", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("tiles_x", ctypes.c_int32),
                ("tiles_y", ctypes.c_int32), ("num_tiles", ctypes.c_int32),
                ("tile_bits", ctypes.c_int32), ("num_clips", ctypes.c_int32),
                ("stage", ctypes.c_int32), ("max_entries", ctypes.c_int64),
                ("pixels", ctypes.c_int64),
                ("cfg", Config), ("ws_bytes", ctypes.c_uint64), ("off", ctypes.c_uint64 * 24),
                ("magic", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libgs2d.so (building it first only if asked)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    f"libgs2d.so not found at {path}; build it with "
                    "paper_2505_09324_gb300.build.build() (the CUDA library is required)")
            _build.build()
        lib = ctypes.CDLL(path)
        P, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        pp = ctypes.POINTER(Plan)
        pc = ctypes.POINTER(Clip)
        pcfg = ctypes.POINTER(Config)
        sig = {
            "gs2d_config_default": (None, [ctypes.POINTER(Config)]),
            "gs2d_sizeof_plan": (ctypes.c_size_t, []),
            "gs2d_sizeof_config": (ctypes.c_size_t, []),
            "gs2d_plan_init": (i32, [pp, i32, i32, i32, i64, ctypes.POINTER(Config)]),
            "gs2d_plan_init_batch": (i32, [pp, pc, i32, i64, pcfg]),
            "gs2d_ws_set_clips": (i32, [pp, P, pc, P]),
            "gs2d_clip_losses": (i32, [pp, P, P, P]),
            "gs2d_encode_batch": (i32, [pp, P, P, P, P, P, i32, P, P]),
            "gs2d_autotune_ws_bytes": (ctypes.c_uint64, [pc, i32, i64, pcfg, P, i32]),
            "gs2d_autotune": (i32, [pc, i32, i64, pcfg, P, P, P, ctypes.c_uint64, P, i32, P, i32,
                                    P, i32, i32, P, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), P]),
            "gs2d_project": (i32, [pp, P, P, P]),
            "gs2d_bin_sort": (i32, [pp, P, P]),
            "gs2d_prepare": (i32, [pp, P, P, P]),
            "gs2d_render_fwd": (i32, [pp, P, P, P]),
            "gs2d_render_fwd_noalloc": (i32, [P, i32, i32, i32, ctypes.POINTER(Config), P, P,
                                              P]),
            "gs2d_render_bwd": (i32, [pp, P, P, P, P, P]),
            "gs2d_render_l2": (i32, [pp, P, P, P, P, P, P, P]),
            "gs2d_adam_step": (i32, [P, P, P, P, i64, i32, P, ctypes.POINTER(Config), P]),
            "gs2d_encode_frame": (i32, [pp, P, P, P, P, P, i32, f32, i32, P, P, P, P]),
            "gs2d_fit_step": (i32, [pp, P, P, P, P, P, P]),
            "gs2d_fit_reset": (i32, [pp, P, P, P, P]),
            "gs2d_select_changed": (i32, [pp, P, P, P, f32, P, ctypes.POINTER(i32), P]),
            "gs2d_pframe_step": (i32, [pp, P, P, P, P, P, P, P]),
            "gs2d_encode_pframe": (i32, [pp, P, P, P, P, P, P, i32, ctypes.POINTER(f32), P]),
            "gs2d_quantize": (i32, [P, i32, ctypes.POINTER(Quant), P, P, P, P]),
            "gs2d_fit_step_qat": (i32, [pp, P, P, P, P, P, ctypes.POINTER(Quant), P]),
            "gs2d_code_entropy_scratch_bytes": (ctypes.c_size_t, []),
            "gs2d_frame_from_rgb8": (i32, [P, i32, i32, i64, P, P]),
            "gs2d_fit_step_rgb8": (i32, [pp, P, P, P, P, P, P, P, P, P, P]),
            "gs2d_fit_rebins": (i32, [pp, P, ctypes.POINTER(i64), P]),
            "gs2d_fit_state_get": (i32, [pp, P, ctypes.POINTER(FitState), P]),
            "gs2d_fit_state_set": (i32, [pp, P, ctypes.POINTER(FitState), P]),
            "gs2d_conv_bf16": (i32, [P, i32, i32, i32, i32, i32, i32, i32, P, i32, i32, i32, P,
                                     P, i32, P, P]),
            "gs2d_code_entropy": (i32, [P, i32, ctypes.POINTER(i32), P, P, ctypes.c_size_t, P,
                                        P]),
            "gs2d_sequence_bits": (i32, [ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                         i32, i32, ctypes.POINTER(SeqBits)]),
            "gs2d_read_bins": (i32, [pp, P, P, P, P, i64, P, P, P]),
            "gs2d_count_pairs": (i32, [pp, P, ctypes.POINTER(i64), ctypes.POINTER(i64), P]),
            "gs2d_ws_status": (i32, [pp, P, i32, P]),
            "gs2d_roi_init_scratch_bytes": (ctypes.c_uint64, [i32, i32, i32]),
            "gs2d_roi_init": (i32, [P, P, i32, i32, i32, f32, P, P, ctypes.POINTER(i32), P,
                                    ctypes.c_uint64, P]),
            "gs2d_roi_init_trace": (i32, [P, P, i32, i32, i32, f32, P, P, ctypes.POINTER(i32),
                                          P, ctypes.c_uint64, P, P, P]),
            "gs2d_last_error": (i32, [ctypes.c_char_p, ctypes.c_size_t]),
            "gs2d_probe_ops": (i64, [i32, i32]),
            "gs2d_probe_peak": (i32, [i32, i32, i32, P, P]),
            "gs2d_gemm_wait_check": (i32, [P, P, P, P, ctypes.c_uint64, P]),
            "gs2d_quant_calibrate_scratch_bytes": (ctypes.c_size_t, []),
            "gs2d_frame_bits_scratch_bytes": (ctypes.c_size_t, []),
            "gs2d_frame_bits": (i32, [P, i32, ctypes.POINTER(i32), P, i32, P, ctypes.c_size_t, P,
                                      P]),
            "gs2d_quant_calibrate": (i32, [P, i32, ctypes.POINTER(i32), ctypes.c_double, P,
                                           ctypes.c_size_t,
                                           ctypes.POINTER(f32), ctypes.POINTER(f32), P]),
            "gs2d_gemm_bf16": (i32, [P, i32, P, i32, i32, i32, i32, P, i32, P, P, i32, i32, P, P,
                                     P]),
            "gs2d_gemm_partial_bytes": (ctypes.c_uint64, [i32, i32, i32, i32, i32]),
            "gs2d_cnn_input": (i32, [P, P, i32, i32, i32, P, P]),
            "gs2d_conv_wait_check": (i32, [i32, P, P, P, P, ctypes.c_uint64, P]),
            "gs2d_conv_frame_bf16": (i32, [P, P, i32, i32, i32, i32, i32, i32, P, i32, i32, i32, P,
                                           P, i32, P, P]),
            "gs2d_im2col": (i32, [P, i32, i32, i32, i32, i32, i32, i32, P, i32, P]),
            "gs2d_col2im": (i32, [P, i32, i32, i32, i32, i32, i32, i32, i32, P, P, P]),
            "gs2d_transpose_bf16": (i32, [P, i32, i32, i32, P, i32, P]),
            "gs2d_relu_bwd": (i32, [P, i32, i32, i32, P, i32, P, i32, P]),
            "gs2d_cast_weights": (i32, [P, i32, i32, P, P, P]),
            "gs2d_head_decode": (i32, [P, i32, i32, i32, i32, i32, i32, f32, i32, P, i32, P, P]),
            "gs2d_head_smem_bytes": (ctypes.c_uint64, [i32, i32, i32]),
            "gs2d_head_decode_bwd": (i32, [P, i32, i32, i32, i32, i32, i32, f32, i32, P, P, i32,
                                           P, P]),
            "gs2d_chamfer": (i32, [P, i32, i32, P, i32, i32, i32, f32, P, P, P, P]),
            "gs2d_chamfer_scratch_bytes": (ctypes.c_uint64, [i32, i32, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if lib.gs2d_sizeof_plan() != ctypes.sizeof(Plan):
            raise RuntimeError("gs2d_plan layout mismatch between library and binding")
        if lib.gs2d_sizeof_config() != ctypes.sizeof(Config):
            raise RuntimeError("gs2d_config layout mismatch between library and binding")
        _lib = lib
        return lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load().gs2d_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int, what: str = ""):
    if status != GS2D_OK:
        raise Gs2dError(status, f"{what}: {last_error()}")


def default_config() -> Config:
    c = Config()
    load().gs2d_config_default(ctypes.byref(c))
    return c


def plan_init(width: int, height: int, n: int, max_entries: int = 0,
              config: Config | None = None) -> Plan:
    p = Plan()
    cfg = ctypes.byref(config) if config is not None else None
    check(load().gs2d_plan_init(ctypes.byref(p), width, height, n, max_entries, cfg),
          "gs2d_plan_init")
    return p


def plan_init_batch(sizes, max_entries: int = 0, config: Config | None = None):
    """sizes: sequence of (width, height, n).  Returns (plan, clips array)."""
    clips = (Clip * len(sizes))()
    for k, (w, h, n) in enumerate(sizes):
        clips[k].width, clips[k].height, clips[k].n = int(w), int(h), int(n)
    p = Plan()
    cfg = ctypes.byref(config) if config is not None else None
    check(load().gs2d_plan_init_batch(ctypes.byref(p), clips, len(sizes), max_entries, cfg),
          "gs2d_plan_init_batch")
    return p, clips


def ws_set_clips(plan: Plan, ws: int, clips, stream: int):
    check(load().gs2d_ws_set_clips(ctypes.byref(plan), _p(ws), clips, _p(stream)),
          "gs2d_ws_set_clips")


def clip_losses(plan: Plan, ws: int, stream: int):
    """[(mse, clamped mse)] per clip of the last render_l2."""
    out = (ctypes.c_float * (2 * plan.num_clips))()
    check(load().gs2d_clip_losses(ctypes.byref(plan), _p(ws), out, _p(stream)),
          "gs2d_clip_losses")
    return [(out[2 * k], out[2 * k + 1]) for k in range(plan.num_clips)]


def encode_batch(plan: Plan, ws: int, targets: int, params: int, m: int, v: int, iters: int,
                 stream: int):
    """Returns the per-clip PSNR list after `iters` iterations."""
    out = (ctypes.c_float * plan.num_clips)()
    check(load().gs2d_encode_batch(ctypes.byref(plan), _p(ws), _p(targets), _p(params), _p(m),
                                   _p(v), iters, out, _p(stream)), "gs2d_encode_batch")
    return [out[k] for k in range(plan.num_clips)]


def autotune_ws_bytes(sizes, tiles, max_entries: int = 0, config: Config | None = None) -> int:
    clips = (Clip * len(sizes))()
    for k, (w, h, n) in enumerate(sizes):
        clips[k].width, clips[k].height, clips[k].n = int(w), int(h), int(n)
    t = (ctypes.c_int32 * len(tiles))(*tiles)
    cfg = ctypes.byref(config) if config is not None else None
    return int(load().gs2d_autotune_ws_bytes(clips, len(sizes), max_entries, cfg, t, len(tiles)))


def autotune(sizes, params: int, targets: int, ws: int, ws_bytes: int, tiles, stages, launches,
             reps: int, stream: int, max_entries: int = 0, config: Config | None = None):
    """Returns ({(tile, stage, launch): ms}, best_tile, best_stage, best_launch)."""
    clips = (Clip * len(sizes))()
    for k, (w, h, n) in enumerate(sizes):
        clips[k].width, clips[k].height, clips[k].n = int(w), int(h), int(n)
    t = (ctypes.c_int32 * len(tiles))(*tiles)
    st = (ctypes.c_int32 * len(stages))(*stages)
    la = (ctypes.c_int32 * len(launches))(*launches)
    ms = (ctypes.c_float * (len(tiles) * len(stages) * len(launches)))()
    bt, bs, bl = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    cfg = ctypes.byref(config) if config is not None else None
    check(load().gs2d_autotune(clips, len(sizes), max_entries, cfg, _p(params), _p(targets),
                               _p(ws), ws_bytes, t, len(tiles), st, len(stages), la,
                               len(launches), reps, ms, ctypes.byref(bt), ctypes.byref(bs),
                               ctypes.byref(bl), _p(stream)), "gs2d_autotune")
    table = {}
    k = 0
    for a in tiles:
        for b in stages:
            for c in launches:
                table[(a, b, c)] = ms[k]
                k += 1
    return table, bt.value, bs.value, bl.value


def _p(x):
    return None if x is None or x == 0 else ctypes.c_void_p(x)


def project(plan: Plan, ws: int, params: int, stream: int):
    check(load().gs2d_project(ctypes.byref(plan), _p(ws), _p(params), _p(stream)), "gs2d_project")


def bin_sort(plan: Plan, ws: int, stream: int):
    check(load().gs2d_bin_sort(ctypes.byref(plan), _p(ws), _p(stream)), "gs2d_bin_sort")


def prepare(plan: Plan, ws: int, params: int, stream: int):
    check(load().gs2d_prepare(ctypes.byref(plan), _p(ws), _p(params), _p(stream)), "gs2d_prepare")


def render_fwd(plan: Plan, ws: int, img: int, stream: int):
    check(load().gs2d_render_fwd(ctypes.byref(plan), _p(ws), _p(img), _p(stream)),
          "gs2d_render_fwd")


def render_bwd(plan: Plan, ws: int, params: int, dimg: int, grads: int, stream: int):
    check(load().gs2d_render_bwd(ctypes.byref(plan), _p(ws), _p(params), _p(dimg), _p(grads),
                                 _p(stream)), "gs2d_render_bwd")


def render_l2(plan: Plan, ws: int, params: int, target: int, grads: int, img: int, loss: int,
              stream: int):
    check(load().gs2d_render_l2(ctypes.byref(plan), _p(ws), _p(params), _p(target), _p(grads),
                                _p(img), _p(loss), _p(stream)), "gs2d_render_l2")


def adam_step(params: int, grads: int, m: int, v: int, count: int, step: int, mask: int,
              config: Config | None, stream: int):
    cfg = ctypes.byref(config) if config is not None else None
    check(load().gs2d_adam_step(_p(params), _p(grads), _p(m), _p(v), count, step, _p(mask), cfg,
                                _p(stream)), "gs2d_adam_step")


def fit_step(plan: Plan, ws: int, target: int, params: int, m: int, v: int, stream: int):
    check(load().gs2d_fit_step(ctypes.byref(plan), _p(ws), _p(target), _p(params), _p(m), _p(v),
                               _p(stream)), "gs2d_fit_step")


def fit_reset(plan: Plan, ws: int, m: int, v: int, stream: int):
    check(load().gs2d_fit_reset(ctypes.byref(plan), _p(ws), _p(m), _p(v), _p(stream)),
          "gs2d_fit_reset")


def select_changed(plan: Plan, ws: int, reference: int, frame: int, threshold: float,
                   selected: int, stream: int) -> int:
    cnt = ctypes.c_int32(0)
    check(load().gs2d_select_changed(ctypes.byref(plan), _p(ws), _p(reference), _p(frame),
                                     threshold, _p(selected), ctypes.byref(cnt), _p(stream)),
          "gs2d_select_changed")
    return cnt.value


def pframe_step(plan: Plan, ws: int, target: int, params: int, m: int, v: int, selected: int,
                stream: int):
    check(load().gs2d_pframe_step(ctypes.byref(plan), _p(ws), _p(target), _p(params), _p(m),
                                  _p(v), _p(selected), _p(stream)), "gs2d_pframe_step")


def encode_pframe(plan: Plan, ws: int, target: int, params: int, m: int, v: int, selected: int,
                  iters: int, stream: int) -> float:
    psnr = ctypes.c_float(0.0)
    check(load().gs2d_encode_pframe(ctypes.byref(plan), _p(ws), _p(target), _p(params), _p(m),
                                    _p(v), _p(selected), iters, ctypes.byref(psnr), _p(stream)),
          "gs2d_encode_pframe")
    return psnr.value


def encode_frame(plan: Plan, ws: int, target: int, params: int, m: int, v: int, iters: int,
                 target_psnr: float, check_every: int, stream: int):
    """Returns (status, iters_done, final_psnr, psnr_trace list)."""
    nchk = iters // max(check_every, 1) + 2
    trace = (ctypes.c_float * nchk)()
    done = ctypes.c_int32(0)
    final = ctypes.c_float(0.0)
    st = load().gs2d_encode_frame(ctypes.byref(plan), _p(ws), _p(target), _p(params), _p(m), _p(v),
                                  iters, target_psnr, check_every, trace, ctypes.byref(done),
                                  ctypes.byref(final), _p(stream))
    checks = -(-done.value // max(check_every, 1)) if done.value else 0
    return st, done.value, final.value, [trace[i] for i in range(min(checks, nchk))]


def read_bins(plan: Plan, ws: int, stream: int, max_keys: int = -1, want_keys=True,
              want_ranges=True, want_counts=True):
    import numpy as np
    n_entries = ctypes.c_int64(0)
    lib = load()
    check(lib.gs2d_read_bins(ctypes.byref(plan), _p(ws), ctypes.byref(n_entries), None, None, 0,
                             None, None, _p(stream)), "gs2d_read_bins")
    e = n_entries.value if max_keys < 0 else min(n_entries.value, max_keys)
    keys = np.zeros(max(e, 1), np.uint32) if want_keys else None
    vals = np.zeros(max(e, 1), np.uint32) if want_keys else None
    ranges = np.zeros((plan.num_tiles, 2), np.int32) if want_ranges else None
    counts = np.zeros(max(plan.n, 1), np.int32) if want_counts else None

    def ptr(a):
        return None if a is None else a.ctypes.data_as(ctypes.c_void_p)

    check(lib.gs2d_read_bins(ctypes.byref(plan), _p(ws), ctypes.byref(n_entries), ptr(keys),
                             ptr(vals), e, ptr(ranges), ptr(counts), _p(stream)),
          "gs2d_read_bins")
    return {"n_entries": n_entries.value,
            "keys": None if keys is None else keys[:e],
            "values": None if vals is None else vals[:e],
            "ranges": ranges,
            "counts": None if counts is None else counts[:plan.n]}


def count_pairs(plan: Plan, ws: int, stream: int):
    """(pairs, hits) of the current sorted list."""
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    check(load().gs2d_count_pairs(ctypes.byref(plan), _p(ws), ctypes.byref(a), ctypes.byref(b),
                                  _p(stream)), "gs2d_count_pairs")
    return a.value, b.value


def ws_status(plan: Plan, ws: int, reset: bool, stream: int) -> int:
    return int(load().gs2d_ws_status(ctypes.byref(plan), _p(ws), int(reset), _p(stream)))


def gemm_bf16(A: int, lda: int, B: int, ldb: int, M: int, N: int, K: int, bias: int, relu: bool,
              out_f32: int, out_bf16: int, ldc: int, splits: int, partial: int, status: int,
              stream: int):
    check(load().gs2d_gemm_bf16(_p(A), lda, _p(B), ldb, M, N, K, _p(bias), int(relu), _p(out_f32),
                                _p(out_bf16), ldc, splits, _p(partial), _p(status), _p(stream)),
          "gs2d_gemm_bf16")


def call(name: str, *args):
    """Calls a gs2d_* entry point whose arguments are plain ints / floats /
    device pointers (0 = NULL) and raises on an error status."""
    fn = getattr(load(), name)
    conv = []
    for a, t in zip(args, fn.argtypes):
        conv.append(_p(a) if t is ctypes.c_void_p else a)
    check(fn(*conv), name)


def make_quant(bits, lo=None, hi=None, refine: bool = False) -> Quant:
    """Quantiser spec: bits per row (-16 half, 0 none, 1..16 uniform over
    [lo, hi]); scale and step computed in double, rounded to float.  With
    refine the library derives each uniform row's range on the device."""
    q = Quant()
    q.refine = int(bool(refine))
    for r in range(9):
        b = int(bits[r])
        q.bits[r] = b
        if b > 0 and not refine:
            lo_r, hi_r = float(lo[r]), float(hi[r])
            q.lo[r], q.hi[r] = lo_r, hi_r
            levels = (1 << b) - 1
            q.scale[r] = levels / (hi_r - lo_r)
            q.step[r] = (hi_r - lo_r) / levels
    return q


def quantize(params: int, n: int, q: Quant, codes: int, dequant: int, ranges: int, stream: int):
    check(load().gs2d_quantize(_p(params), n, ctypes.byref(q), _p(codes), _p(dequant),
                               _p(ranges), _p(stream)), "gs2d_quantize")


def fit_step_qat(plan: Plan, ws: int, target: int, params: int, m: int, v: int, q: Quant,
                 stream: int):
    check(load().gs2d_fit_step_qat(ctypes.byref(plan), _p(ws), _p(target), _p(params), _p(m),
                                   _p(v), ctypes.byref(q), _p(stream)), "gs2d_fit_step_qat")


def code_entropy(codes: int, n: int, bits, select: int, scratch: int, scratch_bytes: int,
                 out: int, stream: int):
    b = (ctypes.c_int32 * 9)(*[int(x) for x in bits])
    check(load().gs2d_code_entropy(_p(codes), n, b, _p(select), _p(scratch), scratch_bytes,
                                   _p(out), _p(stream)), "gs2d_code_entropy")


def sequence_bits(counts, payload_bits, gop: int) -> dict:
    F = len(counts)
    c = (ctypes.c_int32 * max(F, 1))(*[int(x) for x in counts])
    pb = (ctypes.c_double * max(F, 1))(*[float(x) for x in payload_bits])
    out = SeqBits()
    check(load().gs2d_sequence_bits(c, pb, F, gop, ctypes.byref(out)), "gs2d_sequence_bits")
    return {k: getattr(out, k) for k, _ in SeqBits._fields_}


def frame_from_rgb8(rgb: int, width: int, height: int, row_bytes: int, frame: int, stream: int):
    check(load().gs2d_frame_from_rgb8(_p(rgb), width, height, row_bytes, _p(frame), _p(stream)),
          "gs2d_frame_from_rgb8")


def fit_step_rgb8(plan: Plan, ws: int, rgb_host: int, rgb_dev: int, frame_dev: int,
                  params_host: int, params: int, m: int, v: int, params_out_host: int,
                  stream: int):
    check(load().gs2d_fit_step_rgb8(ctypes.byref(plan), _p(ws), _p(rgb_host), _p(rgb_dev),
                                    _p(frame_dev), _p(params_host), _p(params), _p(m), _p(v),
                                    _p(params_out_host), _p(stream)), "gs2d_fit_step_rgb8")


def fit_rebins(plan: Plan, ws: int, stream: int) -> int:
    out = ctypes.c_int64(0)
    check(load().gs2d_fit_rebins(ctypes.byref(plan), _p(ws), ctypes.byref(out), _p(stream)),
          "gs2d_fit_rebins")
    return int(out.value)


PROBE_FFMA = 0
PROBE_EX2 = 1
CHECK_CONV_FRAME = 0
CHECK_CONV_TAP = 1
CHECK_CONV_ROWS = 2


def probe_ops(blocks: int, iters: int) -> int:
    return int(load().gs2d_probe_ops(blocks, iters))


def probe_peak(kind: int, blocks: int, iters: int, sink: int, stream: int):
    check(load().gs2d_probe_peak(kind, blocks, iters, _p(sink), _p(stream)), "gs2d_probe_peak")


def fit_state_get(plan: Plan, ws: int, stream: int) -> FitState:
    st = FitState()
    check(load().gs2d_fit_state_get(ctypes.byref(plan), _p(ws), ctypes.byref(st), _p(stream)),
          "gs2d_fit_state_get")
    return st


def fit_state_set(plan: Plan, ws: int, st: FitState, stream: int):
    check(load().gs2d_fit_state_set(ctypes.byref(plan), _p(ws), ctypes.byref(st), _p(stream)),
          "gs2d_fit_state_set")


def quant_calibrate(params: int, n: int, bits, coverage: float, scratch: int,
                    scratch_bytes: int, stream: int):
    """gs2d_quant_calibrate: (lo, hi) lists of 9 floats."""
    b = (ctypes.c_int32 * 9)(*[int(x) for x in bits])
    lo, hi = (ctypes.c_float * 9)(), (ctypes.c_float * 9)()
    check(load().gs2d_quant_calibrate(_p(params), n, b, float(coverage), _p(scratch),
                                      scratch_bytes, lo, hi, _p(stream)), "gs2d_quant_calibrate")
    return list(lo), list(hi)
