"""The C-ABI library builds, loads and exports every function declared in
include/gs2d.h; host-only entry points (config, plan layout, argument checks)
behave as documented.  No kernel is launched: these run without a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nat():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    return _native


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs2d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs2d_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_function_is_exported(nat):
    lib = ctypes.CDLL(nat.library_path())
    decl = declared_functions()
    assert len(decl) >= 14
    for name in decl:
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert set(decl) == set(nat.EXPORTS)


def test_every_declared_constant_is_bound(nat):
    """Each enum constant of include/gs2d.h has the same value in the Python
    binding (under its full name or without the GS2D_ prefix)."""
    src = open(os.path.join(ROOT, "include", "gs2d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = re.findall(r"\b(GS2D_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)
    assert len(consts) >= 15
    for name, value in consts:
        bound = getattr(nat, name, getattr(nat, name[len("GS2D_"):], None))
        assert bound == int(value), f"{name} = {value} bound as {bound}"


def test_struct_layouts_match(nat):
    lib = nat.load()
    assert lib.gs2d_sizeof_plan() == ctypes.sizeof(nat.Plan)
    assert lib.gs2d_sizeof_config() == ctypes.sizeof(nat.Config)
    assert ctypes.sizeof(nat.Clip) == 40


def test_default_config(nat):
    c = nat.default_config()
    assert c.tile == 16 and c.stage == 64 and c.launch == nat.LAUNCH_GRID
    assert abs(c.sigma_cut - 4.5) < 1e-7
    assert abs(c.alpha_min - 1 / 255) < 1e-9 and abs(c.lr - 1e-2) < 1e-9
    # the Python wrapper's defaults are the library's
    from paper_2505_09324_gb300.raster import RasterConfig
    rc = RasterConfig().to_c()
    for name, _ in nat.Config._fields_:
        assert getattr(rc, name) == getattr(c, name), name
    assert c.bin_margin == 4.0


def test_plan_layout(nat):
    p = nat.plan_init(1920, 1080, 20000)
    assert (p.tiles_x, p.tiles_y, p.num_tiles) == (120, 68, 8160)
    assert p.tile_bits == 13 and p.num_clips == 1 and p.stage == 64
    assert p.max_entries == max(1 << 20, 16 * 20000) and p.pixels == 1920 * 1080
    offs = list(p.off)[:22]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs) and p.ws_bytes > offs[-1]
    q = nat.plan_init(16, 16, 5)
    assert q.num_tiles == 1 and q.tile_bits == 0


@pytest.mark.parametrize("args", [(0, 10, 5, 0), (10, -1, 5, 0), (10, 10, -1, 0),
                                  (10, 10, 5, -3), (10, 10, 5, 1 << 31), (10, 10, 5, 1 << 28),
                                  (10, 10, (1 << 27) + 1, 0)])
def test_plan_rejects_bad_sizes(nat, args):
    with pytest.raises(nat.Gs2dError) as e:
        nat.plan_init(*args)
    assert e.value.status == nat.GS2D_ERR_INVALID_ARG


def test_plan_size_limits_keep_kernel_indices_in_32_bits(nat):
    # 8 floats per entry and 9 parameter rows must stay below 2^31
    p = nat.plan_init(64, 64, 10, (1 << 28) - 1)
    assert 8 * p.max_entries + 7 < 1 << 31
    big = nat.plan_init(64, 64, 1 << 27)           # the default capacity is clamped
    assert big.max_entries == (1 << 28) - 1 and 9 * big.n < 1 << 31
    c = nat.default_config()
    c.tile = 8
    assert nat.plan_init(64, 64, 1 << 27, 0, c).max_entries == (1 << 28) - 1


@pytest.mark.parametrize("tile,stage,tiles", [(8, 32, (8, 6)), (16, 128, (4, 3)), (32, 0, (2, 2))])
def test_plan_tile_and_stage(nat, tile, stage, tiles):
    c = nat.default_config()
    c.tile, c.stage = tile, stage
    p = nat.plan_init(64, 48, 10, 0, c)
    assert (p.tiles_x, p.tiles_y) == tiles and p.tile == tile
    assert p.stage == (stage or 64)
    assert p.max_entries == max(1 << 20, (64 if tile == 8 else 16) * 10)


def test_batch_plan_offsets(nat):
    """Clip table: Gaussians side by side, tiles and images one after another."""
    sizes = [(640, 360, 2000), (17, 9, 0), (1280, 720, 5000), (1, 1, 3)]
    p, clips = nat.plan_init_batch(sizes)
    assert p.num_clips == 4 and p.n == 7003 and p.width == 0 and p.height == 0
    q, qc = nat.plan_init_batch([(100, 70, 5)])  # one clip: a single-frame plan
    assert (q.width, q.height, q.tiles_x, q.tiles_y) == (100, 70, 7, 5)
    g, t, px = 0, 0, 0
    for c, (w, h, n) in zip(clips, sizes):
        assert (c.width, c.height, c.n) == (w, h, n)
        assert (c.tiles_x, c.tiles_y) == (-(-w // 16), -(-h // 16))
        assert (c.g_off, c.tile_off, c.pix_off) == (g, t, 3 * px)
        g, t, px = g + n, t + c.tiles_x * c.tiles_y, px + w * h
    assert p.num_tiles == t and p.pixels == px
    offs = list(p.off)[:22]
    assert all(o % 256 == 0 for o in offs) and offs == sorted(offs)


def test_batch_plan_rejects_bad_clips(nat):
    for sizes in ([], [(0, 5, 1)], [(5, 5, -1)]):
        with pytest.raises((nat.Gs2dError, ValueError)):
            if not sizes:
                p = nat.Plan()
                nat.check(nat.load().gs2d_plan_init_batch(ctypes.byref(p), None, 0, 0, None))
            else:
                nat.plan_init_batch(sizes)
    p, clips = nat.plan_init_batch([(32, 32, 4), (16, 16, 2)])
    clips[1].tile_off += 1                      # not the table the plan was laid out from
    with pytest.raises(nat.Gs2dError):
        nat.ws_set_clips(p, 0x1000, clips, 0)


def test_autotune_ws_bytes_covers_every_candidate(nat):
    sizes = [(640, 360, 2000), (320, 200, 800)]
    most = nat.autotune_ws_bytes(sizes, [8, 16, 32])
    for t in (8, 16, 32):
        c = nat.default_config()
        c.tile = t
        p, _ = nat.plan_init_batch(sizes, 0, c)
        assert p.ws_bytes <= most
    assert nat.autotune_ws_bytes(sizes, [12]) == 0


def test_plan_rejects_bad_config(nat):
    for tile, stage, launch in ((12, 64, 0), (16, 48, 0), (64, 64, 0), (16, 64, 2)):
        c = nat.default_config()
        c.tile, c.stage, c.launch = tile, stage, launch
        with pytest.raises(nat.Gs2dError):
            nat.plan_init(64, 64, 10, 0, c)
    c = nat.default_config()
    c.sigma_cut = -1.0
    with pytest.raises(nat.Gs2dError):
        nat.plan_init(64, 64, 10, 0, c)
    c = nat.default_config()
    c.bin_margin = float("nan")
    with pytest.raises(nat.Gs2dError):
        nat.plan_init(64, 64, 10, 0, c)
    c.bin_margin = -1.0  # per-iteration binning
    nat.plan_init(64, 64, 10, 0, c)
    for reduce in (-1, 2):
        c = nat.default_config()
        c.reduce = reduce
        with pytest.raises(nat.Gs2dError):
            nat.plan_init(64, 64, 10, 0, c)
    c = nat.default_config()
    c.reduce, c.stage = nat.REDUCE_ATOMIC, 256
    q = nat.plan_init(64, 64, 10, 0, c)
    assert q.stage == 256 and q.cfg.reduce == nat.REDUCE_ATOMIC


def test_calls_reject_bad_arguments_without_touching_the_gpu(nat):
    p = nat.plan_init(64, 64, 10)
    with pytest.raises(nat.Gs2dError):
        nat.project(p, 0, 0x1000, 0)            # NULL workspace
    with pytest.raises(nat.Gs2dError):
        nat.project(p, 0x1001, 0x1000, 0)       # misaligned workspace
    with pytest.raises(nat.Gs2dError):
        nat.render_fwd(p, 0x1000, 0, 0)         # NULL image
    bad = nat.Plan()
    with pytest.raises(nat.Gs2dError):
        nat.bin_sort(bad, 0x1000, 0)            # plan never initialised
    with pytest.raises(nat.Gs2dError):
        nat.adam_step(0x1000, 0x1000, 0x1000, 0x1000, 9, 0, 0, None, 0)  # step 0
    assert "step" in nat.last_error()
    # a frame too large for the ROI initialiser's 32-bit pixel indices
    lib = nat.load()
    st = lib.gs2d_roi_init(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000), 65536, 32768, 10,
                           ctypes.c_float(0.7), ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000),
                           None, ctypes.c_void_p(0x1000), ctypes.c_uint64(1 << 40), None)
    assert st == nat.GS2D_ERR_INVALID_ARG and "sizes" in nat.last_error()
    with pytest.raises(nat.Gs2dError):
        nat.fit_rebins(bad, 0x1000, 0)          # plan never initialised
    with pytest.raises(nat.Gs2dError):
        nat.fit_rebins(p, 0, 0)                 # NULL workspace


def test_quantizer_arguments_checked_before_any_launch(nat):
    ok = nat.make_quant([-16] * 9)
    bad_bits = nat.Quant()
    bad_bits.bits[0] = 17
    assert nat.load().gs2d_quantize(None, 0, ctypes.byref(bad_bits), None, None, None,
                                    None) == nat.GS2D_ERR_INVALID_ARG
    # neither codes nor values asked for
    assert nat.load().gs2d_quantize(ctypes.c_void_p(256), 4, ctypes.byref(ok), None, None,
                                    None, None) == nat.GS2D_ERR_INVALID_ARG
    # a uniform row without a valid range (and no refine)
    nr = nat.Quant()
    nr.bits[0], nr.lo[0], nr.hi[0] = 8, 1.0, 1.0        # scale and step 0
    assert nat.load().gs2d_quantize(None, 0, ctypes.byref(nr), None, None, None,
                                    None) == nat.GS2D_ERR_INVALID_ARG
    p = nat.plan_init(64, 64, 10)
    assert nat.load().gs2d_fit_step_qat(ctypes.byref(p), None, None, None, None, None,
                                        ctypes.byref(ok), None) == nat.GS2D_ERR_INVALID_ARG


def test_quantizer_spec_host_side():
    import numpy as np
    from paper_2505_09324_gb300.quant import HALF, Quantizer
    bits = (HALF, HALF, 8, 8, 8, 8, 8, 8, 8)
    q = Quantizer(bits, [-1.0] * 9, [1.0] * 9)
    assert q.bits_per_gaussian == 32 + 7 * 8
    assert q.lo[2] == -1.0 and q.hi[2] == 1.0
    assert q.c.scale[2] == np.float32(255 / 2) and q.c.step[2] == np.float32(2 / 255)
    assert q.frame_bytes(20000) == 20000 * 88 // 8 + 7 * 8
    assert Quantizer(refine=True).bits_per_gaussian == 2 * 16 + 3 * 10 + 4 * 8
    with pytest.raises(ValueError):
        Quantizer([HALF] * 8)
    with pytest.raises(ValueError):
        Quantizer([8] * 9)               # uniform rows need ranges or refine


def test_sequence_bits_host_arithmetic_matches_oracle(nat):
    """gs2d_sequence_bits is host arithmetic (no device work): Eq. 3-4 totals
    against the oracle's plain sums (lgamma vs a sum of logarithms)."""
    import numpy as np
    from oracle import bitstream as B
    rng = np.random.default_rng(3)
    for F, K in ((1, 1), (7, 3), (60, 4), (61, 8), (10, 100)):
        counts = [int(x) for x in rng.integers(0, 20000, F)]
        payload = [float(x) for x in rng.uniform(0, 2e6, F)]
        got = nat.sequence_bits(counts, payload, K)
        ref = B.sequence_bits(counts, payload, K)
        for k in ("i_bits", "p_bits", "savings", "total_bits"):
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-9), (F, K, k)
        assert (got["i_frames"], got["p_frames"]) == (ref["i_frames"], ref["p_frames"])
    assert nat.sequence_bits([], [], 4)["total_bits"] == 0.0
    for bad in (([1], [1.0], 0), ([-1, 2], [1.0, 1.0], 2), ([1, 2], [1.0, float("nan")], 2)):
        with pytest.raises(nat.Gs2dError):
            nat.sequence_bits(*bad)
