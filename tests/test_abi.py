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


def test_struct_layouts_match(nat):
    lib = nat.load()
    assert lib.gs2d_sizeof_plan() == ctypes.sizeof(nat.Plan)
    assert lib.gs2d_sizeof_config() == ctypes.sizeof(nat.Config)


def test_default_config(nat):
    c = nat.default_config()
    assert c.tile == 16 and abs(c.sigma_cut - 4.5) < 1e-7
    assert abs(c.alpha_min - 1 / 255) < 1e-9 and abs(c.lr - 1e-2) < 1e-9


def test_plan_layout(nat):
    p = nat.plan_init(1920, 1080, 20000)
    assert (p.tiles_x, p.tiles_y, p.num_tiles) == (120, 68, 8160)
    assert p.tile_bits == 13 and p.sort_passes == 1
    assert p.max_entries == max(1 << 20, 16 * 20000)
    offs = list(p.off)[:13]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs) and p.ws_bytes > offs[-1]
    q = nat.plan_init(16, 16, 5)
    assert q.num_tiles == 1 and q.tile_bits == 0


@pytest.mark.parametrize("args", [(0, 10, 5, 0), (10, -1, 5, 0), (10, 10, -1, 0),
                                  (10, 10, 5, -3), (10, 10, 5, 1 << 31)])
def test_plan_rejects_bad_sizes(nat, args):
    with pytest.raises(nat.Gs2dError) as e:
        nat.plan_init(*args)
    assert e.value.status == nat.GS2D_ERR_INVALID_ARG


def test_plan_rejects_bad_config(nat):
    c = nat.default_config()
    c.tile = 8
    with pytest.raises(nat.Gs2dError):
        nat.plan_init(64, 64, 10, 0, c)
    c = nat.default_config()
    c.sigma_cut = -1.0
    with pytest.raises(nat.Gs2dError):
        nat.plan_init(64, 64, 10, 0, c)


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
