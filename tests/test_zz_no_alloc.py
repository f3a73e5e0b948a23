"""gs2d_render_fwd_noalloc: the forward render for callers that cannot allocate
device memory (it works out of a fixed scratch array the library reserves at
load time).  Its output must match the workspace-based entry points
(gs2d_project + gs2d_bin_sort + gs2d_render_fwd) on consecutive calls, so that
nothing left in the shared scratch by one call leaks into the next.  This file
is named to be collected last."""

import ctypes

import numpy as np
import pytest

from gs2d_inputs import random_gaussians

IMG_TOL = 1e-5


@pytest.fixture(scope="module")
def nat():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    return _native


def noalloc_render(nat, torch, params_np, W, H):
    p = torch.from_numpy(np.ascontiguousarray(params_np, np.float32)).cuda()
    img = torch.full((3, H, W), float("nan"), device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lib = nat.load()
    rc = lib.gs2d_render_fwd_noalloc(ctypes.c_void_p(p.data_ptr()), p.shape[1], W, H, None,
                                     ctypes.c_void_p(img.data_ptr()),
                                     ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))
    nat.check(rc, "gs2d_render_fwd_noalloc")
    torch.cuda.synchronize()
    return img.cpu().numpy(), int(status.item())


def workspace_render(torch, params_np, W, H):
    from paper_2505_09324_gb300 import GaussianRasterizer
    r = GaussianRasterizer(W, H, params_np.shape[1])
    r.prepare(torch.from_numpy(np.ascontiguousarray(params_np, np.float32)).cuda())
    return r.render_fwd().cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_workspace_render_on_consecutive_calls(nat):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    cases = [(256, 256, random_gaussians(2000, 256, 256, seed=0)),
             (100, 70, random_gaussians(300, 100, 70, seed=11))]
    for W, H, p in cases:
        got, status = noalloc_render(nat, torch, p, W, H)
        ref = workspace_render(torch, p, W, H)
        assert status == nat.GS2D_OK
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref, rtol=0, atol=IMG_TOL)
    # the same call twice in a row gives the same image
    W, H, p = cases[0]
    a, _ = noalloc_render(nat, torch, p, W, H)
    b, _ = noalloc_render(nat, torch, p, W, H)
    np.testing.assert_allclose(a, b, rtol=0, atol=IMG_TOL)


def test_noalloc_rejects_sizes_beyond_its_scratch(nat):
    lib = nat.load()
    img = ctypes.c_void_p(0x1000)  # never dereferenced: the call fails on the host first
    rc = lib.gs2d_render_fwd_noalloc(ctypes.c_void_p(0x1000), 1 << 20, 4096, 4096, None, img,
                                     None, None)
    assert rc == nat.GS2D_ERR_INVALID_ARG
    assert "static scratch" in nat.last_error()


@pytest.mark.gpu
def test_noalloc_reports_capacity_overflow_then_recovers(nat):
    """Tile entries beyond the scratch's entry capacity: the call renders zero
    and reports GS2D_ERR_CAPACITY through its status word; the next call, which
    fits, must not see that status (the header is cleared per call) and must
    match the workspace render again."""
    torch = pytest.importorskip("torch")
    W, H = 512, 512
    p = random_gaussians(1000, W, H, seed=4)
    p[2] = 150.0  # every Gaussian covers the whole frame: ~1e6 (tile, Gaussian) entries
    p[3] = 0.0
    p[4] = 150.0
    got, status = noalloc_render(nat, torch, p, W, H)
    assert status == nat.GS2D_ERR_CAPACITY
    assert float(np.abs(got).max()) == 0.0
    q = random_gaussians(300, 100, 70, seed=11)
    got, status = noalloc_render(nat, torch, q, 100, 70)
    assert status == nat.GS2D_OK
    np.testing.assert_allclose(got, workspace_render(torch, q, 100, 70), rtol=0, atol=IMG_TOL)
