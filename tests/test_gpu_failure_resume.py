"""Failure detection and resume.

* The tensor-core GEMM bounds every mbarrier wait in time.  The failure is
  made on the host: gs2d_gemm_wait_check launches the GEMM kernel with its
  operand loads withheld, so a wait on a barrier that nothing will complete
  runs out after a short limit (no copy or MMA is in flight).  The kernel
  must report GS2D_ERR_TIMEOUT through its status word, leave its output
  alone and return, and the context must stay usable.
* A fit interrupted after K1 iterations and resumed from a checkpoint
  (parameters, Adam moments and the workspace's optimiser state) in a fresh
  workspace continues bit for bit as the uninterrupted fit."""

import ctypes
import time

import numpy as np
import pytest

from gs2d_inputs import random_gaussians, smooth_noise_target

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    return _native


def test_gemm_wait_runs_out_and_reports_timeout(nat):
    lib = nat.load()
    g = torch.Generator(device="cpu").manual_seed(0)
    A = torch.randn(128, 64, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(32, 64, generator=g).to(torch.bfloat16).cuda()
    out = torch.full((128, 32), 7.0, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = lib.gs2d_gemm_wait_check(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(status.data_ptr()), 20_000_000,
                                  ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nat.check(rc, "gs2d_gemm_wait_check")
    assert int(status.item()) == nat.GS2D_ERR_TIMEOUT
    assert dt >= 0.02                       # the wait ran to its limit
    assert bool(torch.all(out == 7.0))      # the output tile was left unwritten
    # the context is still usable: the same GEMM, loads issued, is correct
    status.zero_()
    C = torch.empty(128, 32, device="cuda")
    nat.check(lib.gs2d_gemm_bf16(ctypes.c_void_p(A.data_ptr()), 64, ctypes.c_void_p(B.data_ptr()),
                                 64, 128, 32, 64, None, 0, ctypes.c_void_p(C.data_ptr()), None, 32,
                                 1, None, ctypes.c_void_p(status.data_ptr()),
                                 ctypes.c_void_p(stream)), "gs2d_gemm_bf16")
    torch.cuda.synchronize()
    assert int(status.item()) == nat.GS2D_OK
    ref = A.float() @ B.float().T
    assert float((C - ref).abs().max()) <= 2e-5 * float((A.float().abs() @ B.float().abs().T).max())



@pytest.mark.parametrize("kernel", ["frame", "tap", "rows"])
def test_conv_wait_runs_out_and_reports_timeout(nat, kernel):
    """The persistent convolutions with every load withheld: each role's
    first wait runs out, the groups that share a named barrier leave it
    together, and the kernel reports GS2D_ERR_TIMEOUT without writing its
    output; then the same convolution, loads issued, is right."""
    lib = nat.load()
    g = torch.Generator(device="cpu").manual_seed(1)
    if kernel == "frame":
        which, ldk, co = nat.CHECK_CONV_FRAME, 80, 32
        x = torch.rand(1, 3, 16, 256, generator=g).cuda()
    else:
        which, ldk, co = nat.CHECK_CONV_TAP if kernel == "tap" else nat.CHECK_CONV_ROWS, 296, 64
        x = torch.randn(1, 16, 256, 32, generator=g).to(torch.bfloat16).cuda()
    w = (torch.randn(co, ldk, generator=g) * 0.1).to(torch.bfloat16).cuda()
    out = torch.full((8 * 128, co), 7.0, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = lib.gs2d_conv_wait_check(which, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(status.data_ptr()), 20_000_000,
                                  ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nat.check(rc, "gs2d_conv_wait_check")
    assert int(status.item()) == nat.GS2D_ERR_TIMEOUT
    assert dt >= 0.02                       # the waits ran to their limit
    assert bool(torch.all(out == 7.0))      # nothing was stored
    # the context is still usable: the same convolution with its loads
    status.zero_()
    if kernel == "frame":
        nat.call("gs2d_conv_frame_bf16", x.data_ptr(), 0, 1, 16, 256, 3, 2, 1, w.data_ptr(), ldk,
                 co, 1, 0, out.data_ptr(), co, status.data_ptr(), stream)
        xin = torch.empty((1, 16, 256, 8), dtype=torch.bfloat16, device="cuda")
        nat.call("gs2d_cnn_input", x.data_ptr(), 0, 1, 16, 256, xin.data_ptr(), stream)
        cin = 8
    else:
        nat.call("gs2d_conv_bf16", x.data_ptr(), 1, 16, 256, 32, 3, 2, 1, w.data_ptr(), ldk, co,
                 1, 0, out.data_ptr(), co, status.data_ptr(), stream)
        xin, cin = x, 32
    col = torch.empty((8 * 128, ldk), dtype=torch.bfloat16, device="cuda")
    nat.call("gs2d_im2col", xin.data_ptr(), 1, 16, 256, cin, 3, 2, 1, col.data_ptr(), ldk, stream)
    ref = torch.relu(col.float() @ w.float().T)
    torch.cuda.synchronize()
    assert int(status.item()) == nat.GS2D_OK
    assert float((out.float() - ref).abs().max()) <= 1e-2 * float(ref.abs().max()) + 1e-6

def test_wait_check_rejects_bad_arguments(nat):
    lib = nat.load()
    rc = lib.gs2d_gemm_wait_check(None, None, None, None, 20_000_000, None)
    assert rc == nat.GS2D_ERR_INVALID_ARG
    p = ctypes.c_void_p(0x1000)  # never dereferenced: rejected on the host
    assert lib.gs2d_gemm_wait_check(p, p, p, p, 10, None) == nat.GS2D_ERR_INVALID_ARG


@pytest.mark.parametrize("schedule", ["plain", "fast"])
def test_fit_resumes_bit_for_bit_from_a_checkpoint(nat, schedule):
    from paper_2505_09324_gb300 import GaussianRasterizer, RasterConfig
    from paper_2505_09324_gb300.raster import FAST_FIT
    W, H, n = 160, 96, 400
    cfg = RasterConfig(tile=16, **(FAST_FIT if schedule == "fast" else {}))
    p0 = torch.from_numpy(random_gaussians(n, W, H, seed=21)).cuda()
    target = torch.from_numpy(smooth_noise_target(W, H, seed=22)).cuda()
    K1, K2 = 23, 17
    # uninterrupted
    r = GaussianRasterizer(W, H, n, config=cfg)
    p = p0.clone()
    adam = (torch.empty_like(p), torch.empty_like(p))
    r.fit_reset(adam)
    for _ in range(K1 + K2):
        r.fit_step(target, p, adam)
    # interrupted after K1, checkpointed to the host, resumed in a new workspace
    r1 = GaussianRasterizer(W, H, n, config=cfg)
    q = p0.clone()
    adam1 = (torch.empty_like(q), torch.empty_like(q))
    r1.fit_reset(adam1)
    for _ in range(K1):
        r1.fit_step(target, q, adam1)
    ckpt = r1.fit_checkpoint(q, adam1)
    assert ckpt["step"] == K1
    del r1, q, adam1
    r2 = GaussianRasterizer(W, H, n, config=cfg)
    q = torch.empty_like(p0)
    adam2 = (torch.empty_like(q), torch.empty_like(q))
    r2.fit_restore(ckpt, q, adam2)
    for _ in range(K2):
        r2.fit_step(target, q, adam2)
    torch.cuda.synchronize()
    assert r.status() == nat.GS2D_OK and r2.status() == nat.GS2D_OK
    assert torch.equal(p, q)
    assert torch.equal(adam[0], adam2[0]) and torch.equal(adam[1], adam2[1])
    s1 = nat.fit_state_get(r.plan, r.ws_ptr, 0)
    s2 = nat.fit_state_get(r2.plan, r2.ws_ptr, 0)
    assert (s1.step, s1.beta1_pow, s1.beta2_pow, s1.decay_pow) == (
        s2.step, s2.beta1_pow, s2.beta2_pow, s2.decay_pow) and s1.step == K1 + K2
