"""Frame sequences with inter-frame reuse (warm start from the previous
frame's Gaussians) on the moving-subject conferencing scene, and a fit loop
driven through torch.autograd against the library's fused fit loop."""

import numpy as np
import pytest

from gs2d_inputs import background_positions, conferencing_frame, random_motion

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def sequence(W, H, frames, seed):
    mo = random_motion(seed)
    out = [conferencing_frame(W, H, seed=seed, t=t, motion=mo) for t in range(frames)]
    return [torch.from_numpy(f).cuda() for f, _ in out], [m for _, m in out]


def test_warm_start_beats_fresh_initialisation(gs):
    W, H, n, seed = 480, 270, 2000, 2
    frames, masks = sequence(W, H, 6, seed)
    bg = torch.from_numpy(background_positions(masks[0], n, seed=seed + 10)).cuda()
    mk = torch.from_numpy(masks[0].astype(np.uint8)).cuda()
    p0, _ = gs.roi_init(frames[0], mk, n, 0.7, bg)
    r = gs.GaussianRasterizer(W, H, n)
    stream = torch.cuda.Stream()
    p = p0.clone()
    with torch.cuda.stream(stream):
        recs = gs.encode_sequence(r, frames, p, 300, 60, stream=stream)
    stream.synchronize()
    assert [x["iters"] for x in recs] == [300] + [60] * 5
    # a frame fitted from scratch (its own ROI initialisation) for as many iterations
    for k in (1, 5):
        mk = torch.from_numpy(masks[k].astype(np.uint8)).cuda()
        bgk = torch.from_numpy(background_positions(masks[k], n, seed=seed + 10)).cuda()
        q, _ = gs.roi_init(frames[k], mk, n, 0.7, bgk)
        with torch.cuda.stream(stream):
            fresh = r.encode_frame(frames[k], q, 60, target_psnr=0.0, check_every=60,
                                   stream=stream)
        stream.synchronize()
        assert recs[k]["psnr"] > fresh["psnr"] + 1.0, (k, recs[k]["psnr"], fresh["psnr"])
    assert min(x["psnr"] for x in recs) > 25.0


def test_autograd_fit_loop_tracks_fused_fit_loop(gs):
    """An optimisation loop written in PyTorch around the autograd function
    (L2 loss by torch, the library's Adam step) follows the fused, graph-
    captured loop of gs2d_encode_frame: same Gaussians to FP32 noise."""
    from paper_2505_09324_gb300.autograd import rasterize
    W, H, n = 96, 64, 300
    frames, masks = sequence(W, H, 1, 4)
    target = frames[0]
    bg = torch.from_numpy(background_positions(masks[0], n, seed=3)).cuda()
    p0, _ = gs.roi_init(target, torch.from_numpy(masks[0].astype(np.uint8)).cuda(), n, 0.7, bg)
    iters = 20
    r = gs.GaussianRasterizer(W, H, n)
    fused = p0.clone()
    r.encode_frame(target, fused, iters, target_psnr=0.0, check_every=iters)
    q = p0.clone().requires_grad_(True)
    m, v = torch.zeros_like(p0), torch.zeros_like(p0)
    r2 = gs.GaussianRasterizer(W, H, n)
    for it in range(1, iters + 1):
        q.grad = None
        loss = ((rasterize(q, r2) - target) ** 2).mean()
        loss.backward()
        with torch.no_grad():
            gs.adam_step(q.data, q.grad.contiguous(), m, v, it)
    d = (q.detach() - fused).abs()
    scale = p0.abs().amax(dim=1, keepdim=True).clamp_min(1e-3)
    assert float((d / scale).max()) < 1e-3


def test_fit_step_equals_the_encoder_loop(gs):
    """gs2d_fit_step, called k times after gs2d_fit_reset, is the encoder's
    iteration: the same Gaussians bit for bit as gs2d_encode_frame(k)."""
    from paper_2505_09324_gb300 import _native as nat
    W, H, n, k = 160, 96, 400, 12
    frames, masks = sequence(W, H, 1, 7)
    bg = torch.from_numpy(background_positions(masks[0], n, seed=8)).cuda()
    p0, _ = gs.roi_init(frames[0], torch.from_numpy(masks[0].astype(np.uint8)).cuda(), n, 0.7, bg)
    r = gs.GaussianRasterizer(W, H, n)
    a = p0.clone()
    r.encode_frame(frames[0], a, k, target_psnr=0.0, check_every=k)
    b = p0.clone()
    m, v = torch.empty_like(b), torch.empty_like(b)
    s = int(torch.cuda.current_stream().cuda_stream)
    nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
    for _ in range(k):
        nat.fit_step(r.plan, r.ws_ptr, frames[0].data_ptr(), b.data_ptr(), m.data_ptr(),
                     v.data_ptr(), s)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert not torch.equal(a, p0)
