"""The learned initialiser's network on the tensor cores, layer by layer
against the oracle (each layer fed the GPU's own input to it, so that BF16
roundings upstream do not mask a wiring error), and a short training run."""

import numpy as np
import pytest

from oracle import cnn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module")
def tiny():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    from paper_2505_09324_gb300.learned import LearnedInitializer, NetConfig
    from gs2d_inputs import conferencing_frame
    W, H, n, B = 96, 64, 20, 2
    net = LearnedInitializer(W, H, n, B, NetConfig(channels=(8, 16, 16, 24, 16, 32), slots=4),
                             seed=3)
    fr = [conferencing_frame(W, H, seed=s) for s in (5, 6)]
    frames = torch.from_numpy(np.stack([f for f, _ in fr])).cuda()
    masks = torch.from_numpy(np.stack([m for _, m in fr]).astype(np.uint8)).cuda()
    return net, frames, masks


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_forward_layers_match_oracle(tiny):
    net, frames, masks = tiny
    params = net.forward(frames, masks)
    torch.cuda.synchronize()
    net.check_status()
    B = net.B
    for li in range(net.L):
        ci, co, ks, ldk = net.layers[li]
        hi, wi = net.sizes[li]
        a = f64(net.x[li]).reshape(B, hi, wi, ci)
        w = f64(net.wb[li])
        ref = np.maximum(cnn.conv(a, w[:, :9 * ci + 1], 3, 2, 1), 0.0)
        got = f64(net.x[li + 1]).reshape(ref.shape)
        scale = cnn.gemm_abs(cnn.im2col(a, 3, 2, 1, ldk), w).reshape(ref.shape)
        assert np.all(np.abs(got - ref) <= REL * scale + np.abs(ref) * 2.0 ** -8 + 1e-30), li
    ci, co, ks, ldk = net.layers[-1]
    a = f64(net.x[net.L]).reshape(B, net.gh, net.gw, ci)
    w = f64(net.wb[-1])
    ref = cnn.conv(a, w[:, :ci + 1], 1, 1, 0).reshape(-1, co)
    scale = cnn.gemm_abs(cnn.im2col(a, 1, 1, 0, ldk), w)
    assert np.all(np.abs(f64(net.out) - ref) <= REL * scale + 1e-30)
    # the decoded Gaussians are those of the head output
    out = net.out.cpu().numpy()
    ref_p, ref_sel = cnn.head_decode(out, net.gh, net.gw, net.cfg.slots, net.cell,
                                     net.cfg.scale, net.n)
    np.testing.assert_array_equal(net.sel.cpu().numpy(), ref_sel)
    got_p = params.cpu().numpy().reshape(9, B, net.n).transpose(1, 0, 2)
    assert np.all(np.abs(got_p - ref_p) <= 1e-6 * np.abs(ref_p) + 1e-5)


def test_backward_layers_match_oracle(tiny):
    net, frames, masks = tiny
    net.forward(frames, masks)
    g = np.random.Generator(np.random.PCG64(2))
    dparams = torch.from_numpy(g.normal(size=(9, net.B * net.n)).astype(np.float32)).cuda()
    net.backward(dparams)
    torch.cuda.synchronize()
    net.check_status()
    B = net.B
    for li in range(net.L, -1, -1):
        ci, co, ks, ldk = net.layers[li]
        col = f64(net.col[li])
        dz = f64(net.dz[li])
        ref = dz.T @ col
        bound = REL * (np.abs(dz).T @ np.abs(col)) + 1e-30
        assert np.all(np.abs(f64(net.dw[li]) - ref) <= bound), li
        if li == 0:
            break
        hi, wi = net.sizes[li] if li < net.L else net.sizes[-1]
        stride, pad = (2, 1) if ks == 3 else (1, 0)
        w = f64(net.wb[li])
        a = f64(net.x[li]).reshape(B, hi, wi, ci)
        want = cnn.col2im(dz @ w, a.shape, ks, stride, pad) * (a > 0)
        got = f64(net.dz[li - 1]).reshape(a.shape)
        scale = cnn.col2im(np.abs(dz) @ np.abs(w), a.shape, ks, stride, pad) * (a > 0)
        # FP32 GEMM + FP32 tap sums, then one BF16 rounding
        assert np.all(np.abs(got - want) <= 1e-4 * scale + np.abs(want) * 2.0 ** -7 + 1e-30), li


def test_training_lowers_the_render_loss():
    from paper_2505_09324_gb300.learned import (LearnedInitializer, NetConfig, make_dataset,
                                                train)
    W, H, n, B = 128, 96, 120, 4
    data = make_dataset(W, H, n, list(range(300, 316)), cap=300)
    net = LearnedInitializer(W, H, n, B, NetConfig(channels=(8, 16, 32, 32, 32, 64), slots=10,
                                                   lr=3e-3), seed=1)
    hist = train(net, data, epochs=12, seed=0)
    net.check_status()
    first, last = hist[0]["render_mse_per_frame"], hist[-1]["render_mse_per_frame"]
    assert np.isfinite(last) and last < 0.5 * first, (first, last)


def test_trained_network_beats_roi_initialisation():
    """What the learned initialiser gains over the method without it: trained
    on encoder-fitted frames, it starts held-out frames at a higher PSNR and
    reaches the target in fewer fit iterations than the ROI initialiser, at
    equal Gaussian count."""
    from paper_2505_09324_gb300.learned import (LearnedInitializer, NetConfig, evaluate,
                                                make_dataset, train)
    W, H, n, B = 320, 192, 480, 4   # 10 x 6 cells x 10 slots
    data = make_dataset(W, H, n, list(range(500, 548)), cap=600)
    net = LearnedInitializer(W, H, n, B, NetConfig(channels=(8, 32, 64, 64, 128, 128),
                                                   slots=10, lr=2e-3), seed=2)
    train(net, data, epochs=25, seed=1)
    net.check_status()
    res = evaluate(net, list(range(900, 908)), target_psnr=30.0, cap=600)
    ln, roi = res["learned"], res["roi"]
    assert ln["psnr0_mean"] > roi["psnr0_mean"] + 3.0, (ln, roi)
    assert ln["iters_mean"] < roi["iters_mean"], (ln, roi)


def test_packaged_initialiser_on_a_held_out_frame():
    """The shipped 1080p initialiser (trained on seeds 10000 ... 14999) on a
    frame of another seed: its Gaussians render the frame far better than the
    ROI initialiser's (whose initial PSNR is about 16 dB)."""
    from gs2d_inputs import conferencing_frame
    from paper_2505_09324_gb300 import GaussianRasterizer
    from paper_2505_09324_gb300.learned import packaged
    W, H, n = 1920, 1080, 20000
    net = packaged(W, H, n)
    assert net is not None
    f, m = conferencing_frame(W, H, seed=31337)
    frame = torch.from_numpy(f).cuda()
    p = net.forward(frame.unsqueeze(0), torch.from_numpy(m.astype(np.uint8)).cuda().unsqueeze(0))
    r = GaussianRasterizer(W, H, n)
    r.prepare(p)
    _, loss, _ = r.render_l2(p, frame)
    psnr = 10 * np.log10(1.0 / float(loss[1]))
    assert psnr > 30.0, psnr


def test_captured_forward_replays_bit_for_bit():
    """The whole network recorded as one CUDA graph: replays on new contents
    of the captured input tensors equal direct forward calls, bit for bit."""
    from gs2d_inputs import conferencing_frame
    from paper_2505_09324_gb300.learned import packaged
    W, H, n = 1920, 1080, 20000
    net = packaged(W, H, n)
    frame = torch.empty((1, 3, H, W), device="cuda")
    mask = torch.empty((1, H, W), dtype=torch.uint8, device="cuda")
    f0, m0 = conferencing_frame(W, H, seed=4242)
    frame.copy_(torch.from_numpy(f0))
    mask.copy_(torch.from_numpy(m0.astype(np.uint8)))
    net.capture(frame, mask)
    for seed in (4243, 4244):
        f, m = conferencing_frame(W, H, seed=seed)
        frame.copy_(torch.from_numpy(f))
        mask.copy_(torch.from_numpy(m.astype(np.uint8)))
        got = net.replay().clone()
        want = net.forward(frame, mask).clone()
        torch.cuda.synchronize()
        net.check_status()
        assert torch.equal(got, want)


def test_implicit_forward_equals_im2col_forward():
    """Inference without im2col operands (every convolution an implicit GEMM)
    gives the same Gaussians bit for bit, on the shipped 1080p network and on a
    small random network with a batch of three."""
    from gs2d_inputs import conferencing_frame
    from paper_2505_09324_gb300.learned import LearnedInitializer, packaged
    for net, W, H, B in ((packaged(1920, 1080, 20000), 1920, 1080, 1),
                         (LearnedInitializer(200, 136, 200, 3, seed=5), 200, 136, 3)):
        fr = [conferencing_frame(W, H, seed=300 + b) for b in range(B)]
        frames = torch.from_numpy(np.stack([f for f, _ in fr])).cuda()
        masks = torch.from_numpy(np.stack([m for _, m in fr]).astype(np.uint8)).cuda()
        a = net.forward(frames, masks, keep_col=True).clone()
        b = net.forward(frames, masks, keep_col=False).clone()
        torch.cuda.synchronize()
        net.check_status()
        assert torch.equal(a, b)


@pytest.mark.parametrize("case", ["moved_rotated", "off_centre", "small_round"])
def test_packaged_initialiser_out_of_distribution(case):
    """The shipped 1080p initialiser was trained on the centred, upright
    subject only.  On subjects moved by 240-400 px, rotated by up to 60
    degrees, or smaller and round, it still starts far above the ROI
    initialiser (measured: 38-40 dB against 15-17 dB; about 44 dB on
    centred held-out frames) and reaches 40 dB with the fast schedule in
    fewer iterations."""
    import math

    from gs2d_inputs import SubjectMotion, background_positions, conferencing_frame
    from paper_2505_09324_gb300 import GaussianRasterizer, RasterConfig, roi_init
    from paper_2505_09324_gb300.learned import packaged
    from paper_2505_09324_gb300.raster import FAST_FIT
    W, H, n = 1920, 1080, 20000
    kw = {"moved_rotated": dict(seed=20001, t=60, motion=SubjectMotion(4.0, math.pi / 4, 1.0)),
          "off_centre": dict(seed=20002, t=100, motion=SubjectMotion(4.0, 0.0, 0.0)),
          "small_round": dict(seed=20004, t=50, motion=SubjectMotion(3.0, 2.5, 0.5),
                              area_frac=0.15, aspect=1.0)}[case]
    f, m = conferencing_frame(W, H, **kw)
    frame = torch.from_numpy(f).cuda()
    mask = torch.from_numpy(m.astype(np.uint8)).cuda()
    net = packaged(W, H, n)
    p_l = net.forward(frame.unsqueeze(0), mask.unsqueeze(0)).clone()
    bg = torch.from_numpy(background_positions(m, n, seed=kw["seed"] + 7)).cuda()
    p_r, _ = roi_init(frame, mask, n, 0.7, bg)
    r = GaussianRasterizer(W, H, n, config=RasterConfig(tile=32, stage=128, **FAST_FIT))
    ps_l, ps_r = r.psnr(frame, p_l), r.psnr(frame, p_r)
    assert ps_l > 35.0 and ps_l > ps_r + 15.0, (ps_l, ps_r)
    it_l = r.encode_frame(frame, p_l, 300, target_psnr=40.0, check_every=5)["iters"]
    it_r = r.encode_frame(frame, p_r, 300, target_psnr=40.0, check_every=5)["iters"]
    assert it_l < it_r, (it_l, it_r)
