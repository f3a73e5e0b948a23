"""The atomic backward reduction (GS2D_REDUCE_ATOMIC): float atomics add each
(tile, Gaussian) pair's eight sums into the Gaussian's sums instead of writing
one record per pair.  The sums are the same up to the order of the additions,
so the gradients are held to the oracle bars of the deterministic reduction,
and fits to the deterministic fit's loss; the per-Gaussian sums must be
cleared after every reduction (a P-frame's unselected Gaussians included)."""

import numpy as np
import pytest

from gs2d_inputs import random_gaussians, smooth_noise_target

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_REL = 1e-3


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def check_grads(g_gpu, ref, unc, rel=GRAD_REL):
    g = g_gpu.detach().cpu().numpy().astype(np.float64)
    rms = np.sqrt(np.mean(ref * ref, axis=1, keepdims=True))
    bound = rel * np.abs(ref) + rel * rms + unc
    bad = np.abs(g - ref) > bound
    assert not bad.any(), f"{bad.sum()} gradient entries off"


def atomic(gs, **kw):
    from paper_2505_09324_gb300 import _native as nat
    return gs.RasterConfig(reduce=nat.REDUCE_ATOMIC, **kw)


@pytest.mark.parametrize("tile,stage", [(8, 32), (16, 64), (32, 128), (32, 256)])
def test_atomic_gradients_match_oracle(gs, oracle, tile, stage):
    W, H, n = 100, 70, 300
    p = random_gaussians(n, W, H, seed=11)
    target = smooth_noise_target(W, H, seed=13)
    r = gs.GaussianRasterizer(W, H, n, config=atomic(gs, tile=tile, stage=stage))
    r.prepare(to_dev(p))
    res = oracle.loss_and_grad(p, target)
    for _ in range(2):  # the second call sees the sums the first one cleared
        grads, loss, _ = r.render_l2(to_dev(p), to_dev(target))
        check_grads(grads, res["grad"], res["grad_unc"])
    dimg = (smooth_noise_target(W, H, seed=12).astype(np.float64) - 0.5) * 1e-3
    gref, unc = oracle.render_grad(p, W, H, dimg, uncertainty=True)
    check_grads(r.render_bwd(to_dev(p), to_dev(dimg)), gref, unc)
    assert r.status() == 0


def test_atomic_fit_reaches_the_deterministic_fits_loss(gs):
    W, H, n, iters = 160, 120, 600, 60
    p0 = random_gaussians(n, W, H, seed=31, l_range=(1.5, 8.0))
    t = to_dev(smooth_noise_target(W, H, seed=32))
    out = {}
    for name, cfg in (("slots", gs.RasterConfig.fast_fit()),
                      ("atomic", gs.RasterConfig.fast_fit(reduce=1))):
        r = gs.GaussianRasterizer(W, H, n, config=cfg)
        p = to_dev(p0)
        o = r.encode_frame(t, p, iters, check_every=iters)
        assert o["status"] == 0
        out[name] = o["psnr"]
    assert abs(out["atomic"] - out["slots"]) < 0.05, out


def test_atomic_pframe_step_leaves_no_stale_sums(gs):
    """A P-frame step renders whole tiles, so unselected Gaussians there get
    sums too; the reduction must clear them, or the next full backward would
    add them in."""
    from paper_2505_09324_gb300 import _native as nat
    W, H, n = 120, 96, 400
    p = to_dev(random_gaussians(n, W, H, seed=33, l_range=(1.5, 7.0)))
    t = to_dev(smooth_noise_target(W, H, seed=34))
    sel = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sel[::3] = 1
    grads = {}
    for name, red in (("slots", 0), ("atomic", 1)):
        r = gs.GaussianRasterizer(W, H, n, config=gs.RasterConfig(reduce=red))
        q = p.clone()
        m, v = torch.empty_like(q), torch.empty_like(q)
        s = int(torch.cuda.current_stream().cuda_stream)
        nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
        nat.pframe_step(r.plan, r.ws_ptr, t.data_ptr(), q.data_ptr(), m.data_ptr(),
                        v.data_ptr(), sel.data_ptr(), s)
        assert torch.equal(q[:, sel == 0], p[:, sel == 0])
        r.prepare(q)
        g, _, _ = r.render_l2(q, t)
        grads[name] = (q, g)
    qa, ga = grads["atomic"]
    qs, gs_ = grads["slots"]
    # the selected Gaussians moved by (nearly) the same Adam step
    assert float((qa - qs).abs().max()) < 2e-2
    scale = gs_.abs().amax(dim=1, keepdim=True).clamp_min(1e-12)
    assert float(((ga - gs_).abs() / scale).max()) < 1e-2


def test_stage_256_renders_like_stage_64(gs, oracle):
    """Lists longer than 256 Gaussians in one tile: several 256-wide batches.
    The batch size changes neither a pixel's accumulation order nor any
    pair's sums, so stage 256 equals stage 64 bit for bit; both against the
    oracle (colours scaled down so that FP32 sums of hundreds of terms stay
    within the absolute image tolerance)."""
    W, H, n = 64, 48, 900
    p = random_gaussians(n, W, H, seed=35, l_range=(2.0, 14.0))
    p[5:8] *= 0.05
    target = smooth_noise_target(W, H, seed=36)
    res = oracle.loss_and_grad(p, target)
    out = {}
    for stage in (64, 256):
        for launch in (0, 1):
            r = gs.GaussianRasterizer(W, H, n, config=gs.RasterConfig(tile=16, stage=stage,
                                                                      launch=launch))
            r.prepare(to_dev(p))
            grads, loss, img = r.render_l2(to_dev(p), to_dev(target), want_image=True)
            assert r.status() == 0
            out[(stage, launch)] = (img, grads, loss)
    for key, (img, grads, loss) in out.items():
        ref = out[(64, key[1])]
        assert torch.equal(img, ref[0]) and torch.equal(grads, ref[1])
        assert torch.equal(loss, ref[2])
    img, grads, _ = out[(256, 1)]
    d = img.cpu().numpy().astype(np.float64) - res["img"]
    assert np.all(d >= res["amb_lo"] - 1e-5) and np.all(d <= res["amb_hi"] + 1e-5)
    check_grads(grads, res["grad"], res["grad_unc"])
