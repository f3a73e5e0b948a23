"""Tile lists kept across fit iterations (gs2d_config.bin_margin >= 0).

A Gaussian adds nothing to a tile outside its cut-off box, so lists built from
widened rectangles and rebuilt only when a Gaussian leaves them must give the
fit loop exactly the results of lists rebuilt every iteration: the render skips
uncovered (tile, Gaussian) pairs and the backward slots, hence the order of
every per-Gaussian sum, stay those of the tight rectangles.  Everything here is
compared bit for bit against the same loop with bin_margin < 0.
"""

import numpy as np
import pytest

from gs2d_inputs import random_gaussians, smooth_noise_target

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def fit_steps(gs, cfg, p0, target, steps, W, H, max_entries=0):
    from paper_2505_09324_gb300 import _native as nat
    r = gs.GaussianRasterizer(W, H, p0.shape[1], max_entries=max_entries, config=cfg)
    p = to_dev(p0)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    t = to_dev(target)
    s = torch.cuda.current_stream().cuda_stream
    nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
    for _ in range(steps):
        nat.fit_step(r.plan, r.ws_ptr, t.data_ptr(), p.data_ptr(), m.data_ptr(), v.data_ptr(), s)
    torch.cuda.synchronize()
    return p, m, v, r


def assert_same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x, y), f"{(x != y).sum().item()} entries differ"


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("fast", [False, True])
def test_fit_steps_bit_identical_to_per_iteration_binning(gs, tile, fast):
    W, H, n, steps = 203, 131, 700, 40  # ragged in every tile size
    p0 = random_gaussians(n, W, H, seed=41, l_range=(1.0, 9.0))
    target = smooth_noise_target(W, H, seed=42)
    mk = gs.RasterConfig.fast_fit if fast else gs.RasterConfig
    ref = fit_steps(gs, mk(tile=tile, bin_margin=-1.0), p0, target, steps, W, H)
    for margin in (0.0, 2.0, 12.0):
        got = fit_steps(gs, mk(tile=tile, bin_margin=margin), p0, target, steps, W, H)
        assert got[3].status() == 0
        assert_same(got[:3], ref[:3])
        rebins = got[3].rebins()
        assert 1 <= rebins <= steps
    assert ref[3].rebins() == 0  # per-iteration binning keeps no lists


def test_wide_margin_rebuilds_rarely(gs):
    """Plain Adam (lr 1e-2) moves a box edge by a few hundredths of a pixel
    per step: with a 4-pixel margin the lists outlive most iterations."""
    W, H, n, steps = 160, 112, 400, 60
    p0 = random_gaussians(n, W, H, seed=43, l_range=(1.5, 6.0))
    target = smooth_noise_target(W, H, seed=44)
    ref = fit_steps(gs, gs.RasterConfig(bin_margin=-1.0), p0, target, steps, W, H)
    got = fit_steps(gs, gs.RasterConfig(bin_margin=4.0), p0, target, steps, W, H)
    assert_same(got[:3], ref[:3])
    assert got[3].rebins() < steps // 2


def test_encode_frame_and_batch_identical(gs):
    W, H, n, iters = 96, 80, 150, 30
    p0 = random_gaussians(n, W, H, seed=45, l_range=(1.5, 7.0))
    target = to_dev(smooth_noise_target(W, H, seed=46))
    outs = []
    for margin in (-1.0, 2.0):
        r = gs.GaussianRasterizer(W, H, n, config=gs.RasterConfig.fast_fit(bin_margin=margin))
        p = to_dev(p0)
        o = r.encode_frame(target, p, iters, check_every=10)
        assert o["status"] == 0
        outs.append((p, o["trace"], o["psnr"]))
    assert torch.equal(outs[0][0], outs[1][0])
    assert list(outs[0][1]) == list(outs[1][1]) and outs[0][2] == outs[1][2]

    sizes = [(64, 48, 60), (37, 29, 25), (96, 80, 150)]
    P = []
    T = []
    for k, (w, h, nn) in enumerate(sizes):
        P.append(to_dev(random_gaussians(nn, w, h, seed=50 + k, l_range=(1.5, 6.0))))
        T.append(to_dev(smooth_noise_target(w, h, seed=60 + k)))
    res = []
    for margin in (-1.0, 3.0):
        b = gs.BatchRasterizer(sizes, config=gs.RasterConfig.fast_fit(bin_margin=margin))
        pp = b.pack_params(P)
        psnr = b.encode_batch(b.pack_images(T), pp, iters)
        res.append((pp, psnr))
    assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


def test_qat_steps_identical(gs):
    from paper_2505_09324_gb300 import _native as nat
    W, H, n, steps = 96, 64, 120, 15
    p0 = random_gaussians(n, W, H, seed=47, l_range=(1.5, 6.0))
    target = to_dev(smooth_noise_target(W, H, seed=48))
    q = gs.Quantizer([6, 6, 5, 5, 5, 5, 5, 5, 5], refine=True)
    outs = []
    for margin in (-1.0, 2.0):
        r = gs.GaussianRasterizer(W, H, n, config=gs.RasterConfig(bin_margin=margin))
        p = to_dev(p0)
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        s = torch.cuda.current_stream().cuda_stream
        nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
        for _ in range(steps):
            nat.fit_step_qat(r.plan, r.ws_ptr, target.data_ptr(), p.data_ptr(), m.data_ptr(),
                             v.data_ptr(), q.c, s)
        torch.cuda.synchronize()
        outs.append((p, m, v))
    assert_same(outs[0], outs[1])


def test_interleaved_eager_binning_invalidates_lists(gs):
    """gs2d_prepare (tight lists) between fit steps: the next fit step must
    rebuild its widened lists, and every render in between sees the same
    images as with per-iteration binning."""
    from paper_2505_09324_gb300 import _native as nat
    W, H, n = 120, 88, 200
    p0 = random_gaussians(n, W, H, seed=49, l_range=(1.5, 7.0))
    t = to_dev(smooth_noise_target(W, H, seed=50))
    outs = []
    for margin in (-1.0, 5.0):
        r = gs.GaussianRasterizer(W, H, n, config=gs.RasterConfig.fast_fit(bin_margin=margin))
        p = to_dev(p0)
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        s = torch.cuda.current_stream().cuda_stream
        nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
        imgs = []
        for it in range(24):
            nat.fit_step(r.plan, r.ws_ptr, t.data_ptr(), p.data_ptr(), m.data_ptr(),
                         v.data_ptr(), s)
            if it % 6 == 5:
                imgs.append(r.render_fwd().clone())   # the retained lists of the last step
                r.prepare(p)
                imgs.append(r.render_fwd().clone())   # tight lists of the current params
        torch.cuda.synchronize()
        outs.append((p, m, v, imgs, r.rebins()))
    assert_same(outs[0][:3], outs[1][:3])
    for a, b in zip(outs[0][3], outs[1][3]):
        assert torch.equal(a, b)
    assert outs[1][4] >= 4  # one rebuild after each interleaved prepare


def test_widened_lists_over_capacity_fall_back_to_tight_lists(gs):
    """A plan sized for the tight lists but not the widened ones: each rebuild
    lists the tight rectangles instead, with the results of per-iteration
    binning; a plan too small for the tight lists reports GS2D_ERR_CAPACITY
    and leaves the parameters untouched."""
    from paper_2505_09324_gb300 import _native as nat
    W, H, n, steps = 128, 128, 300, 12
    p0 = random_gaussians(n, W, H, seed=51, l_range=(1.0, 4.0))
    target = smooth_noise_target(W, H, seed=52)
    probe = gs.GaussianRasterizer(W, H, n, config=gs.RasterConfig(tile=8))
    probe.prepare(to_dev(p0))
    tight = probe.read_bins()["n_entries"]
    ref = fit_steps(gs, gs.RasterConfig(tile=8, bin_margin=-1.0), p0, target, steps, W, H,
                    max_entries=2 * tight)
    assert ref[3].status() == 0
    got = fit_steps(gs, gs.RasterConfig(tile=8, bin_margin=24.0), p0, target, steps, W, H,
                    max_entries=2 * tight)
    assert got[3].status() == 0
    assert_same(got[:3], ref[:3])
    assert got[3].rebins() >= 1
    # too small for the tight lists too
    p, m, v, r = fit_steps(gs, gs.RasterConfig(tile=8, bin_margin=24.0), p0, target, 1, W, H,
                           max_entries=tight - 1)
    assert r.status() == nat.GS2D_ERR_CAPACITY
    assert torch.equal(p, to_dev(p0))


@pytest.mark.parametrize("tile,fast", [(8, False), (16, True), (32, False), (32, True)])
def test_fit_step_equals_pframe_step_with_everything_selected(gs, tile, fast):
    """The fit step (retained widened lists, every tile rendered) and the
    P-frame step with every Gaussian selected (tight lists rebuilt each step,
    only the tiles some Gaussian covers rendered, the masked update) must give
    the same Gaussians and moments bit for bit, step after step, on a frame
    of many tiles per Gaussian."""
    from paper_2505_09324_gb300 import _native as nat
    W, H, n, steps = 640, 360, 5000, 8
    p0 = random_gaussians(n, W, H, seed=53, l_range=(1.0, 24.0))
    t = to_dev(smooth_noise_target(W, H, seed=54))
    mk = gs.RasterConfig.fast_fit if fast else gs.RasterConfig
    r = gs.GaussianRasterizer(W, H, n, config=mk(tile=tile))
    s = int(torch.cuda.current_stream().cuda_stream)
    a, b = to_dev(p0), to_dev(p0)
    ma, va, mb, vb = (torch.empty_like(a) for _ in range(4))
    sel = torch.ones(n, dtype=torch.uint8, device="cuda")
    nat.fit_reset(r.plan, r.ws_ptr, ma.data_ptr(), va.data_ptr(), s)
    for _ in range(steps):
        nat.fit_step(r.plan, r.ws_ptr, t.data_ptr(), a.data_ptr(), ma.data_ptr(), va.data_ptr(),
                     s)
    r2 = gs.GaussianRasterizer(W, H, n, config=mk(tile=tile))
    nat.fit_reset(r2.plan, r2.ws_ptr, mb.data_ptr(), vb.data_ptr(), s)
    for _ in range(steps):
        nat.pframe_step(r2.plan, r2.ws_ptr, t.data_ptr(), b.data_ptr(), mb.data_ptr(),
                        vb.data_ptr(), sel.data_ptr(), s)
    torch.cuda.synchronize()
    assert r.status() == 0 and r2.status() == 0
    assert_same((a, ma, va), (b, mb, vb))
    assert not torch.equal(a, to_dev(p0))


def test_empty_gaussian_sets(gs):
    """No Gaussians at all, with retained and with per-iteration lists; and an
    empty clip in a batch, whose other clip must fit exactly as alone."""
    from paper_2505_09324_gb300 import _native as nat
    W, H = 70, 50
    t = to_dev(smooth_noise_target(W, H, seed=55))
    s = int(torch.cuda.current_stream().cuda_stream)
    for margin in (-1.0, 4.0):
        r = gs.GaussianRasterizer(W, H, 0, config=gs.RasterConfig(bin_margin=margin))
        p = torch.zeros((9, 0), device="cuda")
        o = r.encode_frame(t, p, 5, check_every=5)
        assert o["status"] == 0 and o["iters"] == 5
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
        for _ in range(3):
            nat.fit_step(r.plan, r.ws_ptr, t.data_ptr(), p.data_ptr(), m.data_ptr(),
                         v.data_ptr(), s)
        torch.cuda.synchronize()
        assert r.status() == 0
    w2, h2, n2, iters = 64, 48, 80, 20
    p2 = to_dev(random_gaussians(n2, w2, h2, seed=56, l_range=(1.5, 6.0)))
    t2 = to_dev(smooth_noise_target(w2, h2, seed=57))
    cfg = gs.RasterConfig.fast_fit()
    b = gs.BatchRasterizer([(W, H, 0), (w2, h2, n2)], config=cfg)
    pp = p2.clone()
    b.encode_batch(b.pack_images([t, t2]), pp, iters)
    alone = p2.clone()
    gs.GaussianRasterizer(w2, h2, n2, config=cfg).encode_frame(t2, alone, iters,
                                                                check_every=iters)
    assert torch.equal(pp, alone)
