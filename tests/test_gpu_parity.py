"""GPU path vs the CPU oracle, through the C ABI (ctypes binding).

Bars: tile keys, sorted order, per-tile ranges and tile counts bit-exact;
images within 1e-5 absolute per channel (after accounting for pairs whose
cut-off decision FP32 may take either way, reported by the oracle as an
interval); gradients within 1e-3 relative to the oracle value plus 1e-3 of the
RMS of that parameter row (absolute floor for near-cancelling sums), plus the
oracle's bound for undecidable pairs.
"""

import math

import numpy as np
import pytest

from gs2d_inputs import (conferencing_frame, conferencing_gaussians, random_gaussians,
                         smooth_noise_target)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GRAD_REL = 1e-3


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import build
    build.build()
    import paper_2505_09324_gb300 as pkg
    from paper_2505_09324_gb300 import _native
    _native.load()
    assert torch.cuda.is_available()
    return pkg


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def check_bins(gs, oracle, p, W, H, max_entries=0, separate=False, sigma_cut=4.5,
               alpha_min=1 / 255):
    cfg = gs.RasterConfig(sigma_cut=sigma_cut, alpha_min=alpha_min)
    r = gs.GaussianRasterizer(W, H, p.shape[1], max_entries=max_entries, config=cfg)
    if separate:
        r.project(to_dev(p))
        r.bin_sort()
    else:
        r.prepare(to_dev(p))
    got = r.read_bins()
    ocfg = oracle.Config(sigma_cut=sigma_cut, alpha_min=alpha_min)
    keys, ranges = oracle.sorted_keys(p, W, H, ocfg)
    _, count, total = oracle.tile_rects(p, W, H, ocfg)
    assert got["n_entries"] == total
    np.testing.assert_array_equal(got["keys"].astype(np.uint64), keys >> np.uint64(32))
    np.testing.assert_array_equal(got["values"].astype(np.uint64), keys & np.uint64(0xFFFFFFFF))
    np.testing.assert_array_equal(got["ranges"], ranges)
    np.testing.assert_array_equal(got["counts"], count)
    return r


def check_image(img_gpu, ref, lo, hi, tol=IMG_TOL):
    g = img_gpu.detach().cpu().numpy().astype(np.float64)
    below = (ref + lo - tol) - g
    above = g - (ref + hi + tol)
    worst = max(below.max(initial=0.0), above.max(initial=0.0))
    assert worst <= 0.0, f"image off by {worst + tol:.3e} beyond the interval"


def loss_bound(ref_img, lo, hi, target, clamp=False, tol=IMG_TOL):
    """Largest |L_gpu - L_ref| allowed when every pixel of the GPU image lies in
    [ref + lo - tol, ref + hi + tol]: |a^2 - b^2| <= e (2 |b| + e) per element,
    plus 1e-5 relative for the FP32 accumulation of the sum."""
    e = tol + np.maximum(-lo, hi)
    c = np.clip(ref_img, 0, 1) if clamp else ref_img
    d = np.abs(c - np.asarray(target, np.float64))
    m = ref_img.size
    return (2 * np.sum(d * e) + np.sum(e * e)) / m + 1e-5 * np.sum(d * d) / m


def check_grads(g_gpu, ref, unc, rel=GRAD_REL, which=None):
    g = g_gpu.detach().cpu().numpy().astype(np.float64)
    if which is not None:
        g, ref, unc = g[:, which], ref[:, which], unc[:, which]
    rms = np.sqrt(np.mean(ref * ref, axis=1, keepdims=True))
    bound = rel * np.abs(ref) + rel * rms + unc
    err = np.abs(g - ref)
    bad = err > bound
    assert not bad.any(), (f"{bad.sum()} gradient entries off; worst ratio "
                           f"{(err / np.maximum(bound, 1e-30)).max():.3f}")


CASES = [
    ("config1_256x256_2000", 256, 256, 2000, 0),
    ("ragged_100x70_300", 100, 70, 300, 11),
    ("ragged_33x17_40", 33, 17, 40, 5),
]


@pytest.mark.parametrize("name,W,H,n,seed", CASES)
def test_bins_bit_exact(gs, oracle, name, W, H, n, seed):
    check_bins(gs, oracle, random_gaussians(n, W, H, seed=seed), W, H)


@pytest.mark.parametrize("name,W,H,n,seed", CASES)
def test_bins_bit_exact_separate_calls(gs, oracle, name, W, H, n, seed):
    check_bins(gs, oracle, random_gaussians(n, W, H, seed=seed), W, H, separate=True)


def test_bins_bit_exact_full_size_1080p(gs, oracle):
    frame, mask = conferencing_frame(1920, 1080, seed=1)
    p = conferencing_gaussians(frame, mask, 20000, seed=1)
    check_bins(gs, oracle, p, 1920, 1080)
    check_bins(gs, oracle, p, 1920, 1080, separate=True)


@pytest.mark.parametrize("n", [20, 50, 100, 200, 400, 700])
def test_bins_every_list_length_path(gs, oracle, n):
    """Every Gaussian covers all four tiles of a 32 x 32 frame, so each tile's
    list holds all n: exercises the register sorts for <= 32 .. 512 entries and
    the shared-memory sort beyond."""
    p = random_gaussians(n, 32, 32, seed=n, l_range=(6.0, 8.0))
    p[0:2] = 16.0 + np.random.Generator(np.random.PCG64(n)).uniform(-2, 2, (2, n))
    check_bins(gs, oracle, p, 32, 32)


def test_bins_edge_cases(gs, oracle):
    W, H = 80, 48
    p = random_gaussians(64, W, H, seed=3)
    p[0, 0] = np.nan             # non-finite
    p[2, 1] = p[4, 1] = 1e-6      # degenerate covariance
    p[8, 2] = 0.001               # invisible weight
    p[0, 3] = -500.0              # off-image
    p[2, 4] = p[4, 4] = 400.0     # covers every tile
    p[3, 5] = 1e30                # huge shear (finite)
    p[6, 6] = np.nan              # non-finite colour
    check_bins(gs, oracle, p, W, H)
    check_bins(gs, oracle, np.zeros((9, 0), np.float32), W, H)
    # a single-tile frame (no radix pass) and a wider cut-off
    check_bins(gs, oracle, random_gaussians(5, 16, 16, seed=2), 16, 16)
    check_bins(gs, oracle, random_gaussians(5, 1, 1, seed=2), 1, 1, separate=True)
    check_bins(gs, oracle, random_gaussians(200, 100, 70, seed=9), 100, 70, sigma_cut=8.0,
               alpha_min=1e-6)


@pytest.mark.parametrize("name,W,H,n,seed", CASES)
def test_render_fwd_matches_oracle(gs, oracle, name, W, H, n, seed):
    p = random_gaussians(n, W, H, seed=seed)
    r = gs.GaussianRasterizer(W, H, n)
    r.prepare(to_dev(p))
    img = r.render_fwd()
    ref, lo, hi = oracle.render(p, W, H, ambiguity=True)
    check_image(img, ref, lo, hi)


def test_render_fwd_edge_cases(gs, oracle):
    W, H = 48, 40
    p = random_gaussians(30, W, H, seed=8)
    p[0, 0] = np.nan
    p[2, 1] = p[4, 1] = 1e-6
    p[2, 4] = p[4, 4] = 60.0   # one large Gaussian covering the frame
    p[8, 5] = -0.7             # negative weight
    r = gs.GaussianRasterizer(W, H, p.shape[1])
    r.prepare(to_dev(p))
    ref, lo, hi = oracle.render(p, W, H, ambiguity=True)
    check_image(r.render_fwd(), ref, lo, hi)
    # empty set renders zero
    r0 = gs.GaussianRasterizer(W, H, 0)
    r0.prepare(torch.zeros((9, 0), device="cuda"))
    assert float(r0.render_fwd().abs().max()) == 0.0
    # a 1 x 1 frame
    q = np.array([[0.5], [0.5], [2.0], [0.0], [2.0], [0.25], [0.5], [1.0], [0.8]], np.float32)
    r1 = gs.GaussianRasterizer(1, 1, 1)
    r1.prepare(to_dev(q))
    np.testing.assert_allclose(r1.render_fwd().cpu().numpy()[:, 0, 0], 0.8 * q[5:8, 0], atol=1e-6)


def test_long_tile_lists_span_several_batches(gs, oracle):
    """More than 256 Gaussians in one tile exercises multi-batch staging."""
    W, H = 32, 32
    g = np.random.Generator(np.random.PCG64(4))
    n = 700
    p = random_gaussians(n, W, H, seed=19)
    p[0] = g.uniform(4, 12, n)
    p[1] = g.uniform(4, 12, n)
    p[5:8] *= 0.05
    r = gs.GaussianRasterizer(W, H, n)
    r.prepare(to_dev(p))
    ref, lo, hi = oracle.render(p, W, H, ambiguity=True)
    check_image(r.render_fwd(), ref, lo, hi)
    dimg = smooth_noise_target(W, H, seed=2).astype(np.float64) - 0.5
    gref, unc = oracle.render_grad(p, W, H, dimg, uncertainty=True)
    check_grads(r.render_bwd(to_dev(p), to_dev(dimg)), gref, unc)


@pytest.mark.parametrize("name,W,H,n,seed", CASES)
def test_render_bwd_matches_oracle(gs, oracle, name, W, H, n, seed):
    p = random_gaussians(n, W, H, seed=seed)
    dimg = (smooth_noise_target(W, H, seed=seed + 1).astype(np.float64) - 0.5) * 1e-3
    r = gs.GaussianRasterizer(W, H, n)
    r.prepare(to_dev(p))
    grads = r.render_bwd(to_dev(p), to_dev(dimg))
    gref, unc = oracle.render_grad(p, W, H, dimg, uncertainty=True)
    check_grads(grads, gref, unc)


@pytest.mark.parametrize("name,W,H,n,seed", CASES)
def test_render_l2_matches_oracle(gs, oracle, name, W, H, n, seed):
    p = random_gaussians(n, W, H, seed=seed)
    target = smooth_noise_target(W, H, seed=seed + 2)
    r = gs.GaussianRasterizer(W, H, n)
    r.prepare(to_dev(p))
    grads, loss, img = r.render_l2(to_dev(p), to_dev(target), want_image=True)
    res = oracle.loss_and_grad(p, target)
    check_image(img, res["img"], res["amb_lo"], res["amb_hi"])
    loss = loss.cpu().numpy()
    lo, hi = res["amb_lo"], res["amb_hi"]
    assert abs(loss[0] - res["loss"]) <= loss_bound(res["img"], lo, hi, target)
    mse_c = 10 ** (-oracle.psnr(res["img"], target) / 10)
    assert abs(loss[1] - mse_c) <= loss_bound(res["img"], lo, hi, target, clamp=True)
    check_grads(grads, res["grad"], res["grad_unc"])


@pytest.fixture(scope="module")
def full_size_case(oracle):
    """The benchmark's workload (1920x1080 conferencing frame, 20k Gaussians from
    the oracle's ROI initialiser, background positions of seed 11) with oracle
    references at sampled pixels and for sampled Gaussians."""
    from gs2d_inputs import background_positions
    from oracle import superpixel
    W, H, n = 1920, 1080, 20000
    frame, mask = conferencing_frame(W, H, seed=1)
    bg = background_positions(mask, n, seed=11)
    p = superpixel.roi_init(frame, mask, n, 0.7, bg.T.astype(np.float64))[0].astype(np.float32)
    g = np.random.Generator(np.random.PCG64(77))
    xy = np.stack([g.integers(0, W, 3000), g.integers(0, H, 3000)], axis=1)
    pix = oracle.render_pixels(p, xy, ambiguity=True)
    which = np.sort(g.choice(n, 300, replace=False))
    res = oracle.loss_and_grad(p, frame, fast=True, which=which)
    return {"W": W, "H": H, "n": n, "frame": frame, "p": p, "xy": xy, "pix": pix,
            "which": which, "res": res}


FULL_SCHEDULES = [(t, s, la) for t in (8, 16, 32) for s in (32, 64, 128) for la in (0, 1)] + [
    (16, 256, 0), (32, 256, 1)]


@pytest.mark.parametrize("tile,stage,launch", FULL_SCHEDULES)
def test_full_size_1080p_sampled(gs, full_size_case, tile, stage, launch):
    """Config-2 size (1920x1080, 20k Gaussians) in every launch configuration the
    benchmark's autotuner may pick: sampled pixels of the render and sampled
    Gaussians of the fused L2 gradient against the oracle."""
    c = full_size_case
    W, H, n, frame, p = c["W"], c["H"], c["n"], c["frame"], c["p"]
    cfg = gs.RasterConfig(tile=tile, stage=stage, launch=launch)
    r = gs.GaussianRasterizer(W, H, n, config=cfg)
    r.prepare(to_dev(p))
    grads, loss, img = r.render_l2(to_dev(p), to_dev(frame), want_image=True)
    assert r.status() == 0
    xy = c["xy"]
    ref, lo, hi = c["pix"]
    gi = img.cpu().numpy()[:, xy[:, 1], xy[:, 0]].astype(np.float64)
    assert np.all(gi >= ref + lo - IMG_TOL) and np.all(gi <= ref + hi + IMG_TOL)
    res = c["res"]
    assert abs(float(loss[0]) - res["loss"]) <= loss_bound(res["img"], res["amb_lo"],
                                                           res["amb_hi"], frame)
    # RMS floor from all Gaussians' oracle gradient would need them all; use the sample
    check_grads(grads, res["grad"], res["grad_unc"], which=c["which"])


def test_capacity_overflow_is_reported(gs, oracle):
    from paper_2505_09324_gb300 import _native
    W, H = 64, 64
    p = random_gaussians(100, W, H, seed=2)
    _, _, total = oracle.tile_rects(p, W, H)
    r = gs.GaussianRasterizer(W, H, 100, max_entries=total - 1)
    r.prepare(to_dev(p))
    assert r.status() == _native.GS2D_ERR_CAPACITY
    assert float(r.render_fwd().abs().max()) == 0.0
    assert r.status(reset=True) == _native.GS2D_ERR_CAPACITY
    assert r.status() == _native.GS2D_OK
    r2 = gs.GaussianRasterizer(W, H, 100, max_entries=total)
    r2.prepare(to_dev(p))
    assert r2.status() == _native.GS2D_OK


def test_adam_matches_oracle(gs, oracle):
    g = np.random.Generator(np.random.PCG64(3))
    n = 1001
    p = g.normal(size=(9, n))
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    tp, tm, tv = to_dev(p), to_dev(m), to_dev(v)
    for step in range(1, 6):
        grad = g.normal(size=p.shape) * 10.0 ** g.uniform(-3, 0, size=p.shape)
        gs.adam_step(tp, to_dev(grad), tm, tv, step)
        p, m, v = oracle.adam_step(p, grad, m, v, step)
    np.testing.assert_allclose(tp.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(tv.cpu().numpy(), v, rtol=1e-4, atol=1e-12)


def test_adam_mask_freezes_gaussians(gs):
    n = 40
    p = torch.randn(9, n, device="cuda")
    p0 = p.clone()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    mask[::3] = 1
    gs.adam_step(p, torch.ones_like(p), m, v, 1, mask=mask)
    moved = (p != p0).any(dim=0).cpu().numpy()
    np.testing.assert_array_equal(moved, mask.cpu().numpy().astype(bool))


def test_encode_loop_tracks_oracle_trajectory(gs, oracle):
    """64x64 frame, 50 Gaussians, 50 iterations: the GPU fit loop (captured
    graph) against a loop driven by oracle gradients and oracle Adam."""
    W, H, n, iters = 64, 64, 50, 50
    p0 = random_gaussians(n, W, H, seed=23, l_range=(2.0, 6.0))
    target = smooth_noise_target(W, H, seed=24)
    r = gs.GaussianRasterizer(W, H, n)
    tp = to_dev(p0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        out = r.encode_frame(to_dev(target), tp, iters, check_every=10, stream=stream)
    stream.synchronize()
    assert out["status"] == 0 and out["iters"] == iters
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for it in range(1, iters + 1):
        res = oracle.loss_and_grad(p.astype(np.float32), target)
        p, m, v = oracle.adam_step(p, res["grad"], m, v, it)
    got = tp.cpu().numpy().astype(np.float64)
    scale = np.abs(p).max(axis=1, keepdims=True) + 1e-3
    assert np.abs(got - p).max() / 1.0 < 5e-2
    assert (np.abs(got - p) / scale).max() < 2e-3
    l_gpu = oracle.l2_loss(oracle.render(got, W, H), target)[0]
    l_ref = oracle.l2_loss(oracle.render(p, W, H), target)[0]
    assert abs(l_gpu - l_ref) <= 1e-3 * l_ref
    # the fit reduced the loss
    assert l_ref < 0.5 * oracle.l2_loss(oracle.render(p0, W, H), target)[0]


def test_fast_schedule_tracks_oracle_trajectory(gs, oracle):
    """The fit loop with the per-group learning rates and decay of the fast
    schedule against an oracle-driven loop applying Adam row group by row
    group with lr * scale * decay^(t-1)."""
    from paper_2505_09324_gb300.raster import FAST_FIT
    W, H, n, iters = 64, 64, 50, 20
    p0 = random_gaussians(n, W, H, seed=25, l_range=(2.0, 6.0))
    target = smooth_noise_target(W, H, seed=26)
    cfg = gs.RasterConfig.fast_fit()
    r = gs.GaussianRasterizer(W, H, n, config=cfg)
    tp = to_dev(p0)
    r.encode_frame(to_dev(target), tp, iters, check_every=iters)
    rows = {"lr_mu": slice(0, 2), "lr_shape": slice(2, 5), "lr_color": slice(5, 8),
            "lr_weight": slice(8, 9)}
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for it in range(1, iters + 1):
        g = oracle.loss_and_grad(p.astype(np.float32), target)["grad"]
        for key, sl in rows.items():
            lr = cfg.lr * FAST_FIT[key] * FAST_FIT["lr_decay"] ** (it - 1)
            p[sl], m[sl], v[sl] = oracle.adam_step(p[sl], g[sl], m[sl], v[sl], it, lr=lr)
    got = tp.cpu().numpy().astype(np.float64)
    l_gpu = oracle.l2_loss(oracle.render(got, W, H), target)[0]
    l_ref = oracle.l2_loss(oracle.render(p, W, H), target)[0]
    l_0 = oracle.l2_loss(oracle.render(p0, W, H), target)[0]
    assert abs(l_gpu - l_ref) <= 2e-2 * l_ref, (l_gpu, l_ref)
    assert l_ref < 0.2 * l_0
    scale = np.abs(p).max(axis=1, keepdims=True) + 1e-3
    assert np.median(np.abs(got - p) / scale) < 1e-3


@pytest.mark.parametrize("mode,check_every", [("cap", 7), ("early", 5), ("never", 10)])
def test_device_driven_loop_equals_host_driven_loop(gs, mode, check_every):
    """On a non-default stream gs2d_encode_frame runs the whole fit loop as one
    graph whose WHILE node the device stops (PSNR checked on the device every
    check_every iterations, one host read at the end); on the legacy default
    stream the host drives it.  Both give the same Gaussians bit for bit, the
    same iteration count and the same PSNR trace: with no target (the cap,
    not a multiple of check_every), a target met at the third check, and one
    never met."""
    W, H, n, iters = 96, 80, 120, 53
    p0 = to_dev(random_gaussians(n, W, H, seed=27, l_range=(2.0, 6.0)))
    target = to_dev(smooth_noise_target(W, H, seed=28))

    def run(name, target_psnr):
        r = gs.GaussianRasterizer(W, H, n)
        p = p0.clone()
        s = torch.cuda.default_stream() if name == "host" else torch.cuda.Stream()
        with torch.cuda.stream(s):
            o = r.encode_frame(target, p, iters, target_psnr=target_psnr,
                               check_every=check_every, stream=s)
        s.synchronize()
        return p, o

    goal = {"cap": 0.0, "never": 99.0}.get(mode)
    if goal is None:
        goal = run("host", 0.0)[1]["trace"][2]  # reached at the third check
    (ph, oh), (pd, od) = run("host", goal), run("device", goal)
    assert oh["status"] == od["status"] == 0
    assert oh["iters"] == od["iters"] and oh["trace"] == od["trace"] and oh["psnr"] == od["psnr"]
    assert torch.equal(ph, pd)
    if mode == "early":
        assert od["iters"] <= 3 * check_every and od["psnr"] >= goal
    else:
        assert od["iters"] == iters and len(od["trace"]) == -(-iters // check_every)
