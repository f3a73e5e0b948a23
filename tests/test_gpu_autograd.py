"""torch.autograd integration: gradients of an arbitrary loss through the
rasterizer's backward kernels, against the oracle gradient and against
central finite differences of the GPU forward, on a 64x64 crop of the
conferencing scene (the frame-sequence workload's scene)."""

import numpy as np
import pytest

from gs2d_inputs import conferencing_frame, conferencing_gaussians

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crop():
    W = H = 64
    frame, mask = conferencing_frame(1920, 1080, seed=2)
    # a crop straddling the subject's left edge
    y0 = 540 - 32
    xs = np.nonzero(mask[540])[0]
    x0 = int(xs.min()) - 32
    full = conferencing_gaussians(frame, mask, 20000, seed=2)
    sel = ((full[0] > x0 - 8) & (full[0] < x0 + W + 8) & (full[1] > y0 - 8)
           & (full[1] < y0 + H + 8))
    p = full[:, sel].copy()
    p[0] -= x0
    p[1] -= y0
    target = np.ascontiguousarray(frame[:, y0:y0 + H, x0:x0 + W])
    return p, target, W, H


def test_autograd_matches_oracle_gradient(crop, oracle):
    from paper_2505_09324_gb300 import GaussianRasterizer
    from paper_2505_09324_gb300.autograd import rasterize
    p, target, W, H = crop
    r = GaussianRasterizer(W, H, p.shape[1])
    tp = torch.from_numpy(p).cuda().requires_grad_(True)
    img = rasterize(tp, r)
    loss = ((img - torch.from_numpy(target).cuda()) ** 2).mean()
    loss.backward()
    res = oracle.loss_and_grad(p, target)
    g = tp.grad.cpu().numpy().astype(np.float64)
    ref, unc = res["grad"], res["grad_unc"]
    rms = np.sqrt(np.mean(ref * ref, axis=1, keepdims=True))
    assert np.all(np.abs(g - ref) <= 1e-3 * np.abs(ref) + 1e-3 * rms + unc)


def test_autograd_matches_finite_differences(crop):
    """Against central differences of the GPU forward.  The cut-off makes the
    loss piecewise smooth: moving a Gaussian moves its cut-off ellipse, which
    adds a boundary term that the analytic gradient of the rasterizer leaves
    out (a few percent for positions at the default cut).  The check therefore
    runs with the cut-off pushed out to sigma <= 40 (exp(-40) ~ 4e-18), where
    the loss is smooth to FP32 precision."""
    from paper_2505_09324_gb300 import GaussianRasterizer, RasterConfig
    from paper_2505_09324_gb300.autograd import rasterize
    p, target, W, H = crop
    r = GaussianRasterizer(W, H, p.shape[1], config=RasterConfig(sigma_cut=40.0, alpha_min=1e-30))
    T = torch.from_numpy(target).cuda().double()
    weights = torch.from_numpy(np.random.Generator(np.random.PCG64(3)).uniform(
        0.5, 1.5, (3, H, W))).cuda()

    def L(x):
        with torch.no_grad():
            return float((((rasterize(x, r).double() - T) ** 2) * weights).sum())

    tp = torch.from_numpy(p).cuda().requires_grad_(True)
    loss = (((rasterize(tp, r).double() - T) ** 2) * weights).sum()
    loss.backward()
    g = tp.grad.cpu().numpy().astype(np.float64)
    # the largest gradient entries of the position, shape and colour rows
    checked = 0
    for row in range(9):
        i = int(np.argmax(np.abs(g[row])))
        # 0.01 px for positions, 1 % of the value for factors, colours, weights
        h = 1e-2 if row < 2 else 1e-2 * max(1e-2, abs(float(p[row, i])))
        a = torch.from_numpy(p).cuda()
        b = a.clone()
        a[row, i] += h
        b[row, i] -= h
        fd = (L(a) - L(b)) / (2 * h)
        assert abs(fd - g[row, i]) <= 3e-2 * abs(g[row, i]) + 1e-4, (row, fd, g[row, i])
        checked += 1
    assert checked == 9


def test_backward_rebins_after_workspace_reuse(crop):
    """A second forward on the same rasterizer before backward must not feed
    the first backward stale lists."""
    from paper_2505_09324_gb300 import GaussianRasterizer
    from paper_2505_09324_gb300.autograd import rasterize
    p, target, W, H = crop
    r = GaussianRasterizer(W, H, p.shape[1])
    tp = torch.from_numpy(p).cuda().requires_grad_(True)
    img1 = rasterize(tp, r)
    q = p.copy()
    q[0] += 3.0
    _ = rasterize(torch.from_numpy(q).cuda(), r)  # overwrites the workspace lists
    img1.sum().backward()
    r2 = GaussianRasterizer(W, H, p.shape[1])
    tp2 = torch.from_numpy(p).cuda().requires_grad_(True)
    rasterize(tp2, r2).sum().backward()
    np.testing.assert_array_equal(tp.grad.cpu().numpy(), tp2.grad.cpu().numpy())


@pytest.mark.parametrize("fit", ["encode_frame", "encode_pframe"])
def test_backward_rebins_after_a_fit_on_the_rasterizer(crop, oracle, fit):
    """A fit loop on the rasterizer between forward and backward re-bins the
    workspace for other parameters; the backward must notice and re-bin, and
    its gradient must still be the oracle's."""
    from paper_2505_09324_gb300 import GaussianRasterizer
    from paper_2505_09324_gb300.autograd import rasterize
    p, target, W, H = crop
    r = GaussianRasterizer(W, H, p.shape[1])
    tp = torch.from_numpy(p).cuda().requires_grad_(True)
    T = torch.from_numpy(target).cuda()
    img = rasterize(tp, r)
    q = torch.from_numpy(p).cuda()
    q[0] += 2.5  # moved Gaussians: other tile lists
    if fit == "encode_frame":
        r.encode_frame(T, q, 5, check_every=5)
    else:
        sel = torch.ones(p.shape[1], dtype=torch.uint8, device="cuda")
        r.prepare(q)
        r.encode_pframe(T, q, sel, 5)
    loss = ((img - T) ** 2).mean()
    loss.backward()
    res = oracle.loss_and_grad(p, target)
    g = tp.grad.cpu().numpy().astype(np.float64)
    ref, unc = res["grad"], res["grad_unc"]
    rms = np.sqrt(np.mean(ref * ref, axis=1, keepdims=True))
    assert np.all(np.abs(g - ref) <= 1e-3 * np.abs(ref) + 1e-3 * rms + unc)


def test_check_status_raises_on_capacity_overflow(crop):
    """With check_status, a plan too small for the tile entries raises instead
    of returning the zero image the kernels leave behind."""
    from paper_2505_09324_gb300 import GaussianRasterizer
    from paper_2505_09324_gb300 import _native as nat
    from paper_2505_09324_gb300.autograd import rasterize
    p, target, W, H = crop
    r = GaussianRasterizer(W, H, p.shape[1], max_entries=8)
    tp = torch.from_numpy(p).cuda()
    img = rasterize(tp, r)  # default: no status read, a zero image
    assert float(img.abs().max()) == 0.0
    assert r.status() == nat.GS2D_ERR_CAPACITY
    r2 = GaussianRasterizer(W, H, p.shape[1], max_entries=8)
    with pytest.raises(nat.Gs2dError):
        rasterize(tp, r2, check_status=True)
