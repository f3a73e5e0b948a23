"""P-frames (selective Gaussian optimisation): the selection of the Gaussians
that contribute to changed pixels against the oracle, a P-frame iteration
against a full iteration, and a selective sequence fit."""

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


def scene(W, H, n, seed, frames=2):
    mo = random_motion(seed)
    fr = [conferencing_frame(W, H, seed=seed, t=t, motion=mo) for t in range(frames)]
    return fr, mo


def fitted(gs, fr, n, seed, iters=150):
    W, H = fr[0][0].shape[2], fr[0][0].shape[1]
    f0 = torch.from_numpy(fr[0][0]).cuda()
    bg = torch.from_numpy(background_positions(fr[0][1], n, seed=seed + 1)).cuda()
    p, _ = gs.roi_init(f0, torch.from_numpy(fr[0][1].astype(np.uint8)).cuda(), n, 0.7, bg)
    r = gs.GaussianRasterizer(W, H, n)
    if iters:
        r.encode_frame(f0, p, iters, target_psnr=0.0, check_every=iters)
    return p, r


def test_selection_matches_oracle(gs, oracle):
    W, H, n = 160, 96, 400
    fr, _ = scene(W, H, n, seed=3)
    p, r = fitted(gs, fr, n, seed=3, iters=60)
    pn = p.cpu().numpy()
    # the reference: the oracle's render of the reference Gaussians, in FP32
    ref = oracle.render(pn, W, H).astype(np.float32)
    cur = fr[1][0]
    thr = np.float32(0.02)
    r.prepare(p)
    sel, cnt = r.select_changed(torch.from_numpy(ref).cuda(), torch.from_numpy(cur).cuda(),
                                float(thr))
    got = sel.cpu().numpy().astype(bool)
    assert cnt == int(got.sum())
    # changed pixels: max over channels of |ref - frame| > threshold, in FP32
    d = np.max(np.abs(ref - cur), axis=0)
    ys, xs = np.nonzero(d > thr)
    assert 0 < len(xs) < W * H
    definite, ambiguous = oracle.contributes(pn, np.stack([xs, ys], axis=1))
    must = definite.any(axis=0)
    may = must | ambiguous.any(axis=0)
    assert np.all(got[must]), "a Gaussian reaching a changed pixel was not selected"
    assert np.all(may[got]), "a Gaussian reaching no changed pixel was selected"
    assert 0 < must.sum() < n


def test_pframe_step_is_the_full_step_on_the_selected(gs):
    from paper_2505_09324_gb300 import _native as nat
    W, H, n = 200, 120, 600
    fr, _ = scene(W, H, n, seed=5)
    p, r = fitted(gs, fr, n, seed=5, iters=60)
    cur = torch.from_numpy(fr[1][0]).cuda()
    r.prepare(p)
    ref = r.render_fwd()
    sel, cnt = r.select_changed(ref, cur, 0.03)
    assert 0 < cnt < n
    s = int(torch.cuda.current_stream().cuda_stream)
    a, b = p.clone(), p.clone()
    ma, va, mb, vb = (torch.empty_like(p) for _ in range(4))
    nat.fit_reset(r.plan, r.ws_ptr, ma.data_ptr(), va.data_ptr(), s)
    nat.fit_step(r.plan, r.ws_ptr, cur.data_ptr(), a.data_ptr(), ma.data_ptr(), va.data_ptr(), s)
    nat.fit_reset(r.plan, r.ws_ptr, mb.data_ptr(), vb.data_ptr(), s)
    nat.pframe_step(r.plan, r.ws_ptr, cur.data_ptr(), b.data_ptr(), mb.data_ptr(),
                    vb.data_ptr(), sel.data_ptr(), s)
    torch.cuda.synchronize()
    on = sel.bool()
    assert torch.equal(a[:, on], b[:, on])        # same update, bit for bit
    assert torch.equal(b[:, ~on], p[:, ~on])      # the rest untouched
    assert not torch.equal(b[:, on], p[:, on])


def test_selective_sequence(gs):
    W, H, n = 320, 180, 1200
    fr, _ = scene(W, H, n, seed=7, frames=4)
    frames = [torch.from_numpy(f).cuda() for f, _ in fr]
    p0, r = fitted(gs, fr, n, seed=7, iters=0)
    stream = torch.cuda.Stream()
    full, sel = p0.clone(), p0.clone()
    with torch.cuda.stream(stream):
        a = gs.encode_sequence(r, frames, full, 300, 80, stream=stream)
        b = gs.encode_sequence(r, frames, sel, 300, 80, stream=stream, selective_threshold=0.02)
    stream.synchronize()
    for x, y in zip(a[1:], b[1:]):
        assert 0 < y["selected"] < n
        assert y["psnr"] > x["psnr"] - 1.5, (x, y)
