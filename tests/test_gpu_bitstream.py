"""Bitstream accounting (Sec. 3.3 B, Eq. 3-4) on the GPU against the oracle:
per-row code lengths of quantised Gaussians (all columns and a selection,
every symbol width, empty input), and a selective sequence with I-frames
every K frames whose totals follow Eq. 3-4 on the coded counts."""

import math

import numpy as np
import pytest

from gs2d_inputs import background_positions, conferencing_frame, random_gaussians, random_motion
from oracle import bitstream as B
from oracle import quant as Q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


def dev_codes(c):
    return torch.from_numpy(np.ascontiguousarray(c).view(np.int16)).cuda()


@pytest.mark.parametrize("n", [0, 1, 33, 5000, 20011])
def test_code_entropy_matches_oracle(gs, n):
    from paper_2505_09324_gb300.quant import code_bits
    rng = np.random.default_rng(n)
    bits = [Q.HALF, 16, 10, 10, 10, 8, 8, 1, 0]
    # skewed symbol distributions: geometric-ish codes, masked to each width
    c = np.zeros((9, n), np.uint16)
    for r, b in enumerate(bits):
        w = 16 if b < 0 else max(b, 1)
        c[r] = np.minimum(rng.geometric(0.02 + 0.05 * r, n) - 1, (1 << w) - 1)
    sel = (rng.random(n) < 0.3).astype(np.uint8)
    for s in (None, sel):
        got = code_bits(dev_codes(c), bits,
                        None if s is None else torch.from_numpy(s).cuda()).cpu().numpy()
        ref = B.code_entropy_bits(c, bits, s)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-8)


def test_code_entropy_of_quantised_gaussians(gs):
    from paper_2505_09324_gb300.quant import code_bits
    p = random_gaussians(20000, 1920, 1080, seed=5)
    q = gs.Quantizer(refine=True)
    codes, _, _ = q.quantize(torch.from_numpy(p).cuda())
    got = code_bits(codes, q.bits).cpu().numpy()
    oc, _, _ = Q.quantize(p, q.bits, refine=True)
    np.testing.assert_allclose(got, B.code_entropy_bits(oc, q.bits), rtol=1e-12)
    # entropy coding never exceeds the fixed-length codes
    assert np.all(got <= np.array([16 if b < 0 else b for b in q.bits]) * 20000 + 1e-6)


def test_selective_sequence_accounting(gs):
    from paper_2505_09324_gb300.quant import frame_bits, sequence_bits
    W, H, n, F, K = 320, 180, 1200, 9, 4
    mo = random_motion(7)
    fr = [conferencing_frame(W, H, seed=7, t=t, motion=mo) for t in range(F)]
    frames = [torch.from_numpy(f).cuda() for f, _ in fr]
    bg = torch.from_numpy(background_positions(fr[0][1], n, seed=8)).cuda()
    p, _ = gs.roi_init(frames[0], torch.from_numpy(fr[0][1].astype(np.uint8)).cuda(), n, 0.7,
                       bg)
    r = gs.GaussianRasterizer(W, H, n)
    q = gs.Quantizer.calibrate([p])
    sizes, sels = [], []

    def on_frame(k, params, sel):
        sizes.append(frame_bits(q, params, sel))
        sels.append(None if sel is None else sel.cpu().numpy())
        # the P-frame size by the oracle: entropy of the selected codes + indices
        oc, _, _ = Q.quantize(params.cpu().numpy(), q.bits, q.lo, q.hi)
        e = B.code_entropy_bits(oc, q.bits, sels[-1]).sum()
        if sel is not None:
            e += int(sels[-1].sum()) * math.ceil(math.log2(n))
        assert sizes[-1] == pytest.approx(e, rel=1e-12)

    recs = gs.encode_sequence(r, frames, p, 150, 40, selective_threshold=0.02, gop=K,
                              on_frame=on_frame)
    counts = [x["coded"] for x in recs]
    assert [c == n for c in counts] == [k % K == 0 for k in range(F)]
    assert all(0 < counts[k] < n for k in range(F) if k % K)
    got = sequence_bits(counts, sizes, K)
    ref = B.sequence_bits(counts, sizes, K)
    for key in ("i_bits", "p_bits", "savings", "total_bits"):
        assert got[key] == pytest.approx(ref[key], rel=1e-12)
    assert got["i_frames"] == 3 and got["p_frames"] == 6
    assert 0 < got["savings"] < got["p_bits"]


def test_frame_bits_i_frame_and_refined_ranges(gs):
    """gs2d_frame_bits on an I-frame (no selection: no index bits) with a
    quantiser that refines its ranges per frame (two float32 per uniform row
    ride along) against the oracle's code lengths."""
    from paper_2505_09324_gb300.quant import frame_bits
    p = random_gaussians(3000, 640, 360, seed=9)
    q = gs.Quantizer(refine=True)
    got = frame_bits(q, torch.from_numpy(p).cuda())
    oc, _, _ = Q.quantize(p, q.bits, refine=True)
    ref = B.code_entropy_bits(oc, q.bits).sum() + 64 * sum(b > 0 for b in q.bits)
    assert got == pytest.approx(ref, rel=1e-12)
