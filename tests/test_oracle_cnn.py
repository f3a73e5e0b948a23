"""Pins of the learned-initialiser oracle (no GPU)."""

import numpy as np

from oracle import cnn


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7, -2.5, 0.0,
                  3.0e38, 1.0 + 2.0 ** -8 + 2.0 ** -20], np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even keeps 1;
    # 1 + 3 * 2^-9 lies above the midpoint: rounds up to 1 + 2^-7
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -7, -2.5, 0.0, 3.0e38,
                     1.0 + 2.0 ** -7], np.float64)
    got = cnn.bf16_round(x).astype(np.float64)
    np.testing.assert_array_equal(got[:6], want[:6])
    assert got[7] == want[7]
    assert abs(got[6] - 3.0e38) / 3.0e38 < 2.0 ** -8
    # already representable values are fixed points; bits are the upper half
    y = cnn.bf16_round(np.random.Generator(np.random.PCG64(0)).normal(size=1000))
    np.testing.assert_array_equal(cnn.bf16_round(y), y)
    assert np.all((y.view(np.uint32) & 0xFFFF) == 0)
    np.testing.assert_array_equal(cnn.bf16_bits(y).astype(np.uint32) << 16, y.view(np.uint32))
    assert np.isnan(cnn.bf16_round(np.array([np.nan], np.float32)))[0]


def test_bf16_rounding_error_bound():
    x = np.random.Generator(np.random.PCG64(1)).uniform(-100, 100, 10000).astype(np.float32)
    r = cnn.bf16_round(x).astype(np.float64)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)


def test_gemm_against_brute_force_and_identity():
    g = np.random.Generator(np.random.PCG64(2))
    a, b = g.normal(size=(5, 7)), g.normal(size=(3, 7))
    bias = g.normal(size=3)
    c = cnn.gemm(a, b, bias, relu=True)
    for m in range(5):
        for n in range(3):
            s = bias[n]
            for k in range(7):
                s += a[m, k] * b[n, k]
            assert abs(c[m, n] - max(s, 0.0)) < 1e-12
    np.testing.assert_allclose(cnn.gemm(a, np.eye(7)), a)
    assert np.all(cnn.gemm_abs(a, b) >= np.abs(cnn.gemm(a, b)))


torch = None
try:
    import torch
except ImportError:  # pragma: no cover
    pass


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv_matches_torch_conv2d():
    import pytest
    if torch is None:
        pytest.skip("torch")
    g = _rng(3)
    B, H, W, C, co, ks, st, pad = 2, 9, 7, 8, 5, 3, 2, 1
    x = g.normal(size=(B, H, W, C))
    w = g.normal(size=(co, ks * ks * C + 1))
    got = cnn.conv(x, w, ks, st, pad)
    wt = torch.from_numpy(w[:, :ks * ks * C].reshape(co, ks, ks, C).transpose(0, 3, 1, 2).copy())
    ref = torch.nn.functional.conv2d(torch.from_numpy(x.transpose(0, 3, 1, 2).copy()), wt,
                                     torch.from_numpy(w[:, -1].copy()), stride=st, padding=pad)
    np.testing.assert_allclose(got, ref.numpy().transpose(0, 2, 3, 1), rtol=1e-12, atol=1e-12)


def test_conv_is_im2col_times_weights():
    g = _rng(4)
    x = g.normal(size=(1, 6, 5, 8))
    w = g.normal(size=(4, 73))
    col = cnn.im2col(x, 3, 2, 1, 80)
    wf = np.zeros((4, 80))
    wf[:, :73] = w
    np.testing.assert_allclose((col @ wf.T).reshape(1, 3, 3, 4), cnn.conv(x, w, 3, 2, 1),
                               rtol=1e-12, atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    g = _rng(5)
    for (H, W, ks, st, pad) in [(7, 6, 3, 2, 1), (4, 4, 1, 1, 0), (8, 5, 3, 1, 1)]:
        x = g.normal(size=(2, H, W, 8))
        ldk = -(-(ks * ks * 8 + 1) // 8) * 8
        col = cnn.im2col(x, ks, st, pad, ldk)
        y = g.normal(size=col.shape)
        y[:, ks * ks * 8:] = 0.0   # the bias and padding columns have no image adjoint
        lhs = float((col * y).sum())
        rhs = float((x * cnn.col2im(y, x.shape, ks, st, pad)).sum())
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_conv_backward_matches_torch_autograd():
    import pytest
    if torch is None:
        pytest.skip("torch")
    g = _rng(6)
    B, H, W, C, co = 2, 7, 6, 8, 3
    x = g.normal(size=(B, H, W, C))
    w = g.normal(size=(co, 73))
    dz = g.normal(size=(B, 4, 3, co))
    dw, dx = cnn.conv_backward(x, w, dz, 3, 2, 1, 80)
    xt = torch.from_numpy(x.transpose(0, 3, 1, 2).copy()).requires_grad_(True)
    wt = torch.from_numpy(w[:, :72].reshape(co, 3, 3, C).transpose(0, 3, 1, 2).copy())
    wt.requires_grad_(True)
    bt = torch.from_numpy(w[:, 72].copy()).requires_grad_(True)
    z = torch.nn.functional.conv2d(xt, wt, bt, stride=2, padding=1)
    z.backward(torch.from_numpy(dz.transpose(0, 3, 1, 2).copy()))
    np.testing.assert_allclose(dx, xt.grad.numpy().transpose(0, 2, 3, 1), rtol=1e-10, atol=1e-10)
    dwt = wt.grad.numpy().transpose(0, 2, 3, 1).reshape(co, 72)
    np.testing.assert_allclose(dw[:, :72], dwt, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(dw[:, 72], bt.grad.numpy(), rtol=1e-10, atol=1e-10)
    assert np.all(dw[:, 73:] == 0.0)


def test_head_select_ties_and_order():
    gh, gw, slots = 1, 2, 3
    out = np.zeros((2, 27), np.float32)
    # |0.25 + o8| per slot: cell 0: 0.75, 0.25, 0.75; cell 1: 0.0, 1.25, 0.75
    for cell, vals in enumerate([(0.5, 0.0, -1.0), (-0.25, 1.0, 0.5)]):
        for s, v in enumerate(vals):
            out[cell, 9 * s + 8] = v
    sel = cnn.head_select(out, gh, gw, slots, 3)
    # largest 1.25 (slot 4); then the three 0.75 ties at slots 0, 2, 5: lowest first
    assert sel.tolist() == [[0, 2, 4]]
    p, s2 = cnn.head_decode(out, gh, gw, slots, 32, 6.0, 3)
    assert s2.tolist() == sel.tolist()
    # tanh(0) = 0: the slot anchors; 3 slots on a 2 x 2 grid of quarter cells
    np.testing.assert_allclose(p[0, 0], [8.0, 8.0, 32 + 24.0])
    np.testing.assert_allclose(p[0, 1], [8.0, 24.0, 8.0])
    assert cnn.slot_anchor(9, 10) == (1.5 / 4, 2.5 / 3)
    np.testing.assert_allclose(p[0, 8], [0.75, -0.75, 1.25])
    np.testing.assert_allclose(p[0, 2], [6.0, 6.0, 6.0])        # exp(0) * scale


def test_head_decode_backward_matches_finite_differences():
    g = _rng(7)
    gh, gw, slots, n = 2, 3, 4, 10
    out = g.normal(size=(2 * gh * gw, 40)) * 0.7
    out[3, 9 * 1 + 2] = 3.5   # a clamped exponent: zero derivative
    params, sel = cnn.head_decode(out, gh, gw, slots, 16, 5.0, n)
    dp = g.normal(size=params.shape)
    d = cnn.head_decode_bwd(out, sel, dp, gh, gw, slots, 16, 5.0)
    for (r, c) in [(0, 0), (1, 10), (2, 20), (3, 11), (4, 13), (5, 18), (3, 9 + 2), (7, 26)]:
        h = 1e-6
        a, b = out.copy(), out.copy()
        a[r, c] += h
        b[r, c] -= h
        pa, sa = cnn.head_decode(a, gh, gw, slots, 16, 5.0, n)
        pb, sb = cnn.head_decode(b, gh, gw, slots, 16, 5.0, n)
        assert (sa == sel).all() and (sb == sel).all()
        fd = float(((pa - pb) * dp).sum() / (2 * h))
        assert abs(fd - d[r, c]) <= 1e-6 * max(1.0, abs(fd)), (r, c, fd, d[r, c])


def test_chamfer_pins():
    g = _rng(8)
    p = g.uniform(0, 50, (40, 2))
    loss, grad = cnn.chamfer(p, p[::-1].copy())
    assert loss == 0.0 and np.all(grad == 0.0)
    # one point each: |p - q|^2 twice
    loss, grad = cnn.chamfer(np.array([[1.0, 2.0]]), np.array([[4.0, 6.0]]))
    assert loss == 50.0
    np.testing.assert_allclose(grad, [[-12.0, -16.0]])
    # gradient by central differences (assignment unchanged for small steps)
    q = g.uniform(0, 50, (30, 2))
    loss, grad = cnn.chamfer(p, q)
    for i in (0, 7, 33):
        for c in (0, 1):
            a, b = p.copy(), p.copy()
            a[i, c] += 1e-6
            b[i, c] -= 1e-6
            fd = (cnn.chamfer(a, q)[0] - cnn.chamfer(b, q)[0]) / 2e-6
            assert abs(fd - grad[i, c]) < 1e-6 * max(1.0, abs(fd))
