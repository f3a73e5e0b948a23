"""BF16 tensor-core GEMM (tcgen05) and the learned initialiser's kernels
against the double-precision oracle.

BF16 inputs are exact in both computations (products of BF16 values are exact
in FP32); the GPU accumulates in FP32, so each output may differ from the
double-precision sum by FP32 rounding of partial sums: the bar is 2e-5 of
sum_k |a_k b_k| (about 170 FP32 ulps of that scale)."""

import numpy as np
import pytest

from oracle import cnn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module")
def nat():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    return _native


def bf16_dev(x):
    bits = cnn.bf16_bits(x)
    return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()


def run_gemm(nat, a, b, bias=None, relu=False, splits=1, out="f32", lda=None, ldc=None):
    M, K = a.shape
    N = b.shape[0]
    lda = lda or -(-K // 8) * 8
    ldb = -(-K // 8) * 8
    A = np.zeros((M, lda), np.float32)
    A[:, :K] = a
    B = np.zeros((N, ldb), np.float32)
    B[:, :K] = b
    ldc = ldc or N
    dA, dB = bf16_dev(A), bf16_dev(B)
    dbias = torch.from_numpy(np.asarray(bias, np.float32)).cuda() if bias is not None else None
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    pb = nat.load().gs2d_gemm_partial_bytes(M, N, ldc, K, splits)
    part = torch.empty(max(pb // 4, 1), device="cuda")
    if out == "f32":
        C = torch.full((M, ldc), float("nan"), device="cuda")
        nat.gemm_bf16(dA.data_ptr(), lda, dB.data_ptr(), ldb, M, N, K,
                      dbias.data_ptr() if dbias is not None else 0, relu, C.data_ptr(), 0, ldc,
                      splits, part.data_ptr(), status.data_ptr(), 0)
        res = C.cpu().numpy()[:, :N].astype(np.float64)
    else:
        C = torch.zeros((M, ldc), dtype=torch.bfloat16, device="cuda")
        nat.gemm_bf16(dA.data_ptr(), lda, dB.data_ptr(), ldb, M, N, K,
                      dbias.data_ptr() if dbias is not None else 0, relu, 0, C.data_ptr(), ldc,
                      splits, part.data_ptr(), status.data_ptr(), 0)
        res = C.float().cpu().numpy()[:, :N].astype(np.float64)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return res


@pytest.mark.parametrize("M,N,K,splits", [
    (128, 32, 64, 1), (200, 64, 136, 1), (300, 384, 576, 1), (1000, 96, 2304, 4),
    (77, 256, 1152, 3), (4096, 192, 320, 1), (64, 16, 8, 1), (130, 300, 64, 1)])
def test_gemm_f32_matches_oracle(nat, M, N, K, splits):
    g = np.random.Generator(np.random.PCG64(M * 7 + N + K))
    a = cnn.bf16_round(g.normal(size=(M, K)))
    b = cnn.bf16_round(g.normal(size=(N, K)))
    got = run_gemm(nat, a, b, splits=splits)
    ref = cnn.gemm(a, b)
    bound = REL * cnn.gemm_abs(a, b) + 1e-30
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


@pytest.mark.parametrize("splits", [1, 5])
def test_gemm_bias_relu_bf16_output(nat, splits):
    M, N, K = 256, 128, 320
    g = np.random.Generator(np.random.PCG64(9))
    a = cnn.bf16_round(g.normal(size=(M, K)))
    b = cnn.bf16_round(g.normal(size=(N, K)) * 0.1)
    bias = g.normal(size=N).astype(np.float32)
    got = run_gemm(nat, a, b, bias=bias, relu=True, splits=splits, out="bf16", ldc=136)
    ref = cnn.gemm(a, b, bias, relu=True)
    # the BF16 store rounds once more: half a BF16 ulp of the value
    bound = REL * (cnn.gemm_abs(a, b) + np.abs(bias)[None, :]) + np.abs(ref) * 2.0 ** -8
    assert np.all(np.abs(got - ref) <= bound + 1e-30)
    assert np.all(got >= 0.0)


def test_gemm_padded_leading_dimension(nat):
    M, N, K = 150, 40, 100
    g = np.random.Generator(np.random.PCG64(4))
    a = cnn.bf16_round(g.normal(size=(M, K)))
    b = cnn.bf16_round(g.normal(size=(N, K)))
    got = run_gemm(nat, a, b, lda=104, ldc=48)
    ref = cnn.gemm(a, b)
    assert np.all(np.abs(got - ref) <= REL * cnn.gemm_abs(a, b) + 1e-30)


# ---------------------------------------------------------------------------
# convolution helpers and the head

def to_np_bf16(t):
    return t.float().cpu().numpy().astype(np.float64)


def dev_f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def bf16_ulp_close(got, ref, ulps=1):
    """|got - bf16_round(ref)| within `ulps` BF16 units of the value (rounding
    of an FP32 result that differs from the double-precision one in the last
    FP32 bits may land on the neighbouring BF16 value)."""
    r = cnn.bf16_round(ref).astype(np.float64)
    tol = ulps * np.maximum(np.abs(r), 1e-30) * 2.0 ** -7
    return np.all(np.abs(got - r) <= tol)


def test_cnn_input_layout(nat):
    from gs2d_inputs import conferencing_frame
    f, m = conferencing_frame(37, 21, seed=1)
    x = torch.empty((2, 21, 37, 8), dtype=torch.bfloat16, device="cuda")
    frames = dev_f32(np.stack([f, f[:, ::-1].copy()]))
    masks = torch.from_numpy(np.stack([m, ~m]).astype(np.uint8)).cuda()
    nat.call("gs2d_cnn_input", frames.data_ptr(), masks.data_ptr(), 2, 21, 37, x.data_ptr(), 0)
    got = to_np_bf16(x)
    want = np.zeros((2, 21, 37, 8))
    want[0, ..., :3] = f.transpose(1, 2, 0)
    want[1, ..., :3] = f[:, ::-1].transpose(1, 2, 0)
    want[0, ..., 3] = m
    want[1, ..., 3] = ~m
    np.testing.assert_array_equal(got, cnn.bf16_round(want).astype(np.float64))


@pytest.mark.parametrize("B,H,W,C,ks,st,pad", [(2, 9, 7, 8, 3, 2, 1), (1, 33, 20, 32, 3, 2, 1),
                                                (3, 5, 6, 16, 1, 1, 0), (1, 8, 8, 8, 3, 1, 1)])
def test_im2col_and_col2im(nat, B, H, W, C, ks, st, pad):
    g = np.random.Generator(np.random.PCG64(H * W + C))
    x = cnn.bf16_round(g.normal(size=(B, H, W, C)))
    ldk = -(-(ks * ks * C + 1) // 8) * 8
    Ho, Wo = cnn.out_size(H, ks, st, pad), cnn.out_size(W, ks, st, pad)
    dx = bf16_dev(x)
    col = torch.full((B * Ho * Wo, ldk), 7.0, dtype=torch.bfloat16, device="cuda")
    nat.call("gs2d_im2col", dx.data_ptr(), B, H, W, C, ks, st, pad, col.data_ptr(), ldk, 0)
    np.testing.assert_array_equal(to_np_bf16(col), cnn.im2col(x, ks, st, pad, ldk))
    # gradient, with and without the ReLU mask
    dcol = g.normal(size=(B * Ho * Wo, ldk)).astype(np.float32)
    act = cnn.bf16_round(g.normal(size=x.shape))
    ref = cnn.col2im(dcol, x.shape, ks, st, pad)
    d_dcol, d_act = dev_f32(dcol), bf16_dev(act)  # held: the calls below are asynchronous
    for use_act in (False, True):
        out = torch.empty(x.shape, dtype=torch.bfloat16, device="cuda")
        nat.call("gs2d_col2im", d_dcol.data_ptr(), ldk, B, H, W, C, ks, st, pad,
                 d_act.data_ptr() if use_act else 0, out.data_ptr(), 0)
        want = ref * (act > 0) if use_act else ref
        assert bf16_ulp_close(to_np_bf16(out), want)


def test_transpose_relu_bwd_cast(nat):
    g = np.random.Generator(np.random.PCG64(5))
    a = cnn.bf16_round(g.normal(size=(70, 45)))
    out = torch.zeros((45, 72), dtype=torch.bfloat16, device="cuda")
    d_a = bf16_dev(a)  # device buffers stay referenced until the calls have run
    nat.call("gs2d_transpose_bf16", d_a.data_ptr(), 70, 45, 45, out.data_ptr(), 72, 0)
    np.testing.assert_array_equal(to_np_bf16(out)[:, :70], a.T)
    dx = g.normal(size=(70, 45)).astype(np.float32)
    dz = torch.zeros((70, 48), dtype=torch.bfloat16, device="cuda")
    d_dx = dev_f32(dx)
    nat.call("gs2d_relu_bwd", d_dx.data_ptr(), 70, 45, 45, d_a.data_ptr(), 45, dz.data_ptr(), 48,
             0)
    np.testing.assert_array_equal(to_np_bf16(dz)[:, :45], cnn.bf16_round(dx * (a > 0)))
    w = g.normal(size=(24, 80)).astype(np.float32)
    wb = torch.empty((24, 80), dtype=torch.bfloat16, device="cuda")
    wt = torch.empty((80, 24), dtype=torch.bfloat16, device="cuda")
    d_w = dev_f32(w)
    nat.call("gs2d_cast_weights", d_w.data_ptr(), 24, 80, wb.data_ptr(), wt.data_ptr(), 0)
    np.testing.assert_array_equal(to_np_bf16(wb), cnn.bf16_round(w))
    np.testing.assert_array_equal(to_np_bf16(wt), cnn.bf16_round(w).T)


@pytest.mark.parametrize("B,H,W,ci,co", [(2, 40, 33, 8, 32), (1, 24, 30, 32, 64),
                                         (2, 12, 9, 256, 384)])
def test_conv_layer_via_im2col_gemm(nat, B, H, W, ci, co):
    """A stride-2 3 x 3 convolution with bias and ReLU as im2col + tensor-core
    GEMM (BF16 out) against the direct convolution of the oracle."""
    g = np.random.Generator(np.random.PCG64(co + H))
    ks, st, pad = 3, 2, 1
    ldk = -(-(ks * ks * ci + 1) // 8) * 8
    x = cnn.bf16_round(g.normal(size=(B, H, W, ci)))
    w = np.zeros((co, ldk), np.float32)
    w[:, :ks * ks * ci + 1] = g.normal(size=(co, ks * ks * ci + 1)) / np.sqrt(9 * ci)
    w = cnn.bf16_round(w)
    Ho, Wo = cnn.out_size(H, ks, st, pad), cnn.out_size(W, ks, st, pad)
    P = B * Ho * Wo
    col = torch.empty((P, ldk), dtype=torch.bfloat16, device="cuda")
    d_x, d_w = bf16_dev(x), bf16_dev(w)
    nat.call("gs2d_im2col", d_x.data_ptr(), B, H, W, ci, ks, st, pad, col.data_ptr(), ldk, 0)
    z = torch.empty((P, co), dtype=torch.bfloat16, device="cuda")
    st_ = torch.zeros(1, dtype=torch.int32, device="cuda")
    nat.gemm_bf16(col.data_ptr(), ldk, d_w.data_ptr(), ldk, P, co, ldk, 0, True, 0,
                  z.data_ptr(), co, 1, 0, st_.data_ptr(), 0)
    torch.cuda.synchronize()
    ref = np.maximum(cnn.conv(x, w[:, :ks * ks * ci + 1], ks, st, pad), 0.0).reshape(P, co)
    scale = cnn.gemm_abs(cnn.im2col(x, ks, st, pad, ldk), w)
    got = to_np_bf16(z)
    assert np.all(np.abs(got - ref) <= REL * scale + np.abs(ref) * 2.0 ** -8 + 1e-30)


def test_head_decode_select_and_backward(nat):
    g = np.random.Generator(np.random.PCG64(11))
    B, gh, gw, slots, ldo, n, cell, scale = 2, 5, 7, 10, 96, 300, 32, 6.0
    out = (g.normal(size=(B * gh * gw, ldo)) * 0.8).astype(np.float32)
    out[0, 9 * 3 + 8] = out[0, 9 * 4 + 8]          # a tie in |w|
    out[5, 2] = 5.0                                 # clamped exponent
    d_out = dev_f32(out)
    ldp = B * n + 8
    params = torch.empty((9, ldp), device="cuda")
    sel = torch.empty((B, n), dtype=torch.int32, device="cuda")
    nat.call("gs2d_head_decode", d_out.data_ptr(), ldo, B, gh, gw, slots, cell, scale, n,
             params.data_ptr(), ldp, sel.data_ptr(), 0)
    ref_p, ref_sel = cnn.head_decode(out, gh, gw, slots, cell, scale, n)
    np.testing.assert_array_equal(sel.cpu().numpy(), ref_sel)
    got = params.cpu().numpy()[:, :B * n].reshape(9, B, n).transpose(1, 0, 2).astype(np.float64)
    assert np.all(np.abs(got - ref_p) <= 1e-6 * np.abs(ref_p) + 1e-5)
    dp = g.normal(size=(B, 9, n)).astype(np.float32)
    dout = torch.full((B * gh * gw, ldo), 3.0, dtype=torch.bfloat16, device="cuda")
    flat = np.zeros((9, ldp), np.float32)
    flat[:, :B * n] = dp.transpose(1, 0, 2).reshape(9, B * n)
    d_dp = dev_f32(flat)
    nat.call("gs2d_head_decode_bwd", d_out.data_ptr(), ldo, B, gh, gw, slots, cell, scale, n,
             sel.data_ptr(), d_dp.data_ptr(), ldp, dout.data_ptr(), 0)
    ref_d = cnn.head_decode_bwd(out, ref_sel, dp, gh, gw, slots, cell, scale)
    assert bf16_ulp_close(to_np_bf16(dout), ref_d, ulps=2)


def test_chamfer_loss_and_gradient(nat):
    g = np.random.Generator(np.random.PCG64(12))
    B, n, m = 2, 700, 500
    P = np.zeros((9, B * n), np.float32)
    Q = np.zeros((9, B * m), np.float32)
    P[:2] = g.uniform(0, 300, (2, B * n))
    Q[:2] = g.uniform(0, 300, (2, B * m))
    scratch = torch.empty(nat.load().gs2d_chamfer_scratch_bytes(n, m, B), dtype=torch.uint8,
                          device="cuda")
    loss = torch.empty(B, device="cuda")
    dP = torch.zeros((9, B * n), device="cuda")
    lam = 0.5
    d_P, d_Q = dev_f32(P), dev_f32(Q)
    nat.call("gs2d_chamfer", d_P.data_ptr(), n, B * n, d_Q.data_ptr(), m, B * m, B, lam,
             dP.data_ptr(), loss.data_ptr(), scratch.data_ptr(), 0)
    for b in range(B):
        ref_l, ref_g = cnn.chamfer(P[:2, b * n:(b + 1) * n].T, Q[:2, b * m:(b + 1) * m].T)
        assert abs(float(loss[b]) - ref_l) <= 1e-5 * ref_l
        got = dP[:2, b * n:(b + 1) * n].cpu().numpy().T.astype(np.float64)
        assert np.all(np.abs(got - lam * ref_g) <= 1e-4 * np.abs(lam * ref_g).max())
    assert float(dP[2:].abs().max()) == 0.0


@pytest.mark.parametrize("B,H,W,ci,co,ks,st,pad,out", [
    (2, 40, 33, 8, 32, 3, 2, 1, "bf16"),     # ragged M (2 x 20 x 17 = 680 rows)
    (1, 24, 30, 32, 64, 3, 2, 1, "bf16"),
    (2, 12, 9, 256, 384, 3, 2, 1, "bf16"),   # N over two 192-column tiles, 37 k-tiles
    (3, 7, 11, 384, 90, 1, 1, 0, "f32"),     # the head: 1 x 1, N = 90, FP32 out
    # output rows of 64 pixels or more and C of 16, 32 or 64 j: the
    # persistent kernel with TMA tap loads (128-pixel row segments, the last
    # one ragged); C = 8 stays with the gathering kernel
    (1, 135, 240, 64, 128, 3, 2, 1, "bf16"),  # 128-byte blocks, weights streamed
    (2, 40, 300, 8, 32, 3, 2, 1, "bf16"),     # C = 8, wide rows: the gathering kernel
    (1, 30, 260, 16, 48, 3, 2, 1, "bf16"),    # 32-byte swizzle, N below the tile
    (2, 24, 200, 32, 64, 3, 2, 1, "bf16"),    # 64-byte swizzle, weights resident
    (1, 17, 150, 128, 256, 3, 2, 1, "bf16"),  # two chunks per tap, N = 256
    # more tiles than CTAs with streamed weights: two tiles per weight box
    # in some CTAs, one in the others
    (2, 160, 256, 64, 128, 3, 2, 1, "bf16"),
    (2, 200, 130, 128, 256, 3, 2, 1, "bf16"),
    (1, 9, 70, 64, 90, 1, 1, 0, "f32"),       # stride 1, a k-tile of bias and zeros only
    (1, 8, 140, 8, 32, 3, 1, 1, "bf16"),      # stride 1, C = 8
    (1, 9, 600, 32, 64, 3, 2, 1, "bf16"),     # three row segments, the last ragged
    (2, 11, 400, 64, 32, 3, 2, 1, "f32"),     # C = 64 with resident weights, odd height
    (1, 10, 300, 32, 160, 3, 2, 1, "bf16"),   # C = 32, weights streamed: k-tiles across input rows
    (1, 12, 260, 128, 96, 3, 2, 1, "f32"),    # C = 128, N = 96
    (1, 21, 259, 32, 64, 3, 2, 1, "bf16"),    # odd width
    (2, 19, 261, 64, 128, 3, 2, 1, "bf16"),   # odd width, weights streamed
    (1, 12, 200, 16, 32, 5, 2, 4, "bf16"),    # 5 x 5, pad 4: taps start 4 pixels left of the image
    (1, 20, 258, 32, 32, 3, 2, 0, "f32")])    # no padding
def test_implicit_conv_equals_im2col_gemm(nat, B, H, W, ci, co, ks, st, pad, out):
    """gs2d_conv_bf16 gathers the im2col tiles itself: its output equals
    gs2d_im2col + gs2d_gemm_bf16 bit for bit, and the oracle's convolution
    within the GEMM bar."""
    g = np.random.Generator(np.random.PCG64(7 * co + H + ks))
    ldk = -(-(ks * ks * ci + 1) // 8) * 8
    x = cnn.bf16_round(g.normal(size=(B, H, W, ci)))
    w = np.zeros((co, ldk), np.float32)
    w[:, :ks * ks * ci + 1] = g.normal(size=(co, ks * ks * ci + 1)) / np.sqrt(ks * ks * ci)
    w = cnn.bf16_round(w)
    Ho, Wo = cnn.out_size(H, ks, st, pad), cnn.out_size(W, ks, st, pad)
    P = B * Ho * Wo
    d_x, d_w = bf16_dev(x), bf16_dev(w)
    relu = out == "bf16"
    dt = torch.bfloat16 if out == "bf16" else torch.float32
    col = torch.empty((P, ldk), dtype=torch.bfloat16, device="cuda")
    z_ref = torch.empty((P, co), dtype=dt, device="cuda")
    z = torch.full((P, co), 7.0, dtype=dt, device="cuda")
    st_ = torch.zeros(1, dtype=torch.int32, device="cuda")
    nat.call("gs2d_im2col", d_x.data_ptr(), B, H, W, ci, ks, st, pad, col.data_ptr(), ldk, 0)
    f32 = z_ref.data_ptr() if out == "f32" else 0
    b16 = z_ref.data_ptr() if out == "bf16" else 0
    nat.gemm_bf16(col.data_ptr(), ldk, d_w.data_ptr(), ldk, P, co, ldk, 0, relu, f32, b16, co, 1,
                  0, st_.data_ptr(), 0)
    nat.call("gs2d_conv_bf16", d_x.data_ptr(), B, H, W, ci, ks, st, pad, d_w.data_ptr(), ldk,
             co, 1 if relu else 0, z.data_ptr() if out == "f32" else 0,
             z.data_ptr() if out == "bf16" else 0, co, st_.data_ptr(), 0)
    torch.cuda.synchronize()
    assert int(st_.item()) == 0
    assert torch.equal(z, z_ref)
    ref = cnn.conv(x, w[:, :ks * ks * ci + 1], ks, st, pad).reshape(P, co)
    if relu:
        ref = np.maximum(ref, 0.0)
    scale = cnn.gemm_abs(cnn.im2col(x, ks, st, pad, ldk), w)
    got = (to_np_bf16(z) if out == "bf16" else z.cpu().numpy()).astype(np.float64)
    tol = REL * scale + (np.abs(ref) * 2.0 ** -8 if relu else 0.0) + 1e-30
    assert np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("B,H,W,ks,st,pad,co,with_mask,out", [
    (2, 37, 304, 3, 2, 1, 32, True, "bf16"),    # two row segments, the last ragged
    (1, 20, 160, 3, 1, 1, 64, False, "bf16"),   # stride 1, no mask (channel 3 zero)
    (3, 9, 272, 1, 1, 0, 90, True, "f32"),      # 1 x 1: one k-tile, N = 90, FP32 out
    (1, 1080, 1920, 3, 2, 1, 32, True, "bf16")])  # the network's first layer at 1080p
def test_conv_frame_equals_input_then_conv(nat, B, H, W, ks, st, pad, co, with_mask, out):
    """gs2d_conv_frame_bf16 forms the 8-channel input of each im2col row from
    the float frame and the mask itself: its output equals gs2d_cnn_input +
    gs2d_conv_bf16 bit for bit."""
    _frame_vs_parts(nat, B, H, W, ks, st, pad, co, with_mask, out)


@pytest.mark.parametrize("ks,st", [(3, 2), (3, 1)])
def test_conv_frame_three_k_tiles(nat, ks, st):
    """A padded weight row (ldk 136: three k-tiles, zero slices past the bias)
    in both operand layouts."""
    _frame_vs_parts(nat, 1, 23, 272, ks, st, 1, 32, True, "bf16", ldk_extra=56)


def _frame_vs_parts(nat, B, H, W, ks, st, pad, co, with_mask, out, ldk_extra=0):
    g = np.random.Generator(np.random.PCG64(11 * co + H + ks))
    frames = torch.from_numpy(g.normal(0.5, 0.4, size=(B, 3, H, W)).astype(np.float32)).cuda()
    masks = None
    if with_mask:
        masks = torch.from_numpy(g.choice(np.array([0, 1, 7], np.uint8), size=(B, H, W))).cuda()
    ldk = -(-(ks * ks * 8 + 1) // 8) * 8 + ldk_extra
    w = np.zeros((co, ldk), np.float32)
    w[:, :ks * ks * 8 + 1] = g.normal(size=(co, ks * ks * 8 + 1)) / np.sqrt(ks * ks * 8)
    d_w = bf16_dev(cnn.bf16_round(w))
    Ho, Wo = cnn.out_size(H, ks, st, pad), cnn.out_size(W, ks, st, pad)
    P = B * Ho * Wo
    dt = torch.bfloat16 if out == "bf16" else torch.float32
    relu = 1 if out == "bf16" else 0
    x = torch.empty((B, H, W, 8), dtype=torch.bfloat16, device="cuda")
    z_ref = torch.empty((P, co), dtype=dt, device="cuda")
    z = torch.full((P, co), 7.0, dtype=dt, device="cuda")
    st_ = torch.zeros(1, dtype=torch.int32, device="cuda")
    mptr = masks.data_ptr() if masks is not None else 0

    def outs(t):
        return (t.data_ptr() if out == "f32" else 0, t.data_ptr() if out == "bf16" else 0)

    nat.call("gs2d_cnn_input", frames.data_ptr(), mptr, B, H, W, x.data_ptr(), 0)
    nat.call("gs2d_conv_bf16", x.data_ptr(), B, H, W, 8, ks, st, pad, d_w.data_ptr(), ldk, co,
             relu, *outs(z_ref), co, st_.data_ptr(), 0)
    nat.call("gs2d_conv_frame_bf16", frames.data_ptr(), mptr, B, H, W, ks, st, pad,
             d_w.data_ptr(), ldk, co, relu, *outs(z), co, st_.data_ptr(), 0)
    torch.cuda.synchronize()
    assert int(st_.item()) == 0
    assert torch.equal(z, z_ref)


def test_conv_frame_bad_arguments(nat):
    d = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    w = torch.zeros(32 * 80, dtype=torch.bfloat16, device="cuda")
    o = torch.zeros(1 << 16, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(nat.Gs2dError):   # W not a multiple of 16
        nat.call("gs2d_conv_frame_bf16", d.data_ptr(), 0, 1, 8, 40, 3, 2, 1, w.data_ptr(), 80,
                 32, 1, 0, o.data_ptr(), 32, 0, 0)
    with pytest.raises(nat.Gs2dError):   # N above 128
        nat.call("gs2d_conv_frame_bf16", d.data_ptr(), 0, 1, 8, 32, 3, 2, 1, w.data_ptr(), 80,
                 160, 1, 0, o.data_ptr(), 160, 0, 0)
    with pytest.raises(nat.Gs2dError):   # no room for the bias column
        nat.call("gs2d_conv_frame_bf16", d.data_ptr(), 0, 1, 8, 32, 3, 2, 1, w.data_ptr(), 72,
                 32, 1, 0, o.data_ptr(), 32, 0, 0)


@pytest.mark.parametrize("H,W,ci,co", [(540, 960, 32, 64), (270, 480, 64, 128),
                                        (135, 240, 128, 256)])
def test_tap_conv_network_layers_full_size(nat, H, W, ci, co):
    """Layers 2-4 of the learned initialiser at 1080p (two frames), in the
    launch configuration the forward uses: the TMA-tap kernel equals
    im2col + GEMM bit for bit everywhere, and 256 sampled outputs equal the
    oracle's convolution of their receptive fields within the GEMM bar."""
    B, ks, st, pad = 2, 3, 2, 1
    g = np.random.Generator(np.random.PCG64(5 * co + H))
    ldk = -(-(ks * ks * ci + 1) // 8) * 8
    x = cnn.bf16_round(g.normal(size=(B, H, W, ci)).astype(np.float32))
    w = np.zeros((co, ldk), np.float32)
    w[:, :ks * ks * ci + 1] = g.normal(size=(co, ks * ks * ci + 1)) / np.sqrt(ks * ks * ci)
    w = cnn.bf16_round(w)
    Ho, Wo = cnn.out_size(H, ks, st, pad), cnn.out_size(W, ks, st, pad)
    P = B * Ho * Wo
    d_x, d_w = bf16_dev(x), bf16_dev(w)
    z = torch.empty((P, co), dtype=torch.bfloat16, device="cuda")
    z_ref = torch.empty_like(z)
    col = torch.empty((P, ldk), dtype=torch.bfloat16, device="cuda")
    st_ = torch.zeros(1, dtype=torch.int32, device="cuda")
    nat.call("gs2d_conv_bf16", d_x.data_ptr(), B, H, W, ci, ks, st, pad, d_w.data_ptr(), ldk, co,
             0, 0, z.data_ptr(), co, st_.data_ptr(), 0)
    nat.call("gs2d_im2col", d_x.data_ptr(), B, H, W, ci, ks, st, pad, col.data_ptr(), ldk, 0)
    nat.gemm_bf16(col.data_ptr(), ldk, d_w.data_ptr(), ldk, P, co, ldk, 0, False, 0,
                  z_ref.data_ptr(), co, 1, 0, st_.data_ptr(), 0)
    torch.cuda.synchronize()
    assert int(st_.item()) == 0
    assert torch.equal(z, z_ref)
    got = to_np_bf16(z).reshape(B, Ho, Wo, co)
    for _ in range(256):
        b, oy, ox = int(g.integers(B)), int(g.integers(Ho)), int(g.integers(Wo))
        patch = np.zeros((1, ks, ks, ci), np.float32)   # the receptive field, zero outside
        for ky in range(ks):
            for kx in range(ks):
                iy, ix = oy * st - pad + ky, ox * st - pad + kx
                if 0 <= iy < H and 0 <= ix < W:
                    patch[0, ky, kx] = x[b, iy, ix]
        ref = cnn.conv(patch, w[:, :ks * ks * ci + 1], ks, 1, 0)[0, 0, 0]
        scale = cnn.gemm_abs(cnn.im2col(patch, ks, 1, 0, ldk), w)[0]
        # one BF16 rounding of the FP32 sum on top of the GEMM bar
        tol = REL * scale + np.abs(ref) * 2.0 ** -8 + 1e-30
        assert np.all(np.abs(got[b, oy, ox] - ref) <= tol), (b, oy, ox)


def test_implicit_conv_bad_arguments(nat):
    d = torch.zeros(64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(nat.Gs2dError):   # C not a multiple of 8
        nat.call("gs2d_conv_bf16", d.data_ptr(), 1, 4, 4, 4, 3, 2, 1, d.data_ptr(), 40, 8, 1, 0,
                 d.data_ptr(), 8, 0, 0)
    with pytest.raises(nat.Gs2dError):   # no room for the bias column
        nat.call("gs2d_conv_bf16", d.data_ptr(), 1, 4, 4, 8, 3, 2, 1, d.data_ptr(), 72, 8, 1, 0,
                 d.data_ptr(), 8, 0, 0)
