"""8-bit RGB frame input: the device conversion to the planar float frame is
c / 255 correctly rounded, bit for bit, for packed and padded rows, odd sizes
and the empty frame; and a fit on the converted frame equals a fit on the
same frame converted on the host."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2505_09324_gb300 import _native, build
    build.build()
    _native.load()
    import paper_2505_09324_gb300 as pkg
    return pkg


@pytest.mark.parametrize("W,H", [(1, 1), (37, 5), (641, 359), (1000, 7), (1920, 1080)])
def test_rgb8_to_planar_bit_exact(gs, W, H):
    rng = np.random.default_rng(W * 7 + H)
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    got = gs.frame_from_rgb8(torch.from_numpy(rgb).cuda()).cpu().numpy()
    want = rgb.transpose(2, 0, 1).astype(np.float32) / np.float32(255.0)
    np.testing.assert_array_equal(got, want)
    assert got[0, 0, 0] == np.float32(rgb[0, 0, 0]) / np.float32(255)


@pytest.mark.parametrize("pad", [61, 64])   # odd rows: byte loads; 4-byte rows: word loads
def test_rgb8_padded_rows(gs, pad):
    from paper_2505_09324_gb300 import _native as nat
    W, H = 100, 33
    rng = np.random.default_rng(3)
    buf = rng.integers(0, 256, (H, 3 * W + pad), dtype=np.uint8)
    d = torch.from_numpy(buf).cuda()
    out = torch.full((3, H, W), -1.0, device="cuda")
    nat.frame_from_rgb8(d.data_ptr(), W, H, 3 * W + pad, out.data_ptr(),
                        int(torch.cuda.current_stream().cuda_stream))
    want = buf[:, :3 * W].reshape(H, W, 3).transpose(2, 0, 1).astype(np.float32) / np.float32(255)
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_rgb8_empty_and_bad_arguments(gs):
    from paper_2505_09324_gb300 import _native as nat
    s = int(torch.cuda.current_stream().cuda_stream)
    nat.frame_from_rgb8(0, 0, 0, 0, 0, s)                      # empty frame: no-op
    with pytest.raises(nat.Gs2dError):
        nat.frame_from_rgb8(0, 4, 4, 12, 0, s)                 # null buffers
    d = torch.zeros((4, 4, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty((3, 4, 4), device="cuda")
    with pytest.raises(nat.Gs2dError):
        nat.frame_from_rgb8(d.data_ptr(), 4, 4, 11, out.data_ptr(), s)  # row too short
    with pytest.raises(nat.Gs2dError):                         # taller than 65535 rows
        nat.frame_from_rgb8(d.data_ptr(), 1, 65536, 3, out.data_ptr(), s)


def test_fit_on_converted_frame(gs):
    from gs2d_inputs import random_gaussians
    W, H, n = 128, 96, 300
    rng = np.random.default_rng(5)
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    dev_frame = gs.frame_from_rgb8(torch.from_numpy(rgb).cuda())
    host_frame = torch.from_numpy(rgb.transpose(2, 0, 1).astype(np.float32)
                                  / np.float32(255)).contiguous().cuda()
    p0 = torch.from_numpy(random_gaussians(n, W, H, seed=6)).cuda()
    a, b = p0.clone(), p0.clone()
    r = gs.GaussianRasterizer(W, H, n)
    r.encode_frame(dev_frame, a, 20, check_every=20)
    r.encode_frame(host_frame, b, 20, check_every=20)
    assert torch.equal(a, b)


@pytest.mark.parametrize("pinned", [True, False])
def test_fit_step_rgb8_is_upload_convert_fit_download(gs, pinned):
    """The one-call end-to-end iteration from host buffers equals its parts:
    with a pinned frame the conversion reads it over the host link itself and
    the Adam kernel stores the Gaussians into the pinned output; with
    pageable buffers they go through the device staging buffer and a copy."""
    from gs2d_inputs import random_gaussians
    from paper_2505_09324_gb300 import _native as nat
    W, H, n = 160, 96, 400
    rng = np.random.default_rng(8)
    rgb = torch.from_numpy(rng.integers(0, 256, (H, W, 3), dtype=np.uint8))
    if pinned:
        rgb = rgb.pin_memory()
    p0 = torch.from_numpy(random_gaussians(n, W, H, seed=9)).pin_memory()
    out = torch.empty_like(p0)  # pinned: the Adam kernel stores it; else a copy
    if pinned:
        out = out.pin_memory()
    r = gs.GaussianRasterizer(W, H, n)
    s = int(torch.cuda.current_stream().cuda_stream)
    d_rgb = torch.empty((H, W, 3), dtype=torch.uint8, device="cuda")
    d_frame = torch.empty((3, H, W), device="cuda")
    d_p = torch.empty((9, n), device="cuda")
    m, v = torch.empty_like(d_p), torch.empty_like(d_p)
    nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
    for _ in range(2):
        nat.fit_step_rgb8(r.plan, r.ws_ptr, rgb.data_ptr(), d_rgb.data_ptr(), d_frame.data_ptr(),
                          p0.data_ptr(), d_p.data_ptr(), m.data_ptr(), v.data_ptr(),
                          out.data_ptr(), s)
    torch.cuda.synchronize()
    # the same by parts
    frame = gs.frame_from_rgb8(rgb.cuda())
    q = p0.cuda()
    m2, v2 = torch.empty_like(q), torch.empty_like(q)
    nat.fit_reset(r.plan, r.ws_ptr, m2.data_ptr(), v2.data_ptr(), s)
    for _ in range(2):
        q.copy_(p0)
        nat.fit_step(r.plan, r.ws_ptr, frame.data_ptr(), q.data_ptr(), m2.data_ptr(),
                     v2.data_ptr(), s)
    torch.cuda.synchronize()
    assert torch.equal(out, q.cpu()) and torch.equal(d_p, q)
    assert torch.equal(d_frame, frame)


def test_fit_step_rgb8_on_a_stream_reads_current_host_buffers(gs):
    """Repeated calls on a non-default stream: each must read the host
    buffers' current contents (a new frame and the previous step's Gaussians
    every call), also after a buffer changes."""
    from gs2d_inputs import random_gaussians
    from paper_2505_09324_gb300 import _native as nat
    W, H, n, steps = 144, 80, 300, 5
    rng = np.random.default_rng(10)
    frames = [rng.integers(0, 256, (H, W, 3), dtype=np.uint8) for _ in range(steps)]
    p0 = torch.from_numpy(random_gaussians(n, W, H, seed=11))
    r = gs.GaussianRasterizer(W, H, n)
    st = torch.cuda.Stream()
    s = int(st.cuda_stream)
    rgb = torch.empty((H, W, 3), dtype=torch.uint8).pin_memory()
    h_p = p0.clone().pin_memory()
    outs = [torch.empty_like(p0).pin_memory() for _ in range(2)]
    d_rgb = torch.empty((H, W, 3), dtype=torch.uint8, device="cuda")
    d_frame = torch.empty((3, H, W), device="cuda")
    d_p = torch.empty((9, n), device="cuda")
    m, v = torch.empty_like(d_p), torch.empty_like(d_p)
    got = []
    with torch.cuda.stream(st):
        nat.fit_reset(r.plan, r.ws_ptr, m.data_ptr(), v.data_ptr(), s)
        for k in range(steps):
            st.synchronize()
            rgb.copy_(torch.from_numpy(frames[k]))
            out = outs[k // 3]  # the fourth call writes to another buffer
            nat.fit_step_rgb8(r.plan, r.ws_ptr, rgb.data_ptr(), d_rgb.data_ptr(),
                              d_frame.data_ptr(), h_p.data_ptr(), d_p.data_ptr(), m.data_ptr(),
                              v.data_ptr(), out.data_ptr(), s)
            st.synchronize()
            got.append(out.clone())
            h_p.copy_(out)
    # the same iterations by parts
    q = p0.cuda()
    m2, v2 = torch.empty_like(q), torch.empty_like(q)
    s0 = int(torch.cuda.current_stream().cuda_stream)
    nat.fit_reset(r.plan, r.ws_ptr, m2.data_ptr(), v2.data_ptr(), s0)
    for k in range(steps):
        frame = gs.frame_from_rgb8(torch.from_numpy(frames[k]).cuda())
        nat.fit_step(r.plan, r.ws_ptr, frame.data_ptr(), q.data_ptr(), m2.data_ptr(),
                     v2.data_ptr(), s0)
        torch.cuda.synchronize()
        assert torch.equal(got[k], q.cpu()), k
