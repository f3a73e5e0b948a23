"""Host control flow of raster.encode_sequence (no GPU): which frames are
I-frames and which P-frames, the iteration budgets, the reference render the
selection compares against, and the per-frame records and callbacks; the
rasterizer is a stand-in that records its calls."""

import pytest

torch = pytest.importorskip("torch")


class FakeRast:
    n = 10

    def __init__(self):
        self.calls = []

    def encode_frame(self, frame, params, iters, target_psnr, check_every, adam_state, stream):
        self.calls.append(("I", int(frame[0, 0, 0]), iters))
        params += 1.0
        return {"iters": iters, "psnr": 30.0 + float(frame[0, 0, 0])}

    def prepare(self, params, stream=None):
        self.calls.append(("prepare", float(params[0, 0])))

    def render_fwd(self, out=None, stream=None):
        self.calls.append(("render", out is not None))
        return torch.zeros(3, 2, 2)

    def select_changed(self, ref, frame, threshold, stream=None):
        self.calls.append(("select", int(frame[0, 0, 0]), threshold))
        sel = torch.zeros(self.n, dtype=torch.uint8)
        sel[:4] = 1
        return sel, 4

    def encode_pframe(self, frame, params, sel, iters, adam_state, stream=None):
        self.calls.append(("P", int(frame[0, 0, 0]), iters))
        params[:, sel.bool()] += 0.5
        return 40.0


def frames(k):
    return [torch.full((3, 2, 2), float(i)) for i in range(k)]


def test_gop_schedule_and_records():
    from paper_2505_09324_gb300.raster import encode_sequence
    r = FakeRast()
    p = torch.zeros(9, FakeRast.n)
    seen = []
    out = encode_sequence(r, frames(7), p, 50, 5, selective_threshold=0.02, gop=3,
                          on_frame=lambda k, params, sel: seen.append((k, sel is None)))
    kinds = [c for c in r.calls if c[0] in ("I", "P")]
    assert kinds == [("I", 0, 50), ("P", 1, 5), ("P", 2, 5), ("I", 3, 5), ("P", 4, 5),
                     ("P", 5, 5), ("I", 6, 5)]
    assert [o["coded"] for o in out] == [10, 4, 4, 10, 4, 4, 10]
    assert [s for _, s in seen] == [True, False, False, True, False, False, True]
    assert all(o.get("selected", 4) == 4 for o in out)
    # each P-frame selects against a fresh render of the current Gaussians,
    # reusing the reference buffer after the first
    renders = [c for c in r.calls if c[0] == "render"]
    assert renders == [("render", False)] + [("render", True)] * 3
    sel = [c for c in r.calls if c[0] == "select"]
    assert [c[1] for c in sel] == [1, 2, 4, 5] and all(c[2] == 0.02 for c in sel)
    assert float(p[0, 0]) == 3 * 1.0 + 4 * 0.5 and float(p[0, -1]) == 3.0


def test_warm_start_without_selection_fits_every_frame_fully():
    from paper_2505_09324_gb300.raster import encode_sequence
    r = FakeRast()
    p = torch.zeros(9, FakeRast.n)
    out = encode_sequence(r, frames(4), p, 20, 3)
    assert [c for c in r.calls] == [("I", 0, 20), ("I", 1, 3), ("I", 2, 3), ("I", 3, 3)]
    assert [o["psnr"] for o in out] == [30.0, 31.0, 32.0, 33.0]
    assert all(o["coded"] == 10 for o in out)
