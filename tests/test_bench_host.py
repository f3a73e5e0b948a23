"""Host helpers of bench.py (no GPU): the clock-sample summary behind the
line's `clocks` key, the ncu traffic lookup (valid only for the captured
schedule and render source), and the HBM peak's fallback."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(sm, mx, hw="Not Active", thermal="Not Active", sw_thermal="Not Active",
         power="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, {thermal}, {sw_thermal}, {power}\n"


def test_clock_summary_within_the_timed_region(bench):
    s = bench.ClockSampler(0)
    s.proc = _Proc()
    s.lines = [(0.5, _row(1000, 2070, hw="Active")),      # before the region
               (1.0, _row(2070, 2070)), (1.2, _row(2055, 2070, power="Active")),
               (1.4, _row(2070, 2070)), (9.0, _row(800, 2070, thermal="Active"))]
    c = s.stop(1.0, 1.5)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]  # the hw / thermal rows fall outside


def test_clock_summary_short_region_and_bad_rows(bench):
    s = bench.ClockSampler(0)
    s.proc = _Proc()
    s.lines = [(1.0, _row(1980, 2070)), (3.0, "garbage\n"), (5.0, _row("[N/A]", 2070))]
    c = s.stop(2.0, 2.01)  # no sample inside: the nearest one
    assert c["sm_mhz"] == 1980.0 and c["samples"] == 1
    s2 = bench.ClockSampler(0)
    assert s2.stop()["reasons"] == ["nvidia-smi unavailable"]  # never started


def test_traffic_only_for_the_captured_schedule_and_source(bench):
    t = bench.render_traffic(bench.NCU_TRAFFIC["schedule"])
    assert t == bench.NCU_TRAFFIC["bytes"]  # the committed render source was captured
    assert bench.render_traffic((16, 64, 1)) is None


def test_hbm_peak_measured_or_fallback(bench, monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak_gbs() == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    assert bench.hbm_peak_gbs() == 7000.5


def test_render_work_counts(bench):
    """The per-listed-pair count (8 FP32 operations per listed pair of tight
    16-px lists in each pass, 3 / 20 more per contributing pair) and the
    strict count (11 / 22 per contributing pair), and one ex2 per listed pair
    and pass."""
    w = bench.render_work(1000, 300)
    assert w["fwd"] == 8 * 1000 + 3 * 300 and w["bwd"] == 8 * 1000 + 20 * 300
    assert w["fused"] == w["fwd"] + w["bwd"]
    assert w["fwd_strict"] == 11 * 300 and w["bwd_strict"] == 22 * 300
    assert w["fused_strict"] == 33 * 300 and w["mufu_per_pass"] == 1000


def test_binning_bytes(bench):
    b = bench.binning_bytes(n=20000, entries=100000, tiles=2040)
    assert b["project"] == (36 + 48 + 16 + 4) * 20000
    assert b["bin_sort"] == 24 * 20000 + 12 * 100000 + 16 * 2040


def test_paper_encode_reference(bench):
    """Table 1's numbers behind the quoted -88 %."""
    p = bench.PAPER_ENCODE
    assert p["superpixel_s"] == 1.5 and p["random_init_s"] == 13.1
    assert abs(p["reduction"] - 0.885) < 1e-3  # the paper rounds it to 88 %
