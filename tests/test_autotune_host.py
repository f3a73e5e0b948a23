"""Host logic of the Python autotuner (no GPU): the choice across backward
reductions, the table keys, the overflow case and the cache, with the C
autotuner replaced by a stand-in that returns fixed timings."""

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def rs(monkeypatch):
    from paper_2505_09324_gb300 import _native as nat
    from paper_2505_09324_gb300 import raster
    calls = []

    def fake_autotune(sizes, params, targets, ws, nbytes, tiles, stages, launches, reps, stream,
                      max_entries, cfg):
        calls.append(cfg.reduce)
        table = {}
        for t in tiles:
            for s in stages:
                for la in launches:
                    # atomic reduction faster at tile 16 only; one overflowing candidate
                    ms = 1.0 + t / 100 + s / 1000 + la / 10
                    if cfg.reduce == nat.REDUCE_ATOMIC and t == 16:
                        ms -= 0.5
                    if t == 8 and s == 32:
                        ms = -1.0
                    table[(t, s, la)] = ms
        best = min((k for k, v in table.items() if v >= 0), key=lambda k: table[k])
        return table, *best

    monkeypatch.setattr(nat, "autotune", fake_autotune)
    monkeypatch.setattr(nat, "autotune_ws_bytes", lambda *a: 1024)
    monkeypatch.setattr(raster, "_check", lambda t, *a, **k: 0)
    monkeypatch.setattr(raster, "_stream", lambda s: 0)
    raster._TUNED.clear()
    return raster, nat, calls


def test_default_considers_only_the_reproducible_reduction(rs):
    raster, nat, calls = rs
    p, t = torch.zeros(9, 4), torch.zeros(12)
    res = raster.autotune([(2, 2, 4)], p, t, cache=False)
    assert calls == [nat.REDUCE_SLOTS]
    assert res["reduce"] == nat.REDUCE_SLOTS and res["config"].reduce == nat.REDUCE_SLOTS
    assert all(len(k) == 3 for k in res["ms"])
    assert (res["tile"], res["stage"], res["launch"]) == (8, 64, 0)  # (8, 32) overflowed
    assert len(res["ms"]) == 3 * 4 * 2


def test_both_reductions_pick_the_faster_and_key_by_reduction(rs):
    raster, nat, calls = rs
    p, t = torch.zeros(9, 4), torch.zeros(12)
    res = raster.autotune([(2, 2, 4)], p, t, cache=False,
                          reduces=(nat.REDUCE_SLOTS, nat.REDUCE_ATOMIC))
    assert calls == [nat.REDUCE_SLOTS, nat.REDUCE_ATOMIC]
    assert res["reduce"] == nat.REDUCE_ATOMIC and res["config"].reduce == nat.REDUCE_ATOMIC
    assert all(len(k) == 4 for k in res["ms"]) and len(res["ms"]) == 2 * 3 * 4 * 2
    best = min(v for v in res["ms"].values() if v >= 0)
    assert res["ms"][(res["tile"], res["stage"], res["launch"], res["reduce"])] == best
    assert res["ms"][(8, 32, 0, nat.REDUCE_SLOTS)] == -1.0  # overflow kept as reported


def test_cache_is_keyed_by_the_candidates(rs):
    raster, nat, calls = rs
    p, t = torch.zeros(9, 4), torch.zeros(12)
    a = raster.autotune([(2, 2, 4)], p, t)
    b = raster.autotune([(2, 2, 4)], p, t)
    assert a is b and calls == [nat.REDUCE_SLOTS]
    c = raster.autotune([(2, 2, 4)], p, t, reduces=(nat.REDUCE_SLOTS, nat.REDUCE_ATOMIC))
    assert c is not a and len(calls) == 3
    with pytest.raises(ValueError):
        raster.autotune([(2, 2, 4)], p, t, reduces=(), cache=False)
