"""The oracle against its stored golden fixtures (``tests/golden/``).

The fixtures were written by ``tests/golden/make_golden.py`` from the oracle
itself on seeded inputs: they guard the oracle against unnoticed change (its
pins to the paper and to mathematics are the other ``test_oracle_*`` files).
Sums and samples must agree within a relative 1e-12, the spread that OpenMP
and BLAS summation order can leave in float64."""

import importlib.util
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ["render", "loss_grad", "conv", "quantize", "roi_init", "sequence_bits"]


@pytest.fixture(scope="module")
def current():
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.fixtures()


def close(a, b, scale):
    return abs(a - b) <= 1e-12 * max(abs(a), abs(b), scale) + 1e-300


@pytest.mark.parametrize("name", NAMES)
def test_oracle_matches_golden(current, name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        stored = json.load(f)
    now = current[name]
    assert now["cites"] == stored["cites"] and now["inputs"] == stored["inputs"]
    assert set(now["outputs"]) == set(stored["outputs"])
    for key, s in stored["outputs"].items():
        c = now["outputs"][key]
        assert c["shape"] == s["shape"] and c["idx"] == s["idx"], key
        scale = np.sqrt(s["sumsq"] / max(1, int(np.prod(s["shape"]))))
        assert close(c["sum"], s["sum"], scale * np.sqrt(np.prod(s["shape"]))), key
        assert close(c["sumsq"], s["sumsq"], s["sumsq"]), key
        for v, w in zip(c["values"], s["values"]):
            assert close(v, w, scale), (key, v, w)


def test_every_fixture_is_tested():
    stored = sorted(f[:-5] for f in os.listdir(GOLDEN) if f.endswith(".json"))
    assert stored == sorted(NAMES)
