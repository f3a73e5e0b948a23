"""Pins of the bitstream-accounting oracle (Sec. 3.3 B, Eq. 3-4): small
factorials by hand, Stirling's bounds, the paper's constant-count form of
Eq. 4, and entropy closed forms (uniform, constant, two-symbol)."""

import math

import numpy as np
import pytest

from oracle import bitstream as B


def test_bitsback_saving_small_cases():
    # log2(m!) - log2(m) = log2((m - 1)!)
    assert B.bitsback_saving(0) == 0.0 and B.bitsback_saving(1) == 0.0
    assert B.bitsback_saving(2) == pytest.approx(0.0, abs=1e-15)
    assert B.bitsback_saving(3) == pytest.approx(1.0)                 # log2 2
    assert B.bitsback_saving(4) == pytest.approx(math.log2(6))
    assert B.bitsback_saving(11) == pytest.approx(math.log2(3628800))


@pytest.mark.parametrize("m", [10, 100, 1000])
def test_log2_factorial_within_stirling_bounds(m):
    # Robbins: sqrt(2 pi m) (m/e)^m e^(1/(12m+1)) < m! < sqrt(2 pi m) (m/e)^m e^(1/(12m))
    base = 0.5 * math.log2(2 * math.pi * m) + m * math.log2(m / math.e)
    lf = B.log2_factorial(m)
    assert base + 1 / (12 * m + 1) / math.log(2) < lf < base + 1 / (12 * m) / math.log(2)


def test_log2_factorial_large_matches_stirling_series():
    m = 20000
    base = 0.5 * math.log2(2 * math.pi * m) + m * math.log2(m / math.e)
    series = base + (1 / (12 * m) - 1 / (360 * m ** 3)) / math.log(2)
    assert B.log2_factorial(m) == pytest.approx(series, rel=1e-12)


def test_sequence_with_constant_p_counts_is_eq4():
    F, K, N = 60, 4, 20000
    m = N // 20
    counts = [N if k % K == 0 else m for k in range(F)]
    payload = [1e6 if k % K == 0 else m * 100.0 for k in range(F)]
    res = B.sequence_bits(counts, payload, K)
    assert res["i_frames"] == F // K and res["p_frames"] == F - F // K
    # Eq. 4: S_total = (F - F/K) S_P
    assert res["savings"] == pytest.approx((F - F / K) * B.bitsback_saving(m), rel=1e-12)
    assert res["i_bits"] == (F // K) * 1e6
    assert res["p_bits"] == (F - F // K) * m * 100.0
    assert res["total_bits"] == pytest.approx(res["i_bits"] + res["p_bits"] - res["savings"])


def test_code_entropy_closed_forms():
    n = 4096
    bits = [12, 8, 1, 16, 0, 8, 8, 8, 8]
    c = np.zeros((9, n), np.uint16)
    c[0] = np.arange(n)                     # all distinct: n log2 n
    c[1] = 7                                # constant: 0
    c[2] = np.arange(n) % 2                 # two equal halves: n bits
    c[3, : n // 4] = 1                      # 1/4 vs 3/4: n H(1/4)
    c[5] = np.arange(n) % 256               # uniform over 256 symbols: 8 n
    e = B.code_entropy_bits(c, bits)
    h = -(0.25 * math.log2(0.25) + 0.75 * math.log2(0.75))
    assert e[0] == pytest.approx(n * 12.0)
    assert e[1] == 0.0
    assert e[2] == pytest.approx(n)
    assert e[3] == pytest.approx(n * h)
    assert e[4] == 32.0 * n                 # float32 row
    assert e[5] == pytest.approx(8.0 * n)
    # never above the fixed-length size of the row
    rng = np.random.default_rng(0)
    r = rng.integers(0, 1 << 10, (9, 3000)).astype(np.uint16)
    assert np.all(B.code_entropy_bits(r, [10] * 9) <= 10 * 3000 + 1e-6)
    # a selection codes only its columns
    sel = np.zeros(n, np.uint8)
    sel[::2] = 1
    es = B.code_entropy_bits(c, bits, sel)
    assert es[0] == pytest.approx((n // 2) * 11.0) and es[2] == 0.0
