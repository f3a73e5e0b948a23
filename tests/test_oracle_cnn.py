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
