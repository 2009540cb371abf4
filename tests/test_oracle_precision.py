"""Pins of oracle.precision (round-to-nearest-even BF16 / FP8-E4M3)."""
import numpy as np

from oracle.precision import bf16, e4m3


def test_bf16_points():
    assert bf16(1.0) == 1.0
    assert bf16(1 + 2**-8) == 1.0  # tie -> even
    assert bf16(1 + 3 * 2**-8) == 1 + 2**-6  # tie -> even
    assert bf16(1 + 2**-7) == 1 + 2**-7
    assert bf16(-3.0) == -3.0
    x = np.random.default_rng(13).normal(size=1000)
    r = bf16(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2**-8 * (1 + 1e-12)


def test_e4m3_points():
    assert e4m3(448.0) == 448.0 and e4m3(500.0) == 448.0 and e4m3(-1e6) == -448.0
    assert e4m3(2**-9) == 2**-9
    assert e4m3(1.5 * 2**-9) == 2**-8  # tie -> even
    assert e4m3(0.3) == 0.3125
    assert e4m3(1.0625) == 1.0  # tie between 1.0 and 1.125 -> even
    assert e4m3(0.0) == 0.0
