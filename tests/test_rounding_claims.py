"""CPU checks of the arithmetic facts the 16-bit kernels rely on (no GPU involved).

- The product of two FP16 values is exact in FP32 (11 + 11 significant bits <= 24), so a
  mixed FP16 x FP16 + FP32 fused multiply-add rounds once, exactly like fmaf of the widened
  operands: the split gather's tap products and the emulation in its rounding-point test.
- Rounding G to FP16 changes a tap product by at most 2^-11 relative (normal range); below
  the normal range the absolute change is at most 2^-25.
"""
import numpy as np


def _random_f16(rng, n):
    bits = rng.integers(0, 2**16, size=n, dtype=np.uint16)
    v = bits.view(np.float16)
    return v[np.isfinite(v)]


def test_f16_products_exact_in_f32():
    rng = np.random.default_rng(5)
    a = _random_f16(rng, 200_000).astype(np.float64)
    b = _random_f16(rng, a.size)[: a.size].astype(np.float64)
    a = a[: b.size]
    p64 = a * b  # exact in FP64 (22 significant bits)
    p32 = (a.astype(np.float32) * b.astype(np.float32)).astype(np.float64)
    finite = np.isfinite(p32) & (np.abs(p64) < np.finfo(np.float32).max)
    # FP32 keeps every such product exactly unless it falls below FP32's normal range
    # (FP16 x FP16 >= 2^-48, which is normal in FP32)
    assert np.array_equal(p32[finite], p64[finite])


def test_g_rounding_bound():
    rng = np.random.default_rng(6)
    g = rng.normal(0.0, 1e-2, size=200_000) * np.exp(rng.uniform(-8, 0, size=200_000))
    g16 = g.astype(np.float16).astype(np.float64)
    normal = np.abs(g) >= 2.0**-14
    assert np.all(np.abs(g16 - g)[normal] <= 2.0**-11 * np.abs(g)[normal])
    assert np.all(np.abs(g16 - g)[~normal] <= 2.0**-25)
