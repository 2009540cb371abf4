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


def test_packed_f16_sums_error_budget():
    """The packed-FP16 gather kernel (gather_split = 4) keeps FP16 sums of 12 tap products:
    on the blur-stage inputs of the GPU tests its emulated arithmetic stays within 1e-3
    relative L2 of the exact gather (the 16-bit tolerance is 2e-3), and the FP16 sums move the
    result by 1e-4 .. 1e-3 against FP32 sums of the same FP16 products (kernel 1's arithmetic,
    itself within 4e-4 of the exact gather)."""
    import oracle
    from paper_2107_11627_gb300 import inputs

    import kernel_emulation

    z, dr0 = inputs.dictionary_draws(600, 35, (0.5, 6.0), 2021)
    H, _ = oracle.psf.make_basis(z, dr0, K=100, taps=33)
    rng = np.random.default_rng(31)
    h, w = 33, 64
    x = inputs.blob_image(h, w, 3, 1003)
    beta = (rng.normal(0.0, 0.05, size=(h, w, 100)) + 0.3 * (np.arange(100) == 0)).astype(np.float32)
    f16 = lambda v: v.astype(np.float16).astype(np.float64)
    ref = oracle.blur.gather(x.astype(np.float64), beta.astype(np.float64), H, 33, 33)
    emu = kernel_emulation.gather_h2(x, beta, H, f16)
    g16 = f16(f16(beta.reshape(h * w, -1).astype(np.float64)) @ f16(H)).reshape(h, w, -1)
    fp32_sums = oracle.blur.gather(f16(x.astype(np.float64)), g16.reshape(h * w, -1), np.eye(33 * 33), 33, 33)
    rel = lambda a, b=ref: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(emu) < 1e-3, rel(emu)
    assert rel(fp32_sums) < 4e-4, rel(fp32_sums)
    assert 1e-4 < rel(emu, fp32_sums) < 1e-3, rel(emu, fp32_sums)
