"""Pins of oracle.warp: kappa from the oracle PSF, and the bilinear sampler."""
import numpy as np

from oracle import psf, warp


def test_integer_tilt_is_exact_roll():
    # alpha_2 = 1/kappa moves the PSF by exactly +1 column (DFT shift theorem), alpha_3 by +1 row.
    n_p, n_f = 32, 64
    k = warp.kappa(n_f, n_p)
    assert abs(k + 4 / np.pi) < 1e-15
    rng = np.random.default_rng(3)
    hi = 0.3 * rng.normal(size=33)
    base = psf.psf_full(np.concatenate([[0.0, 0.0], hi]), [2, 3] + psf.HIGH_ORDER, n_p, n_f)
    tx = psf.psf_full(np.concatenate([[1.0 / k, 0.0], hi]), [2, 3] + psf.HIGH_ORDER, n_p, n_f)
    ty = psf.psf_full(np.concatenate([[0.0, 2.0 / k], hi]), [2, 3] + psf.HIGH_ORDER, n_p, n_f)
    scale = base.max()
    assert np.max(np.abs(tx - np.roll(base, 1, axis=1))) < 1e-12 * scale
    assert np.max(np.abs(ty - np.roll(base, 2, axis=0))) < 1e-12 * scale


def test_integer_shift_and_clamp():
    rng = np.random.default_rng(4)
    x = rng.uniform(size=(12, 15, 3))
    dr = np.full((12, 15), 2.0)
    dc = np.full((12, 15), -3.0)
    xw = warp.bilinear_backward(x, dr, dc)
    for i in range(12):
        for j in range(15):
            si, sj = min(max(i - 2, 0), 11), min(max(j + 3, 0), 14)
            assert np.allclose(xw[i, j], x[si, sj], atol=1e-15)


def test_half_pixel_and_identity():
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(7, 9, 1))
    z = np.zeros((7, 9))
    assert np.array_equal(warp.bilinear_backward(x, z, z), x)
    xw = warp.bilinear_backward(x, z, z + 0.5)
    ref = 0.5 * (x + np.concatenate([x[:, :1], x[:, :-1]], axis=1))
    assert np.allclose(xw, ref, atol=1e-15)


def test_displacement_uses_tilt_modes():
    a = np.zeros((2, 2, 35))
    a[..., 0] = 1.0  # alpha_2 -> columns
    a[..., 1] = 2.0  # alpha_3 -> rows
    dr, dc = warp.displacement(a, -4 / np.pi)
    assert np.allclose(dc, -4 / np.pi) and np.allclose(dr, -8 / np.pi)


def test_blur_and_integer_shift_commute_in_the_interior():
    """Pin for the two orders of the path: with one shift-invariant PSF (constant beta) and a
    constant integer shift, warp(blur(x)) == blur(warp(x)) away from the borders."""
    from oracle import blur, warp

    rng = np.random.default_rng(5)
    h, w, K, T = 40, 44, 3, 5
    x = rng.uniform(size=(h, w, 2))
    Hb = rng.normal(size=(K, T * T))
    beta = np.broadcast_to(rng.normal(size=K), (h, w, K)).copy()
    kap = warp.kappa()
    ap = np.zeros((h, w, 35))
    ap[..., 0] = 3.0 / kap   # alpha_2 -> +3 columns
    ap[..., 1] = -2.0 / kap  # alpha_3 -> -2 rows
    a = warp.warp(blur.scatter(x, beta, Hb, T, T), ap, kap)
    b = blur.scatter(warp.warp(x, ap, kap), beta, Hb, T, T)
    m = 8
    assert np.allclose(a[m:-m, m:-m], b[m:-m, m:-m], atol=1e-12)
