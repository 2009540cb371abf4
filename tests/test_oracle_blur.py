"""Pins of oracle.blur: invariant special cases, adjointness, Eq. 3 vs the basis form."""
import numpy as np
from scipy.signal import convolve2d

from oracle import blur, psf


def _setup(seed=11, h=20, w=23, c=2, K=3, th=5, tw=7):
    rng = np.random.default_rng(seed)
    x = rng.uniform(size=(h, w, c))
    Hb = rng.normal(size=(K, th * tw))
    beta = rng.normal(size=(h, w, K))
    return rng, x, Hb, beta


def test_constant_beta_is_invariant_convolution():
    rng, x, Hb, _ = _setup()
    b = rng.normal(size=3)
    beta = np.broadcast_to(b, (20, 23, 3))
    kern = (b @ Hb).reshape(5, 7)
    ys = blur.scatter(x, beta, Hb, 5, 7)
    yg = blur.gather(x, beta, Hb, 5, 7)
    for c in range(2):
        ref = convolve2d(x[:, :, c], kern, mode="same")
        assert np.max(np.abs(ys[:, :, c] - ref)) < 1e-12
        assert np.max(np.abs(yg[:, :, c] - ref)) < 1e-12


def test_single_basis_vector():
    _, x, Hb, _ = _setup()
    beta = np.zeros((20, 23, 3))
    beta[..., 1] = 2.5
    y = blur.scatter(x, beta, Hb, 5, 7)
    ref = convolve2d(x[:, :, 0], 2.5 * Hb[1].reshape(5, 7), mode="same")
    assert np.max(np.abs(y[:, :, 0] - ref)) < 1e-12


def test_delta_image_gives_that_pixels_psf():
    _, _, Hb, beta = _setup()
    x = np.zeros((20, 23, 1))
    x[9, 11, 0] = 1.0
    y = blur.scatter(x, beta, Hb, 5, 7)
    G = (beta[9, 11] @ Hb).reshape(5, 7)
    assert np.allclose(y[7:12, 8:15, 0], G, atol=1e-14)
    assert abs(y.sum() - G.sum()) < 1e-12


def test_scatter_adjoint_is_gather_with_flipped_psfs():
    rng, x, Hb, beta = _setup()
    z = rng.normal(size=x.shape)
    flip = Hb.reshape(3, 5, 7)[:, ::-1, ::-1].reshape(3, -1)
    lhs = np.sum(blur.scatter(x, beta, Hb, 5, 7) * z)
    rhs = np.sum(x * blur.gather(z, beta, flip, 5, 7))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_exact_blur_vs_basis_with_projected_beta():
    rng = np.random.default_rng(12)
    h, w, th = 10, 12, 5
    T = th * th
    alpha = 0.6 * rng.normal(size=(h, w, 33))
    hp = psf.psf_taps(alpha, th, th, 16, 32)
    x = rng.uniform(size=(h, w, 3))
    y_exact = blur.exact(x, hp)
    Q, _ = np.linalg.qr(rng.normal(size=(T, T)))
    full = Q.T  # K = T orthonormal basis
    beta = hp.reshape(h, w, T) @ full.T
    assert np.max(np.abs(blur.scatter(x, beta, full, th, th) - y_exact)) < 1e-12
    part = full[:7]
    beta7 = hp.reshape(h, w, T) @ part.T
    resid = hp - (beta7 @ part).reshape(h, w, th, th)
    diff = y_exact - blur.scatter(x, beta7, part, th, th)
    assert np.max(np.abs(diff - blur.exact(x, resid))) < 1e-12
