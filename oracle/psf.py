"""Pupil-FFT point spread function (Eq. 2), PSF dictionary and SVD basis (Sec. 3.2).

Eq. 2 forms the incoherent PSF as h = |F{W(rho) exp(-j phi(rho))}|^2 with W
the aperture and phi the Zernike phase of Eq. 1.  Reading of the sampling:

  pupil   N_p x N_p samples, sample centres at (i - (N_p - 1)/2) pupil samples,
          unit-disk radius N_p / 2, W = 1 where r <= 1;
  DFT     zero-padded to N_fft = 2 N_p (forward DFT, NumPy sign convention),
          |.|^2, then shifted so zero frequency sits at (N_fft/2, N_fft/2);
  taps    the centred taps_h x taps_w window, normalised to unit sum.
          Tap (ty, tx) is the fraction of a source pixel's light that lands
          at offset (ty - taps_h//2, tx - taps_w//2) from it.

Basis (Sec. 3.2): a dictionary of N_dict centred PSFs (tilts J = 2, 3 removed)
with D/r0 from weak to strong turbulence, then the top-K right singular
vectors of the N_dict x T dictionary, without mean removal, so that
h ~ sum_k beta_k h_k is exactly the form the blur uses.  The sign of each
basis vector is fixed so that its taps sum to >= 0.

Pins (tests/test_oracle_psf.py): FFT PSF against a direct DFT sum; zero phase
against the Airy pattern |2 J1(v)/v|^2 with error shrinking as N_p grows;
Parseval (energy independent of phi); orthonormal basis and the projection
identity; an integer tilt is an exact roll (which also fixes kappa).
"""
from __future__ import annotations

import numpy as np

from . import noll
from .zernike import zernike


def pupil_grid(n_pupil: int):
    c = (n_pupil - 1) / 2.0
    v, u = np.meshgrid(np.arange(n_pupil) - c, np.arange(n_pupil) - c, indexing="ij")
    rad = n_pupil / 2.0
    x, y = u / rad, v / rad
    r = np.hypot(x, y)
    theta = np.arctan2(y, x)
    mask = (r <= 1.0).astype(np.float64)
    return r, theta, mask


def zernike_stack(js, n_pupil: int) -> np.ndarray:
    """[len(js), N_p, N_p] Zernike modes sampled on the pupil."""
    r, theta, _ = pupil_grid(n_pupil)
    return np.stack([zernike(j, r, theta) for j in js])


def psf_full(alpha: np.ndarray, js, n_pupil: int = 32, n_fft: int = 64) -> np.ndarray:
    """Unnormalised, uncropped PSFs |DFT(W e^{-j phi})|^2, centred.  alpha [..., len(js)]."""
    _, _, mask = pupil_grid(n_pupil)
    Z = zernike_stack(js, n_pupil)
    alpha = np.asarray(alpha, dtype=np.float64)
    phi = np.tensordot(alpha, Z, axes=([-1], [0]))
    field = mask * np.exp(-1j * phi)
    pad = np.zeros(alpha.shape[:-1] + (n_fft, n_fft), dtype=np.complex128)
    pad[..., :n_pupil, :n_pupil] = field
    X = np.fft.fft2(pad)
    h = np.abs(X) ** 2
    return np.fft.fftshift(h, axes=(-2, -1))


def crop_normalise(h: np.ndarray, taps_h: int, taps_w: int) -> np.ndarray:
    n = h.shape[-1]
    c = n // 2
    win = h[..., c - taps_h // 2 : c - taps_h // 2 + taps_h, c - taps_w // 2 : c - taps_w // 2 + taps_w]
    return win / win.sum(axis=(-2, -1), keepdims=True)


HIGH_ORDER = list(range(4, 37))  # J = 4..36, the P2S network input


def psf_taps(alpha_hi: np.ndarray, taps_h: int, taps_w: int, n_pupil: int = 32, n_fft: int = 64) -> np.ndarray:
    """Centred, cropped, unit-sum PSFs of the high-order coefficients alpha_hi [..., 33]."""
    return crop_normalise(psf_full(alpha_hi, HIGH_ORDER, n_pupil, n_fft), taps_h, taps_w)


def dictionary(z: np.ndarray, dr0: np.ndarray, taps_h: int, taps_w: int, n_pupil: int = 32, n_fft: int = 64,
               chunk: int = 2000, phase_scale: float = 1.0) -> np.ndarray:
    """N_dict x T matrix of centred PSFs.

    Draw i has alpha_{2..36} = dr0_i^(5/6) L z_i (L = chol(R_Z)); the tilts
    J = 2, 3 are dropped so the PSF is centred (Sec. 3.2).  phase_scale multiplies
    the phase (the coefficients are in radians at another wavelength: oracle.spectral).
    """
    L = noll.cholesky_lower(noll.noll_cov(36))
    alpha = (dr0[:, None] ** (5.0 / 6.0)) * (z @ L.T)
    hi = alpha[:, 2:] * phase_scale
    rows = []
    for s in range(0, len(hi), chunk):
        rows.append(psf_taps(hi[s : s + chunk], taps_h, taps_w, n_pupil, n_fft).reshape(-1, taps_h * taps_w))
    return np.concatenate(rows)


def svd_basis(D: np.ndarray, K: int) -> np.ndarray:
    """Top-K right singular vectors of the dictionary, [K, T], sign so each sums >= 0."""
    _, _, vt = np.linalg.svd(D, full_matrices=False)
    H = vt[:K].copy()
    neg = H.sum(axis=1) < 0
    H[neg] *= -1.0
    return H


def make_basis(z: np.ndarray, dr0: np.ndarray, K: int, taps: int, n_pupil: int = 32, n_fft: int = 64,
               phase_scale: float = 1.0):
    """Dictionary of the given draws -> basis.  Returns (H [K, T], D [N_dict, T])."""
    D = dictionary(z, dr0, taps, taps, n_pupil, n_fft, phase_scale=phase_scale)
    return svd_basis(D, K), D
