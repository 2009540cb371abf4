"""Offline basis learning (Sec. 3.2): a dictionary of centred PSFs -> SVD basis.

This is the one-off host step that precedes the simulator, not part of the
per-frame path: the paper builds its basis from 50,000 PSFs spanning weak to
strong turbulence and keeps M = 100 principal components (Sec. 3.2).  Here, in
FP64 on the host:

  draws   alpha_{2..36} = (D/r0)^(5/6) chol(R_Z) z, z ~ N(0, I),
          D/r0 ~ U[0.5, 6]; R_Z comes from libp2s (p2s_noll_covariance);
  PSF     Eq. 2 on an N_p x N_p pupil zero-padded to N_fft = 2 N_p, tilts
          J = 2, 3 left out so the PSF is centred; the centred taps window,
          normalised to unit sum;
  basis   top-K right singular vectors of the N_dict x T dictionary (no mean
          removal), each signed so its taps sum to >= 0.

Results are cached under _build/ keyed by every parameter.
"""
from __future__ import annotations

import os
from math import factorial, sqrt

import numpy as np

from . import inputs, p2s

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")


def _noll_nm(j: int):
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    k = j - n * (n + 1) // 2 - 1
    return n, (2 * ((k + 1) // 2) if n % 2 == 0 else 2 * (k // 2) + 1)


def _zernike_modes(js, n_pupil: int) -> np.ndarray:
    """Noll-normalised Zernike modes sampled at the pupil sample centres."""
    c = (n_pupil - 1) / 2.0
    yy, xx = np.meshgrid((np.arange(n_pupil) - c) / (n_pupil / 2.0), (np.arange(n_pupil) - c) / (n_pupil / 2.0),
                         indexing="ij")
    r = np.hypot(xx, yy)
    th = np.arctan2(yy, xx)
    out = []
    for j in js:
        n, m = _noll_nm(j)
        R = np.zeros_like(r)
        for s in range((n - m) // 2 + 1):
            R += ((-1) ** s * factorial(n - s) / (factorial(s) * factorial((n + m) // 2 - s)
                                                  * factorial((n - m) // 2 - s))) * r ** (n - 2 * s)
        if m == 0:
            out.append(sqrt(n + 1) * R)
        else:
            ang = np.cos(m * th) if j % 2 == 0 else np.sin(m * th)
            out.append(sqrt(2 * (n + 1)) * R * ang)
    return np.stack(out), (r <= 1.0).astype(np.float64)


def psf_dictionary(n_dict: int, taps: int, n_pupil: int = 32, n_fft: int = 64, seed: int = 2021,
                   dr0_range=(0.5, 6.0), chunk: int = 2000, with_alpha: bool = False, phase_scale: float = 1.0):
    """[n_dict, taps*taps] unit-sum PSFs (and, with_alpha, the [n_dict, 35] coefficients alpha_2..36).

    phase_scale: the PSFs seen at another wavelength (phase alpha * phase_scale; pass the pupil
    sample count of that wavelength as n_pupil, see build_basis_spectral)."""
    z, dr0 = inputs.dictionary_draws(n_dict, 35, dr0_range, seed)
    L = np.linalg.cholesky(p2s.noll_covariance(36))
    alpha = (dr0[:, None] ** (5.0 / 6.0)) * (z @ L.T)
    Z, mask = _zernike_modes(range(4, 37), n_pupil)
    Zf = Z.reshape(33, -1)
    c = n_fft // 2
    h0 = c - taps // 2
    rows = []
    for s0 in range(0, n_dict, chunk):
        phi = ((alpha[s0:s0 + chunk, 2:] * phase_scale) @ Zf).reshape(-1, n_pupil, n_pupil)
        pad = np.zeros((phi.shape[0], n_fft, n_fft), dtype=np.complex128)
        pad[:, :n_pupil, :n_pupil] = mask * np.exp(-1j * phi)
        h = np.fft.fftshift(np.abs(np.fft.fft2(pad)) ** 2, axes=(-2, -1))[:, h0:h0 + taps, h0:h0 + taps]
        h = h.reshape(h.shape[0], -1)
        rows.append(h / h.sum(axis=1, keepdims=True))
    D = np.concatenate(rows)
    return (D, alpha) if with_alpha else D


def build_basis(K: int = 100, taps: int = 33, n_dict: int = 50_000, n_pupil: int = 32, n_fft: int = 64,
                seed: int = 2021, cache: bool = True) -> np.ndarray:
    """[K, taps*taps] FP64 basis; cached on disk by its parameters."""
    path = os.path.join(_CACHE, f"basis_K{K}_T{taps}_N{n_dict}_P{n_pupil}_F{n_fft}_S{seed}.npy")
    if cache and os.path.exists(path):
        return np.load(path)
    D = psf_dictionary(n_dict, taps, n_pupil, n_fft, seed)
    _, _, vt = np.linalg.svd(D, full_matrices=False)
    H = vt[:K].copy()
    H[H.sum(axis=1) < 0] *= -1.0
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        np.save(path, H)
    return H


def build_basis_spectral(K: int = 100, taps: int = 33, n_dict: int = 50_000, wavelengths_nm=(570.0, 540.0, 450.0),
                         ref_nm: float = 540.0, n_pupil: int = 32, n_fft: int = 64, seed: int = 2021,
                         cache: bool = True):
    """Three [K, taps*taps] bases, one per colour channel (Sec. 3.5): the same draws seen at
    wavelength lambda_c, i.e. the phase scaled by s_c = lambda_ref / lambda_c and the pupil
    sampled with round(n_pupil s_c) samples across in the same n_fft DFT (the image pixel is
    one angle at every wavelength, so the diffraction PSF widens with lambda)."""
    out = []
    for lam in wavelengths_nm:
        s = ref_nm / lam
        npc = int(round(n_pupil * s))
        path = os.path.join(_CACHE, f"basis_K{K}_T{taps}_N{n_dict}_P{npc}_F{n_fft}_S{seed}_L{lam:g}_R{ref_nm:g}.npy")
        if cache and os.path.exists(path):
            out.append(np.load(path))
            continue
        D = psf_dictionary(n_dict, taps, npc, n_fft, seed, phase_scale=s)
        _, _, vt = np.linalg.svd(D, full_matrices=False)
        H = vt[:K].copy()
        H[H.sum(axis=1) < 0] *= -1.0
        if cache:
            os.makedirs(_CACHE, exist_ok=True)
            np.save(path, H)
        out.append(H)
    return out
