"""Wavelength-dependent colour (Sec. 3.5): three PSF sets, one per colour channel.

The paper simulates RGB either with one PSF (525 nm) for all channels or with
three PSFs at 450, 540 and 570 nm, at three times the cost, and prints no
formula for the wavelength dependence.  Readings (one turbulence realisation
seen at three wavelengths):

  channels    R, G, B at 570, 540, 450 nm; the Zernike coefficients alpha are
              radians at the reference 540 nm;
  phase       the optical path difference is achromatic, so at lambda_c the
              phase is alpha * s_c with s_c = lambda_ref / lambda_c;
  sampling    the image pixel is one angle for every channel and the
              diffraction PSF widens with lambda: channel c's pupil has
              N_p,c = round(N_p s_c) samples across in the same N_fft-point DFT
              (sample spacing lambda / (N_fft * pupil pitch));
  tilts       the tilt angle is achromatic, so one warp serves all channels;
  network     beta_c = MLP_c(alpha_4..36 * s_c) over channel c's basis H_c
              (the same weights for every channel unless given per channel).

Test infrastructure, like the rest of the oracle.  Pins (tests/test_oracle_spectral.py):
s = 1 reduces to the single-wavelength functions; the zero-phase PSF width
scales as 1 / N_p,c; the Strehl ratio follows Marechal's exp(-s^2 sum alpha_j^2)
at small aberration; the spectral frame with every channel at the reference
equals the single-wavelength frame; channels do not interact.
"""
from __future__ import annotations

import numpy as np

from . import blur, fields, mlp, noll, psf, warp

WAVELENGTHS_NM = (570.0, 540.0, 450.0)  # R, G, B
REFERENCE_NM = 540.0


def phase_scale(lam_nm: float, ref_nm: float = REFERENCE_NM) -> float:
    return ref_nm / lam_nm


def pupil_samples(n_pupil: int, scale: float) -> int:
    return int(round(n_pupil * scale))


def psf_taps_at(alpha_hi: np.ndarray, taps: int, scale: float, n_pupil: int = 32, n_fft: int = 64) -> np.ndarray:
    """Centred unit-sum PSFs of alpha_hi (radians at the reference) seen at phase scale s."""
    return psf.psf_taps(np.asarray(alpha_hi) * scale, taps, taps, pupil_samples(n_pupil, scale), n_fft)


def make_basis_at(z: np.ndarray, dr0: np.ndarray, K: int, taps: int, scale: float, n_pupil: int = 32,
                  n_fft: int = 64):
    """Channel basis: the dictionary of the same draws seen at phase scale s -> SVD."""
    return psf.make_basis(z, dr0, K, taps, pupil_samples(n_pupil, scale), n_fft, phase_scale=scale)


def simulate_spectral(x: np.ndarray, seed: int, d_over_r0: float, bases, layers, scales, p: fields.CorrParams,
                      taps: tuple[int, int], kap: float | None = None, form: str = "gather"):
    """y [H, W, 3]: one field draw and one warp, then channel c blurred with basis bases[c] and
    coefficients beta_c = MLP(alpha_hi * scales[c]) (layers[c] if a list of three networks)."""
    h, w, c = x.shape
    assert c == 3 and len(bases) == 3 and len(scales) == 3
    L = noll.cholesky_lower(noll.noll_cov(36))
    if kap is None:
        kap = warp.kappa()
    aa = fields.alpha_anchors(seed, d_over_r0, h, w, p, L)
    ap = fields.alpha_pixels(aa, h, w, p.anchor_spacing)
    xw = warp.warp(np.asarray(x, dtype=np.float64), ap, kap)
    hi = ap[..., 2:]
    per_channel = isinstance(layers[0], list)
    y = np.zeros((h, w, 3))
    fn = blur.scatter if form == "scatter" else blur.gather
    for ch in range(3):
        lay = layers[ch] if per_channel else layers
        beta = mlp.forward(hi * scales[ch], lay)
        y[..., ch : ch + 1] = fn(xw[..., ch : ch + 1], beta, bases[ch], taps[0], taps[1])
    return y
