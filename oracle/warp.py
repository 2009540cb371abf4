"""Tilt modes as a sub-pixel backward warp (Sec. 2.2 and Sec. 3.3).

The P2S transform uses the first two Zernike coefficients (tilts) to displace
the pixels (Sec. 3.3, Fig. 8); the collapsed model applies the tilts as a
local shift of the image (Sec. 2.2).  The paper gives no tilt-to-pixel
conversion; this reading follows Eq. 2 itself.  With image pixels equal to
PSF samples of an N_fft-point DFT over an N_p-sample pupil (radius N_p / 2),
the phase ramp alpha_2 Z_2 = alpha_2 * 2 x / (N_p / 2) moves the PSF of
|DFT(W exp(-j phi))|^2 by kappa alpha_2 samples along +x (columns), with

    kappa = -(2 / pi) (N_fft / N_p)        (-4/pi at 2x zero padding),

and alpha_3 likewise along +y (rows).  A point at p therefore images at
p + d(p), d = kappa (alpha_3, alpha_2) in (row, column), and the warped frame
is the backward sample x_w(p) = x(p - d(p)), bilinear, with coordinates
clamped to the image edge.

Pins (tests/test_oracle_warp.py): kappa against the oracle PSF (an integer
tilt is an exact roll of the PSF), integer shift = array shift, half-pixel
shift = neighbour mean, zero field = identity.
"""
from __future__ import annotations

from math import pi

import numpy as np


def kappa(n_fft: int = 64, n_pupil: int = 32) -> float:
    return -(2.0 / pi) * (n_fft / n_pupil)


def displacement(alpha_pix: np.ndarray, kap: float) -> tuple[np.ndarray, np.ndarray]:
    """(d_row, d_col) in pixels from per-pixel coefficients [.., 35] (J = 2..36)."""
    return kap * alpha_pix[..., 1], kap * alpha_pix[..., 0]


def bilinear_backward(x: np.ndarray, d_row: np.ndarray, d_col: np.ndarray) -> np.ndarray:
    """x_w[i, j] = x(i - d_row[i, j], j - d_col[i, j]), bilinear, clamp to edge.

    x is [H, W, C].  The source coordinate is split as integer pixel index plus
    a shift, never formed as one large floating-point coordinate.
    """
    h, w = x.shape[:2]
    ii, jj = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    ty = -np.asarray(d_row, dtype=np.float64)
    tx = -np.asarray(d_col, dtype=np.float64)
    fy = np.floor(ty)
    fx = np.floor(tx)
    wy = ty - fy
    wx = tx - fx
    y0 = ii + fy.astype(np.int64)
    x0 = jj + fx.astype(np.int64)
    y1, x1 = y0 + 1, x0 + 1
    y0c, y1c = np.clip(y0, 0, h - 1), np.clip(y1, 0, h - 1)
    x0c, x1c = np.clip(x0, 0, w - 1), np.clip(x1, 0, w - 1)
    xd = x.astype(np.float64)
    wy = wy[..., None]
    wx = wx[..., None]
    top = (1 - wx) * xd[y0c, x0c] + wx * xd[y0c, x1c]
    bot = (1 - wx) * xd[y1c, x0c] + wx * xd[y1c, x1c]
    return (1 - wy) * top + wy * bot


def warp(x: np.ndarray, alpha_pix: np.ndarray, kap: float) -> np.ndarray:
    dr, dc = displacement(alpha_pix, kap)
    return bilinear_backward(x, dr, dc)
