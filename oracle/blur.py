"""Spatially varying blur through a PSF basis (Sec. 3.1, Eq. 3-5).

Eq. 3 writes the turbulent image as y = H x with one PSF per pixel; Eq. 4
expands each PSF in a basis, h_n = sum_m beta_{m,n} phi_m; Eq. 5 then forms
y_n = sum_m beta_{m,n} phi_m^T x, where the weights belong to the OUTPUT pixel
(gather form).  The simulator's contract instead spreads each SOURCE pixel's
light with its own PSF (scatter form), y = sum_k h_k * (beta_k . x_w).  Both
are stated here, with zero padding outside the image and "same"-size output.

With G[p, t] = sum_k beta[p, k] H[k, t] and tap offset o(t) = (ty - th//2, tx - tw//2):
  scatter  y_c[p + o(t)] += G[p, t] x_c[p]
  gather   y_c[q]        += G[q, t] x_c[q - o(t)]
For constant beta both equal one invariant convolution with sum_k beta_k h_k.

exact() is Eq. 3 itself: every pixel spreads its light with its own PSF;
exact_gather() is its row form, every output pixel weighting its
neighbourhood with its own PSF (what Eq. 5 approximates).

Pins (tests/test_oracle_blur.py): constant beta against scipy.signal's
convolution, a single basis vector, a delta image, the adjoint identity
between scatter and gather, the exact blur against the basis form with the
projected beta.
"""
from __future__ import annotations

import numpy as np


def _shift_add(dst: np.ndarray, src: np.ndarray, dy: int, dx: int) -> None:
    """dst[i + dy, j + dx] += src[i, j] where both are inside the frame."""
    h, w = src.shape[:2]
    ys, ye = max(0, -dy), min(h, h - dy)
    xs, xe = max(0, -dx), min(w, w - dx)
    if ys >= ye or xs >= xe:
        return
    dst[ys + dy : ye + dy, xs + dx : xe + dx] += src[ys:ye, xs:xe]


def _shifted(src: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """out[i, j] = src[i - dy, j - dx], zero outside."""
    out = np.zeros_like(src)
    _shift_add(out, src, dy, dx)
    return out


def tap_offsets(th: int, tw: int):
    return [(ty - th // 2, tx - tw // 2) for ty in range(th) for tx in range(tw)]


def scatter(xw: np.ndarray, beta: np.ndarray, Hb: np.ndarray, th: int, tw: int, chunk: int = 64) -> np.ndarray:
    """y = sum_k h_k * (beta_k . x_w): each source pixel spreads with its own PSF."""
    h, w, c = xw.shape
    xd = xw.astype(np.float64)
    b2 = beta.reshape(-1, beta.shape[-1]).astype(np.float64)
    y = np.zeros((h, w, c), dtype=np.float64)
    offs = tap_offsets(th, tw)
    for s in range(0, len(offs), chunk):
        G = (b2 @ Hb[:, s : s + chunk].astype(np.float64)).reshape(h, w, -1)
        for i, (dy, dx) in enumerate(offs[s : s + chunk]):
            _shift_add(y, G[:, :, i : i + 1] * xd, dy, dx)
    return y


def gather(xw: np.ndarray, beta: np.ndarray, Hb: np.ndarray, th: int, tw: int, chunk: int = 64) -> np.ndarray:
    """y_q = sum_k beta[q, k] (phi_k^T x)_q (Eq. 5): each output pixel uses its own PSF."""
    h, w, c = xw.shape
    xd = xw.astype(np.float64)
    b2 = beta.reshape(-1, beta.shape[-1]).astype(np.float64)
    y = np.zeros((h, w, c), dtype=np.float64)
    offs = tap_offsets(th, tw)
    for s in range(0, len(offs), chunk):
        G = (b2 @ Hb[:, s : s + chunk].astype(np.float64)).reshape(h, w, -1)
        for i, (dy, dx) in enumerate(offs[s : s + chunk]):
            y += G[:, :, i : i + 1] * _shifted(xd, dy, dx)
    return y


def exact(xw: np.ndarray, psfs: np.ndarray) -> np.ndarray:
    """Eq. 3 by brute force: psfs [H, W, th, tw] is every pixel's own PSF (scatter)."""
    h, w, c = xw.shape
    th, tw = psfs.shape[2:]
    xd = xw.astype(np.float64)
    y = np.zeros((h, w, c), dtype=np.float64)
    for ty in range(th):
        for tx in range(tw):
            _shift_add(y, psfs[:, :, ty, tx][:, :, None] * xd, ty - th // 2, tx - tw // 2)
    return y


def exact_gather(xw: np.ndarray, psfs: np.ndarray) -> np.ndarray:
    """Eq. 3 in row form: y[q] = sum_t psfs[q, t] x[q - o(t)], psfs [H, W, th, tw] per OUTPUT pixel."""
    h, w, c = xw.shape
    th, tw = psfs.shape[2:]
    xd = xw.astype(np.float64)
    y = np.zeros((h, w, c), dtype=np.float64)
    for ty in range(th):
        for tx in range(tw):
            y += psfs[:, :, ty, tx][:, :, None] * _shifted(xd, ty - th // 2, tx - tw // 2)
    return y
