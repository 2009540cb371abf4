"""Spatially and inter-mode correlated Zernike fields on an anchor grid (Sec. 3.4).

The paper partitions the image into a grid of anchor points (e.g. 64 x 64),
draws one correlated Zernike vector per anchor and interpolates the
coefficients bilinearly to every pixel (Sec. 3.4); the tilts are drawn by
colouring an i.i.d. Gaussian vector (Sec. 3.2, Fig. 7) and every vector has
the Noll covariance R_Z scaled by (D/r0)^(5/3) (Sec. 2.2).  The angle-of-
arrival correlation formulas it uses (Takato, Chanan, Basu) and the optical
parameters are not printed, so the spatial correlation is the following
stated reading, produced by Fourier-domain filtering of white noise:

  anchors    at pixel coordinates (a_y s, a_x s), a grid of
             A = floor((H-1)/s) + 2 by floor((W-1)/s) + 2 points;
  torus      F_h x F_w, each the next power of two >= A + guard,
             guard = ceil(3 * max(ell) / s) unless given;
  kernel     c[d] = sum over periodic images of exp(-|d|^2 s^2 / (2 ell^2)),
             a Gaussian covariance of length ell pixels wrapped on the torus;
             one shared kernel, or one per radial order n = 1..7;
  filter     f = Re IDFT2( sqrt(max(DFT2(c), 0)) * DFT2(w) ), cropped to the
             A_h x A_w corner; w is unit white noise of stream (seed, mode);
  colouring  alpha(a) = (D/r0)^(5/6) L f(a), L = chol(R_Z[2..36]), where the
             l-th white field uses the kernel of mode l's radial order.

So Cov(alpha_i(a), alpha_j(a + d)) = (D/r0)^(5/3) sum_l L_il L_jl c_n(l)[d]
exactly, and with one shared kernel it is (D/r0)^(5/3) R_Z[i, j] c[d].

Pins (tests/test_oracle_fields.py): the exact covariance identity, the
sample covariance of many seeds against it, the bilinear covariance formula.
Parity with the physical Takato correlation is not attempted (not printed).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import ceil

import numpy as np

from . import noll, philox
from .zernike import radial_order

N_MODES = 35  # Noll J = 2..36
J_MIN, J_MAX = 2, 36


@dataclass
class CorrParams:
    anchor_spacing: int = 8
    corr_len_px: tuple = (16.0,)  # one shared kernel, or 7 (radial orders 1..7)
    fft_guard: int | None = None

    def guard(self) -> int:
        if self.fft_guard is not None:
            return int(self.fft_guard)
        return int(ceil(3.0 * max(self.corr_len_px) / self.anchor_spacing))

    def kernel_of_mode(self, j: int) -> int:
        if len(self.corr_len_px) == 1:
            return 0
        return radial_order(j) - 1


def next_pow2(v: int) -> int:
    p = 1
    while p < v:
        p *= 2
    return p


def anchor_shape(h: int, w: int, s: int) -> tuple[int, int]:
    return (h - 1) // s + 2, (w - 1) // s + 2


def torus_shape(h: int, w: int, p: CorrParams) -> tuple[int, int]:
    ah, aw = anchor_shape(h, w, p.anchor_spacing)
    g = p.guard()
    return next_pow2(ah + g), next_pow2(aw + g)


def kernel_covariance(fh: int, fw: int, ell: float, s: int) -> np.ndarray:
    """c[dy, dx]: Gaussian covariance of length ell px wrapped on an fh x fw torus of anchors."""
    out = np.zeros((fh, fw), dtype=np.float64)
    dy = np.arange(fh, dtype=np.float64)[:, None]
    dx = np.arange(fw, dtype=np.float64)[None, :]
    my = int(ceil(40.0 * ell / (s * fh))) + 1
    mx = int(ceil(40.0 * ell / (s * fw))) + 1
    for m in range(-my, my + 1):
        for n in range(-mx, mx + 1):
            d2 = (dy + m * fh) ** 2 + (dx + n * fw) ** 2
            out += np.exp(-d2 * (s * s) / (2.0 * ell * ell))
    return out


def filter_gain(fh: int, fw: int, ell: float, s: int) -> np.ndarray:
    """sqrt(max(DFT2(c), 0)): the real, non-negative frequency response of the filter."""
    C = np.real(np.fft.fft2(kernel_covariance(fh, fw, ell, s)))
    return np.sqrt(np.maximum(C, 0.0))


def white_noise(seed: int, mode_index: int, fh: int, fw: int) -> np.ndarray:
    """Unit white noise of stream (seed, mode_index) on the torus, row-major."""
    return philox.normals(seed, mode_index, fh * fw).reshape(fh, fw)


def filter_field(wn: np.ndarray, gain: np.ndarray) -> np.ndarray:
    """f = Re IDFT2(gain * DFT2(wn)) on the whole torus."""
    return np.real(np.fft.ifft2(gain * np.fft.fft2(wn)))


def filtered_fields(seed: int, h: int, w: int, p: CorrParams) -> np.ndarray:
    """The 35 spatially correlated unit-variance fields f_l on the anchors: [A_h, A_w, 35]."""
    ah, aw = anchor_shape(h, w, p.anchor_spacing)
    fh, fw = torus_shape(h, w, p)
    gains = [filter_gain(fh, fw, ell, p.anchor_spacing) for ell in p.corr_len_px]
    out = np.empty((ah, aw, N_MODES), dtype=np.float64)
    for l in range(N_MODES):
        j = l + J_MIN
        g = gains[p.kernel_of_mode(j)]
        f = filter_field(white_noise(seed, l, fh, fw), g)
        out[:, :, l] = f[:ah, :aw]
    return out


def gaussian_corr_1d(n: int, ell: float, s: int) -> np.ndarray:
    """C[i, k] = exp(-((i - k) s)^2 / (2 ell^2)) over n anchors along one axis (not wrapped)."""
    d = (np.arange(n)[:, None] - np.arange(n)[None, :]) * float(s)
    return np.exp(-d * d / (2.0 * ell * ell))


def dense_fields(seed: int, h: int, w: int, p: CorrParams) -> np.ndarray:
    """The 35 unit-variance fields drawn directly from the anchors' correlation matrix (the
    paper's dense anchor draw, Sec. 3.4): f_l = chol(Sigma) w_l over the A_h A_w anchors, with
    Sigma[(a_y, a_x), (b_y, b_x)] = exp(-|a - b|^2 s^2 / (2 ell^2)) unwrapped.  That Gaussian
    matrix is the Kronecker product C_y (x) C_x, whose Cholesky factor is L_y (x) L_x, so the
    draw is evaluated as L_y W L_x^T with W the A_h x A_w white noise of stream (seed, mode),
    samples taken row-major over the anchors.  [A_h, A_w, 35]."""
    ah, aw = anchor_shape(h, w, p.anchor_spacing)
    out = np.empty((ah, aw, N_MODES), dtype=np.float64)
    Ls = {}
    for l in range(N_MODES):
        kk = p.kernel_of_mode(l + J_MIN)
        if kk not in Ls:
            ell = p.corr_len_px[kk]
            Ls[kk] = (np.linalg.cholesky(gaussian_corr_1d(ah, ell, p.anchor_spacing)),
                      np.linalg.cholesky(gaussian_corr_1d(aw, ell, p.anchor_spacing)))
        Ly, Lx = Ls[kk]
        wn = philox.normals(seed, l, ah * aw).reshape(ah, aw)
        out[:, :, l] = Ly @ wn @ Lx.T
    return out


def colour(f: np.ndarray, d_over_r0: float, L: np.ndarray) -> np.ndarray:
    """alpha(a) = (D/r0)^(5/6) L f(a) for every anchor a."""
    return (float(d_over_r0) ** (5.0 / 6.0)) * np.einsum("jl,...l->...j", L, f)


def alpha_anchors(seed: int, d_over_r0: float, h: int, w: int, p: CorrParams, L: np.ndarray | None = None,
                  method: str = "fft") -> np.ndarray:
    """Zernike coefficients J = 2..36 on the anchor grid: [A_h, A_w, 35].
    method "fft": Fourier filtering on the torus; "dense": the direct draw of dense_fields."""
    if L is None:
        L = noll.cholesky_lower(noll.noll_cov(J_MAX))
    f = filtered_fields(seed, h, w, p) if method == "fft" else dense_fields(seed, h, w, p)
    return colour(f, d_over_r0, L)


def alpha_pixels(alpha_a: np.ndarray, h: int, w: int, s: int) -> np.ndarray:
    """Bilinear interpolation of anchor coefficients to every pixel: [h, w, n].

    Pixel (i, j) lies in anchor cell (i // s, j // s) at fractional offsets
    ((i % s) / s, (j % s) / s).
    """
    i = np.arange(h)
    j = np.arange(w)
    ay, fy = i // s, (i % s) / s
    ax, fx = j // s, (j % s) / s
    a00 = alpha_a[ay][:, ax]
    a01 = alpha_a[ay][:, ax + 1]
    a10 = alpha_a[ay + 1][:, ax]
    a11 = alpha_a[ay + 1][:, ax + 1]
    wy = fy[:, None, None]
    wx = fx[None, :, None]
    return (1 - wy) * ((1 - wx) * a00 + wx * a01) + wy * ((1 - wx) * a10 + wx * a11)


def anchor_cross_covariance(d: tuple[int, int], fh: int, fw: int, p: CorrParams, L: np.ndarray, d_over_r0: float) -> np.ndarray:
    """Cov(alpha_i(a), alpha_j(a + d)) predicted by the construction, [35, 35]."""
    s = p.anchor_spacing
    cd = []
    for ell in p.corr_len_px:
        g = filter_gain(fh, fw, ell, s)
        c_eff = np.real(np.fft.ifft2(g * g))  # circular autocorrelation of the filter
        cd.append(c_eff[d[0] % fh, d[1] % fw])
    kern = np.array([cd[p.kernel_of_mode(l + J_MIN)] for l in range(N_MODES)])
    return (d_over_r0 ** (5.0 / 3.0)) * (L * kern[None, :]) @ L.T
