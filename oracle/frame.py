"""One synthesised frame, step by step (Sec. 3, Fig. 3 and Fig. 8).

Order of the path: anchor fields (Sec. 3.4) -> per-pixel coefficients by
bilinear interpolation -> tilt warp of the input (Sec. 3.3) -> P2S network on
alpha_{4..36} -> basis blur (Eq. 5, scatter or gather form).

`emulate` rounds the tensors the BF16 GPU variant stores in BF16 (network
input, weights and activations, beta, the basis) so that the expected size of
its error can be read off before the kernels run; it is never the reference
a parity test compares against.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import blur, fields, mlp, noll, psf, warp
from .precision import bf16


@dataclass
class Stages:
    alpha_anchor: np.ndarray  # [A_h, A_w, 35]  J = 2..36
    alpha_pix: np.ndarray  # [H, W, 35]
    xw: np.ndarray  # [H, W, C]
    beta: np.ndarray  # [H, W, K]
    y: np.ndarray  # [H, W, C]


def _round_layers(layers, rnd):
    return [(rnd(W), b) for W, b in layers]


def mlp_emulated(v, layers, rnd):
    h = rnd(v)
    for i, (W, b) in enumerate(layers):
        h = h @ rnd(W).T + b
        if i + 1 < len(layers):
            h = rnd(np.maximum(h, 0.0))
    return h


def simulate(x: np.ndarray, seed: int, d_over_r0: float, Hb: np.ndarray, layers, p: fields.CorrParams,
             taps: tuple[int, int], kap: float | None = None, form: str = "scatter", emulate: str | None = None,
             L: np.ndarray | None = None, order: str = "warp_blur", field_method: str = "fft") -> Stages:
    """The full path on one frame x [H, W, C] (float), FP64 throughout unless `emulate`.

    order "warp_blur": y = blur(warp(x)), the simulator's default; "blur_warp": y = warp(blur(x)),
    the collapsed model's order of Sec. 2.2 (the blurred image shifted by the tilts).  In the
    second case Stages.xw holds the unwarped input."""
    h, w = x.shape[:2]
    if L is None:
        L = noll.cholesky_lower(noll.noll_cov(36))
    if kap is None:
        kap = warp.kappa()
    aa = fields.alpha_anchors(seed, d_over_r0, h, w, p, L, method=field_method)
    ap = fields.alpha_pixels(aa, h, w, p.anchor_spacing)
    if order not in ("warp_blur", "blur_warp"):
        raise ValueError(order)
    xw = warp.warp(x, ap, kap) if order == "warp_blur" else x
    hi = ap[..., 2:]
    if emulate == "bf16":
        beta = bf16(mlp_emulated(hi, layers, bf16))
        Hb_used = bf16(Hb)
    elif emulate is None:
        beta = mlp.forward(hi, layers)
        Hb_used = Hb
    else:
        raise ValueError(emulate)
    fn = blur.scatter if form == "scatter" else blur.gather
    y = fn(xw, beta, Hb_used, taps[0], taps[1])
    if order == "blur_warp":
        y = warp.warp(y, ap, kap)
    return Stages(aa, ap, xw, beta, y)


def exact_frame(x: np.ndarray, seed: int, d_over_r0: float, p: fields.CorrParams, taps: tuple[int, int],
                kap: float | None = None, n_pupil: int = 32, n_fft: int = 64, L: np.ndarray | None = None,
                field_method: str = "fft", form: str = "scatter"):
    """Eq. 3 on a small frame: every pixel's PSF formed by Eq. 2, no basis, no network.

    Same fields and warp as simulate() for the same arguments.  Returns (x_w, per-pixel PSFs
    [H, W, th, tw], y); form "scatter" spreads each source pixel's light with its own PSF,
    "gather" weights each output pixel's neighbourhood with that output pixel's PSF."""
    h, w = x.shape[:2]
    if L is None:
        L = noll.cholesky_lower(noll.noll_cov(36))
    if kap is None:
        kap = warp.kappa(n_fft, n_pupil)
    aa = fields.alpha_anchors(seed, d_over_r0, h, w, p, L, method=field_method)
    ap = fields.alpha_pixels(aa, h, w, p.anchor_spacing)
    xw = warp.warp(x, ap, kap)
    hp = psf.psf_taps(ap[..., 2:], taps[0], taps[1], n_pupil, n_fft)
    fn = blur.exact if form == "scatter" else blur.exact_gather
    return xw, hp, fn(xw, hp)


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - ref) / max(np.linalg.norm(ref), 1e-300))
