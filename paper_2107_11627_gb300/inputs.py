"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the simulator itself: it only draws the
images, turbulence strengths, Philox seeds, network weights and dictionary
draws that both sides take as inputs.  Every generator is a NumPy PCG64 stream
keyed by an explicit seed, so a test, the benchmark and the oracle see the
same arrays.

Stand-in data.  The paper times 256x256 frames (Sec. 4.4, Table 2) and
synthesises training data from Places images with D/r0 ~ U[1, 8] (Sec. 4.3);
those datasets are not available, so smooth random "blob" images of the same
frame sizes stand in for natural images.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "blob_image",
    "block_image",
    "blob_batch",
    "frame_seeds",
    "frame_strengths",
    "mlp_weights",
    "dictionary_draws",
    "uneven_sizes",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def blob_image(h: int, w: int, c: int = 3, seed: int = 1000) -> np.ndarray:
    """Sum of 50 isotropic Gaussian blobs plus uniform noise of std 0.02.

    Centres are uniform in the frame, sigma ~ U[2%, 15%] of the short side,
    per-channel amplitudes ~ U[0, 1].  The sum is divided by its maximum and
    uniform noise on [-0.0346, 0.0346] (std 0.02) is added; no clipping.
    Returns float32 HWC.
    """
    rng = _rng(seed)
    short = min(h, w)
    cy = rng.uniform(0.0, h, size=50)
    cx = rng.uniform(0.0, w, size=50)
    sig = rng.uniform(0.02, 0.15, size=50) * short
    amp = rng.uniform(0.0, 1.0, size=(50, c))
    yy = np.arange(h, dtype=np.float64)[:, None]
    xx = np.arange(w, dtype=np.float64)[None, :]
    img = np.zeros((h, w, c), dtype=np.float64)
    for i in range(50):
        g = np.exp(-((yy - cy[i]) ** 2 + (xx - cx[i]) ** 2) / (2.0 * sig[i] ** 2))
        img += g[:, :, None] * amp[i][None, None, :]
    img /= img.max()
    a = 0.02 * np.sqrt(3.0)
    img += rng.uniform(-a, a, size=img.shape)
    return img.astype(np.float32)


def block_image(h: int = 64, w: int = 64, block: int = 8, c: int = 1, seed: int = 1000) -> np.ndarray:
    """Piecewise-constant image of block x block tiles, each tile ~ U[0, 1]."""
    rng = _rng(seed)
    nby, nbx = -(-h // block), -(-w // block)
    vals = rng.uniform(0.0, 1.0, size=(nby, nbx, c))
    img = np.repeat(np.repeat(vals, block, axis=0), block, axis=1)[:h, :w]
    return np.ascontiguousarray(img.astype(np.float32))


def blob_batch(n: int, h: int, w: int, c: int = 3, first_seed: int = 1000) -> np.ndarray:
    """n blob images, frame i seeded with first_seed + i.  float32 NHWC."""
    return np.stack([blob_image(h, w, c, first_seed + i) for i in range(n)])


def frame_seeds(n: int, first: int = 10**6) -> np.ndarray:
    """Per-frame Philox keys: first + frame index (uint64)."""
    return (np.uint64(first) + np.arange(n, dtype=np.uint64)).astype(np.uint64)


def frame_strengths(n: int, lo: float, hi: float, seed: int = 7) -> np.ndarray:
    """Per-frame D/r0 ~ U[lo, hi] (float32, the precision the path consumes)."""
    return _rng(seed).uniform(lo, hi, size=n).astype(np.float32)


def mlp_weights(dims, seed: int = 42):
    """Random-init fully connected weights, W_l ~ U(+-1/sqrt(fan_in)), b_l likewise.

    dims = [33, 128, 128, 100] gives three layers.  Returns a list of
    (W [out, in], b [out]) float64 pairs.  No trained weights exist for this
    build, so both sides take these seeded draws.
    """
    rng = _rng(seed)
    layers = []
    for fi, fo in zip(dims[:-1], dims[1:]):
        bound = 1.0 / np.sqrt(fi)
        W = rng.uniform(-bound, bound, size=(fo, fi))
        b = rng.uniform(-bound, bound, size=fo)
        layers.append((W, b))
    return layers


def dictionary_draws(n_dict: int, n_modes: int = 35, dr0_range=(0.5, 6.0), seed: int = 2021):
    """Standard-normal Zernike draws and turbulence strengths for a PSF dictionary.

    Returns (z [n_dict, n_modes] float64 ~ N(0, 1), dr0 [n_dict] ~ U[dr0_range]).
    The dictionary step colours z with the Noll covariance itself.
    """
    rng = _rng(seed)
    dr0 = rng.uniform(dr0_range[0], dr0_range[1], size=n_dict)
    z = rng.standard_normal(size=(n_dict, n_modes))
    return z, dr0


def uneven_sizes(n: int, seed: int = 96):
    """Frame sizes for a mixed-resolution batch.

    Long side L uniform over {128, 256, 384, 512, 768, 1024}; aspect a ~ U[1, 16/9];
    short side round(L / a / 8) * 8; landscape or portrait with equal odds.
    Returns a list of (H, W).
    """
    rng = _rng(seed)
    longs = rng.choice([128, 256, 384, 512, 768, 1024], size=n)
    aspect = rng.uniform(1.0, 16.0 / 9.0, size=n)
    land = rng.uniform(size=n) < 0.5
    out = []
    for L, a, ls in zip(longs, aspect, land):
        s = int(round(L / a / 8.0)) * 8
        out.append((int(s), int(L)) if ls else (int(L), int(s)))
    return out
