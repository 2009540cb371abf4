"""Round-to-nearest-even emulation of BF16 and FP8-E4M3 storage.

Used only to predict the error of the reduced-precision GPU variants before
and while they are measured against the FP64 oracle; the parity tests always
compare with the unrounded oracle.  Written from the IEEE-style definitions:
BF16 keeps 8 significand bits of FP32; E4M3 has a 4-bit exponent (bias 7),
3 fraction bits, subnormals down to 2^-9, largest finite 448, no infinities.

Pins (tests/test_oracle_precision.py): exact values at representable points,
ties to even, saturation and the subnormal spacing.
"""
from __future__ import annotations

import numpy as np


def bf16(a) -> np.ndarray:
    """FP64/FP32 -> nearest FP32 -> nearest-even BF16, returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def e4m3(a) -> np.ndarray:
    """Nearest-even FP8 E4M3 value of a (saturating at +-448), as float64."""
    x = np.asarray(a, dtype=np.float64)
    ax = np.abs(x)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    e = np.clip(e, -6, 8)
    q = 2.0 ** (e - 3)
    r = np.rint(ax / q) * q
    r = np.minimum(r, 448.0)
    return np.sign(x) * r
