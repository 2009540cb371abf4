"""P2S network forward pass (Sec. 3.3, Fig. 8).

The phase-to-space network maps each pixel's higher-order Zernike vector to
its basis weights beta through three fully connected layers, evaluated per
pixel (Sec. 3.3).  Widths and activations were only in Fig. 8, which is not in
the text; the reading is: input alpha_{4..36} (33 values, radians, no
normalisation), ReLU after the first two layers, linear output, biases on.

Pin (tests/test_oracle_mlp.py): identity weights reproduce the input; a
single-layer network equals the affine map written element by element.
"""
from __future__ import annotations

import numpy as np


def forward(v: np.ndarray, layers) -> np.ndarray:
    """v [..., d0] -> [..., d_last]; layers = [(W [out, in], b [out]), ...]."""
    h = np.asarray(v, dtype=np.float64)
    for i, (W, b) in enumerate(layers):
        h = h @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        if i + 1 < len(layers):
            h = np.maximum(h, 0.0)
    return h
