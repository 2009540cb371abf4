"""Noll-indexed Zernike polynomials on the unit disk (Sec. 2.2, Eq. 1).

The paper expands the aperture phase as phi(rho) = sum_j alpha_j Z_j(rho) and
names alpha_2, alpha_3 the horizontal and vertical tilts, which fixes Noll's
(1976) single-index ordering.  Normalisation is Noll's: (1/pi) * integral over
the unit disk of Z_i Z_j = delta_ij.  The angle theta is measured from the +x
(column index increasing) axis towards +y (row index increasing).

Pins (tests/test_oracle_zernike.py): orthonormality by exact polar quadrature;
the first modes against their textbook closed forms.
"""
from __future__ import annotations

from math import factorial, sqrt

import numpy as np


def noll_to_nm(j: int) -> tuple[int, int]:
    """Radial order n and azimuthal frequency m >= 0 of Noll mode j >= 1.

    Within radial order n the modes run by increasing m; every m > 0 appears
    twice (even j: cosine, odd j: sine).
    """
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    k = j - n * (n + 1) // 2 - 1  # position inside order n
    if n % 2 == 0:
        m = 2 * ((k + 1) // 2)
    else:
        m = 2 * (k // 2) + 1
    return n, m


def radial(n: int, m: int, r: np.ndarray) -> np.ndarray:
    """Zernike radial polynomial R_n^m(r) as the finite alternating sum."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    for s in range((n - m) // 2 + 1):
        c = (-1) ** s * factorial(n - s) / (
            factorial(s) * factorial((n + m) // 2 - s) * factorial((n - m) // 2 - s)
        )
        out = out + c * r ** (n - 2 * s)
    return out


def zernike(j: int, r: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Z_j(r, theta), Noll normalisation (unit mean square on the disk)."""
    n, m = noll_to_nm(j)
    R = radial(n, m, r)
    if m == 0:
        return sqrt(n + 1) * R
    if j % 2 == 0:
        return sqrt(2 * (n + 1)) * R * np.cos(m * theta)
    return sqrt(2 * (n + 1)) * R * np.sin(m * theta)


def radial_order(j: int) -> int:
    return noll_to_nm(j)[0]
