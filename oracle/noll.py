"""Noll inter-mode covariance R_Z of Kolmogorov Zernike coefficients (Sec. 2.2).

The paper draws alpha ~ N(0, R_Z) with R_Z taken from Noll (1976) and scaled
by (D/r0)^(5/3) (Sec. 2.2 and Sec. 3.2); the matrix itself is not printed.
This is the published closed form, in units of (D/r0)^(5/3):

  E[a_i a_j] = K_c (-1)^((n_i + n_j - 2m)/2) sqrt((n_i+1)(n_j+1))
               Gamma((n_i + n_j - 5/3)/2)
             / [Gamma((n_i - n_j + 17/3)/2) Gamma((n_j - n_i + 17/3)/2)
                Gamma((n_i + n_j + 23/3)/2)]

  K_c = Gamma(14/3) ((24/5) Gamma(6/5))^(5/6) Gamma(11/6)^2 / (2 pi^2)

non-zero only when m_i = m_j and (m = 0 or i - j even).  Summed over all modes
j >= 2 the diagonal tends to 1.0433, about 1.3 % above Noll's tabulated
1.0299; the offset is a common factor (absorbed into D/r0) and the tests pin
the ratios of Noll's residual-error table, in which it cancels.

Pins (tests/test_oracle_noll.py): Noll's residual table Delta_J / Delta_1,
symmetry, positive definiteness, the zero pattern.
"""
from __future__ import annotations

from math import gamma, pi, sqrt

import numpy as np
from scipy.special import gammaln, gammasgn

from .zernike import noll_to_nm

K_C = gamma(14.0 / 3.0) * ((24.0 / 5.0) * gamma(6.0 / 5.0)) ** (5.0 / 6.0) * gamma(11.0 / 6.0) ** 2 / (2.0 * pi**2)


def _order_term(ni: int, nj: int) -> float:
    """The Gamma-function ratio of the closed form, via log|Gamma| and signs."""
    a = (ni + nj - 5.0 / 3.0) / 2.0
    b = (ni - nj + 17.0 / 3.0) / 2.0
    c = (nj - ni + 17.0 / 3.0) / 2.0
    d = (ni + nj + 23.0 / 3.0) / 2.0
    sgn = gammasgn(a) * gammasgn(b) * gammasgn(c) * gammasgn(d)
    return float(sgn * np.exp(gammaln(a) - gammaln(b) - gammaln(c) - gammaln(d)))


def noll_cov_entry(i: int, j: int) -> float:
    """E[a_i a_j] at D/r0 = 1 for Noll indices i, j >= 2."""
    ni, mi = noll_to_nm(i)
    nj, mj = noll_to_nm(j)
    if mi != mj:
        return 0.0
    if mi != 0 and (i - j) % 2 != 0:
        return 0.0
    sign = (-1) ** ((ni + nj - 2 * mi) // 2)
    return K_C * sign * sqrt((ni + 1) * (nj + 1)) * _order_term(ni, nj)


def noll_cov(j_max: int = 36) -> np.ndarray:
    """R_Z for modes J = 2..j_max as a (j_max-1) x (j_max-1) FP64 matrix."""
    idx = range(2, j_max + 1)
    return np.array([[noll_cov_entry(i, j) for j in idx] for i in idx], dtype=np.float64)


def order_variance(n: int) -> float:
    """Per-mode variance of every mode of radial order n >= 1 (D/r0 = 1)."""
    return K_C * (n + 1) * _order_term(n, n)


def residual(J: int, n_max: int = 20000) -> float:
    """Noll's residual phase variance Delta_J = sum_{j > J} E[a_j^2] (D/r0 = 1).

    Orders beyond n_max are summed by the asymptotic tail
    (n+1) var(n) ~ c n^(-8/3), whose integral from n_max is c n^(-5/3) * 3/5.
    """
    total = 0.0
    for n in range(1, n_max + 1):
        total += (n + 1) * order_variance(n)
    c = (n_max + 1) * order_variance(n_max) * n_max ** (8.0 / 3.0)
    total += c * 0.6 * n_max ** (-5.0 / 3.0)
    head = sum(noll_cov_entry(j, j) for j in range(2, J + 1))
    return total - head


def cholesky_lower(R: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor L with L L^T = R (LAPACK via NumPy)."""
    return np.linalg.cholesky(R)
