"""Pins of oracle.zernike: orthonormality on the unit disk and textbook closed forms."""
import numpy as np
import pytest

from oracle.zernike import noll_to_nm, zernike


def _disk_quadrature(nr=12, nt=40):
    # Gauss-Legendre in r on [0, 1] (weight r dr) and uniform theta: exact for the
    # polynomial degrees of J <= 36 (radial degree <= 15, angular frequency <= 14).
    x, w = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * (x + 1.0)
    wr = 0.5 * w * r
    t = 2.0 * np.pi * np.arange(nt) / nt
    wt = np.full(nt, 2.0 * np.pi / nt)
    R, T = np.meshgrid(r, t, indexing="ij")
    W = np.outer(wr, wt)
    return R, T, W


def test_orthonormal_on_unit_disk():
    R, T, W = _disk_quadrature()
    Z = np.stack([zernike(j, R, T) for j in range(1, 37)])
    gram = np.einsum("iab,jab,ab->ij", Z, Z, W) / np.pi
    assert np.max(np.abs(gram - np.eye(36))) < 1e-13


@pytest.mark.parametrize("j,nm", [(1, (0, 0)), (2, (1, 1)), (3, (1, 1)), (4, (2, 0)), (5, (2, 2)),
                                  (6, (2, 2)), (7, (3, 1)), (9, (3, 3)), (11, (4, 0)), (14, (4, 4)),
                                  (22, (6, 0)), (36, (7, 7))])
def test_noll_ordering(j, nm):
    assert noll_to_nm(j) == nm


def test_closed_forms():
    # Noll (1976) Table I, written out by hand.
    rng = np.random.default_rng(0)
    r = rng.uniform(0, 1, 50)
    t = rng.uniform(0, 2 * np.pi, 50)
    ref = {
        2: 2 * r * np.cos(t),
        3: 2 * r * np.sin(t),
        4: np.sqrt(3) * (2 * r**2 - 1),
        5: np.sqrt(6) * r**2 * np.sin(2 * t),
        6: np.sqrt(6) * r**2 * np.cos(2 * t),
        7: np.sqrt(8) * (3 * r**3 - 2 * r) * np.sin(t),
        8: np.sqrt(8) * (3 * r**3 - 2 * r) * np.cos(t),
        9: np.sqrt(8) * r**3 * np.sin(3 * t),
        10: np.sqrt(8) * r**3 * np.cos(3 * t),
        11: np.sqrt(5) * (6 * r**4 - 6 * r**2 + 1),
    }
    for j, v in ref.items():
        assert np.allclose(zernike(j, r, t), v, atol=1e-13), j
