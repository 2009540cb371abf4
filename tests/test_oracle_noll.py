"""Pins of oracle.noll against Noll (1976), Table IV (residual phase variance Delta_J).

The closed form's total variance differs from Noll's numerically integrated
values by a common factor (1.0433 vs 1.0299); the ratios Delta_J / Delta_1
cancel it and are compared at the table's three significant digits.
"""
import os

import numpy as np
import pytest

from oracle import noll
from oracle.zernike import noll_to_nm

_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "noll_1976_table4.txt")
NOLL_TABLE = {int(a): float(b) for a, b in (ln.split() for ln in open(_GOLDEN) if ln.strip() and not ln.startswith("#"))}


@pytest.fixture(scope="module")
def delta1():
    return noll.residual(1)


@pytest.mark.parametrize("J", [2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 21])
def test_residual_ratios(J, delta1):
    ours = noll.residual(J) / delta1
    table = NOLL_TABLE[J] / NOLL_TABLE[1]
    assert abs(ours / table - 1.0) < 4e-3


def test_common_offset(delta1):
    # the uniform factor between the closed form and the table, recorded as a reading
    assert 1.010 < delta1 / NOLL_TABLE[1] < 1.016


def test_matrix_properties():
    R = noll.noll_cov(36)
    assert R.shape == (35, 35)
    assert np.allclose(R, R.T, atol=0)
    ev = np.linalg.eigvalsh(R)
    assert ev.min() > 1e-4
    for a in range(35):
        for b in range(35):
            i, j = a + 2, b + 2
            (ni, mi), (nj, mj) = noll_to_nm(i), noll_to_nm(j)
            allowed = mi == mj and (mi == 0 or (i - j) % 2 == 0)
            if not allowed:
                assert R[a, b] == 0.0
            else:
                assert R[a, b] != 0.0
    # tilt-coma anticorrelation (n = 1 with n = 3, same m and parity)
    assert R[0, 6] < 0 and R[1, 5] < 0


def test_cholesky_reconstructs():
    R = noll.noll_cov(36)
    L = noll.cholesky_lower(R)
    assert np.allclose(L @ L.T, R, atol=1e-15)
    assert np.allclose(L, np.tril(L))
