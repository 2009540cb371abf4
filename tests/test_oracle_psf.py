"""Pins of oracle.psf: direct DFT, Airy pattern, Parseval, SVD basis."""
import numpy as np
from scipy.special import j1

from oracle import psf


def test_fft_psf_equals_direct_dft():
    n_p, n_f = 8, 16
    rng = np.random.default_rng(6)
    alpha = rng.normal(size=33) * 0.5
    h = psf.psf_full(alpha, psf.HIGH_ORDER, n_p, n_f)
    _, _, mask = psf.pupil_grid(n_p)
    phi = np.tensordot(alpha, psf.zernike_stack(psf.HIGH_ORDER, n_p), axes=1)
    P = mask * np.exp(-1j * phi)
    X = np.zeros((n_f, n_f), dtype=complex)
    for k in range(n_f):
        for l in range(n_f):
            for v in range(n_p):
                for u in range(n_p):
                    X[k, l] += P[v, u] * np.exp(-2j * np.pi * (k * v + l * u) / n_f)
    ref = np.fft.fftshift(np.abs(X) ** 2)
    assert np.max(np.abs(h - ref)) < 1e-12 * ref.max()


def test_zero_phase_approaches_airy():
    errs = []
    for n_p in (32, 64, 128):
        h = psf.psf_full(np.zeros(1), [4], n_p, 2 * n_p)
        c = n_p
        row = h[c, c - 6 : c + 7] / h[c, c]
        k = np.arange(-6, 7)
        v = np.pi * k / 2.0
        with np.errstate(invalid="ignore", divide="ignore"):
            airy = np.where(k == 0, 1.0, (2 * j1(v) / v) ** 2)
        errs.append(np.max(np.abs(row - airy)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02


def test_parseval_energy_independent_of_phase():
    n_p, n_f = 32, 64
    _, _, mask = psf.pupil_grid(n_p)
    rng = np.random.default_rng(7)
    for scale in (0.0, 0.5, 3.0):
        h = psf.psf_full(scale * rng.normal(size=33), psf.HIGH_ORDER, n_p, n_f)
        assert abs(h.sum() / (n_f**2 * mask.sum()) - 1) < 1e-12


def test_basis_orthonormal_and_projection():
    rng = np.random.default_rng(8)
    z = rng.normal(size=(300, 35))
    dr0 = rng.uniform(0.5, 6, size=300)
    H, D = psf.make_basis(z, dr0, K=20, taps=9)
    assert np.allclose(H @ H.T, np.eye(20), atol=1e-12)
    assert np.all(H.sum(axis=1) >= 0)
    res = D - (D @ H.T) @ H
    assert np.max(np.abs(res @ H.T)) < 1e-12
    assert np.allclose(D.sum(axis=1), 1.0)
    # the leading singular vector carries most of the dictionary's energy
    assert np.linalg.norm(D @ H[0]) ** 2 / np.linalg.norm(D) ** 2 > 0.5
