"""Pins of oracle.spectral (wavelength-dependent colour, Sec. 3.5)."""
import numpy as np

from oracle import frame, psf, spectral
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs


def test_reference_wavelength_reduces_to_single_wavelength_psf():
    rng = np.random.default_rng(3)
    a = 0.3 * rng.normal(size=(5, 33))
    assert spectral.phase_scale(540.0) == 1.0
    np.testing.assert_array_equal(spectral.psf_taps_at(a, 17, 1.0), psf.psf_taps(a, 17, 17, 32, 64))


def test_diffraction_area_scales_with_wavelength_squared():
    """Zero phase: the peak of the unit-energy PSF is (sum W)^2 / (N_fft^2 sum W) = (pupil
    samples) / N_fft^2 exactly (the peak is |sum W|^2, the energy N_fft^2 sum W^2 by Parseval,
    W^2 = W), so the PSF's area 1 / peak grows as 1 / N_p,c^2 ~ lambda_c^2, the diffraction
    scaling the reading builds in (up to the rounding of N_p,c and the disc's pixelation)."""
    peaks = {}
    for lam in spectral.WAVELENGTHS_NM:
        n_c = spectral.pupil_samples(32, spectral.phase_scale(lam))
        h = psf.psf_full(np.zeros(33), psf.HIGH_ORDER, n_c, 64)
        _, _, mask = psf.pupil_grid(n_c)
        peak = h.max() / h.sum()
        assert abs(peak * 64**2 - mask.sum()) < 1e-9 * mask.sum()
        peaks[lam] = peak
    for lam in spectral.WAVELENGTHS_NM:
        n_c = spectral.pupil_samples(32, spectral.phase_scale(lam))
        assert abs(peaks[540.0] / peaks[lam] - (32.0 / n_c) ** 2) < 0.05 * (32.0 / n_c) ** 2, (lam, peaks)
    assert peaks[450.0] > peaks[540.0] > peaks[570.0]  # blue PSFs are the narrowest


def test_strehl_follows_marechal_with_the_phase_scale():
    """Small aberrations: the peak of the unit-energy PSF relative to the aberration-free one
    is exp(-sigma^2), sigma^2 = s^2 sum_j alpha_j^2 the pupil phase variance (Noll-normalised
    modes are orthonormal over the disk).  Pins both the phase scale and the mode norm."""
    rng = np.random.default_rng(4)
    a = 0.02 * rng.normal(size=33)
    for lam in spectral.WAVELENGTHS_NM:
        s = spectral.phase_scale(lam)
        n_c = spectral.pupil_samples(32, s)
        h0 = psf.psf_full(np.zeros(33), psf.HIGH_ORDER, n_c, 64)
        h = psf.psf_full(a * s, psf.HIGH_ORDER, n_c, 64)
        strehl = h.max() / h0.max()
        var = (s**2) * np.sum(a**2)
        assert abs(strehl - np.exp(-var)) < 0.15 * var, (lam, strehl, np.exp(-var))


def test_spectral_frame_at_reference_equals_single_wavelength_frame():
    rng = np.random.default_rng(6)
    h, w = 20, 24
    T = 9 * 9
    H = np.linalg.qr(rng.normal(size=(T, 12)))[0].T
    layers = inputs.mlp_weights([33, 16, 12], 42)
    x = inputs.blob_image(h, w, 3, 1007).astype(np.float64)
    p = CorrParams(8, (16.0,))
    for form in ("scatter", "gather"):
        y = spectral.simulate_spectral(x, 10**6, 3.0, [H, H, H], layers, [1.0, 1.0, 1.0], p, (9, 9), form=form)
        ref = frame.simulate(x, 10**6, 3.0, H, layers, p, (9, 9), form=form).y
        assert np.max(np.abs(y - ref)) < 1e-12


def test_channels_do_not_interact_and_use_their_own_scale():
    rng = np.random.default_rng(7)
    h, w = 18, 21
    T = 9 * 9
    Hs = [np.linalg.qr(rng.normal(size=(T, 10)))[0].T for _ in range(3)]
    layers = inputs.mlp_weights([33, 16, 10], 43)
    x = inputs.blob_image(h, w, 3, 1008).astype(np.float64)
    p = CorrParams(8, (16.0,))
    sc = [spectral.phase_scale(lam) for lam in spectral.WAVELENGTHS_NM]
    y = spectral.simulate_spectral(x, 5, 4.0, Hs, layers, sc, p, (9, 9))
    Hs2 = [Hs[0], Hs[1], np.linalg.qr(rng.normal(size=(T, 10)))[0].T]
    y2 = spectral.simulate_spectral(x, 5, 4.0, Hs2, layers, sc, p, (9, 9))
    np.testing.assert_array_equal(y[..., :2], y2[..., :2])
    assert np.max(np.abs(y[..., 2] - y2[..., 2])) > 1e-3
    # channel c equals the single-wavelength frame of that channel with its scale folded into W1
    for c in range(3):
        lay_c = [(layers[0][0] * sc[c], layers[0][1])] + list(layers[1:])
        ref = frame.simulate(x[..., c : c + 1], 5, 4.0, Hs[c], lay_c, p, (9, 9), form="gather").y
        assert np.max(np.abs(y[..., c : c + 1] - ref)) < 1e-12


def test_channel_basis_is_orthonormal_and_differs_between_wavelengths():
    z, dr0 = inputs.dictionary_draws(400, 35, (0.5, 6.0), 2021)
    Hb, _ = spectral.make_basis_at(z, dr0, 10, 9, spectral.phase_scale(450.0))
    Hr, _ = spectral.make_basis_at(z, dr0, 10, 9, spectral.phase_scale(570.0))
    assert np.max(np.abs(Hb @ Hb.T - np.eye(10))) < 1e-12
    # the leading (mean-PSF) vectors differ: the blue PSFs are narrower
    assert abs(Hb[0] @ Hr[0]) < 0.9999


def test_product_spectral_basis_matches_oracle():
    """basis.build_basis_spectral (the product's offline builder, written independently of
    the oracle) gives the oracle's channel bases for the same draws."""
    from paper_2107_11627_gb300 import basis

    Hs = basis.build_basis_spectral(K=8, taps=9, n_dict=300, cache=False)
    z, dr0 = inputs.dictionary_draws(300, 35, (0.5, 6.0), 2021)
    for lam, Hp in zip(spectral.WAVELENGTHS_NM, Hs):
        Ho, _ = spectral.make_basis_at(z, dr0, 8, 9, spectral.phase_scale(lam))
        assert np.max(np.abs(Hp - Ho)) < 1e-8, lam
