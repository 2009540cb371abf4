"""P2S network training (Sec. 3.3): pairs from the dictionary, l2 fit of the
projected coefficients; the fitted network must beat both the untrained network
and the best constant predictor, and approach the basis-truncation floor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_training_pairs_are_projections():
    from paper_2107_11627_gb300 import train
    from gpu_common import basis

    H = basis(20, 17, 2000)
    a, beta, psf = train.training_pairs(H, 300, 17)
    assert a.shape == (300, 33) and beta.shape == (300, 20) and psf.shape == (300, 289)
    np.testing.assert_allclose(psf.sum(axis=1), 1.0, atol=1e-12)
    # beta* is the least-squares projection: the residual is orthogonal to the basis
    r = psf - beta @ H
    assert np.abs(r @ H.T).max() < 1e-12


def test_training_reduces_the_loss_towards_the_projection_floor():
    from paper_2107_11627_gb300 import train
    from gpu_common import basis

    H = basis(20, 17, 2000)
    layers, rep = train.train_p2s(H, [33, 64, 64, 20], n_dict=3000, taps=17, epochs=12, batch=128, cache=False)
    assert [W.shape for W, _ in layers] == [(64, 33), (64, 64), (20, 64)]
    # the trained network explains most of the coefficient variance
    assert rep["val_beta_mse"] < 0.2 * rep["val_beta_mse_zero_predictor"]
    assert rep["val_beta_mse"] < 0.5 * rep["val_beta_mse_first_epoch"]
    # and its PSFs are within a small factor of the truncation floor
    assert rep["psf_rel_err_network_median"] < 3.0 * rep["psf_rel_err_projection_median"] + 0.05


def test_trained_network_matches_short_and_long_exposure_psfs():
    """Sec. 4.1, Evaluation 2: the mean of the centred PSFs (short exposure) and of the
    tilt-shifted PSFs (long exposure) produced through the trained network agree with those
    of the pupil-FFT PSFs it replaces, in shape and width; an untrained network does not."""
    from paper_2107_11627_gb300 import inputs, train
    from gpu_common import basis

    H = basis(20, 17, 2000)
    layers, _ = train.train_p2s(H, [33, 64, 64, 20], n_dict=3000, taps=17, epochs=12, batch=128, cache=False)
    untrained = inputs.mlp_weights([33, 64, 64, 20], 42)
    for d in (1.5, 4.0):
        e = train.exposure_psfs(H, layers, 17, d, n=1000)
        u = train.exposure_psfs(H, untrained, 17, d, n=1000)
        for k in ("se", "le"):
            assert e[k]["rel_l2"] < 0.15, (d, k, e[k]["rel_l2"])
            assert abs(e[k]["width_network"] / e[k]["width_psf"] - 1.0) < 0.1, (d, k)
            assert u[k]["rel_l2"] > 0.5
        # the long exposure is wider than the short one (it includes the tilt shifts)
        assert e["le"]["width_psf"] > e["se"]["width_psf"]
