"""Pins of the whole-frame oracle against Eq. 3 (Sec. 3.1): the per-pixel PSF blur
with no basis and no network, on 16x16 and 64x64 frames with the 64x64 grey
workload's basis (K = 20 of 17x17 taps from 2,000 PSFs).

With beta_p = H h_p (the least-squares projection; H has orthonormal rows):
  * K = T: the basis blur equals the exact blur (Eq. 4 is then an identity);
  * K < T: exact - basis = the exact blur of the truncation residual h_p - H^T beta_p.
Both forms: the scatter blur against Eq. 3 (each source pixel's PSF), the gather
blur (Eq. 5) against Eq. 3's row form (each output pixel's PSF).
"""
import functools

import numpy as np
import pytest

from oracle import blur, fields, frame, psf
from paper_2107_11627_gb300 import inputs

TH = 17


@functools.lru_cache(maxsize=None)
def _bases():
    z, dr0 = inputs.dictionary_draws(2000, 35, (0.5, 6.0), 2021)
    full, _ = psf.make_basis(z, dr0, K=TH * TH, taps=TH)
    return full, full[:20]


@functools.lru_cache(maxsize=None)
def _frame(h, w, form):
    p = fields.CorrParams(8, (16.0,))
    x = inputs.block_image(h, w, min(8, h // 2), 1, 1000)
    return x, frame.exact_frame(x, 10**6, 2.0, p, (TH, TH), form=form)


def test_full_basis_is_orthonormal():
    full, _ = _bases()
    assert np.max(np.abs(full @ full.T - np.eye(TH * TH))) < 1e-12


@pytest.mark.parametrize("h,w", [(16, 16), (64, 64)])
def test_exact_frame_shares_fields_and_warp_with_simulate(h, w):
    p = fields.CorrParams(8, (16.0,))
    x, (xw, hp, _) = _frame(h, w, "scatter")
    st = frame.simulate(x, 10**6, 2.0, _bases()[1], inputs.mlp_weights([33, 64, 64, 20], 42), p, (TH, TH))
    assert np.array_equal(st.xw, xw)
    assert hp.shape == (h, w, TH, TH)
    assert np.allclose(hp.sum(axis=(2, 3)), 1.0, atol=1e-12)  # unit-sum taps (Sec. 3.1 normalisation)


@pytest.mark.parametrize("form", ["scatter", "gather"])
@pytest.mark.parametrize("h,w", [(16, 16), (64, 64)])
def test_full_basis_equals_exact(h, w, form):
    full, _ = _bases()
    _, (xw, hp, y_exact) = _frame(h, w, form)
    beta = hp.reshape(h, w, -1) @ full.T
    fn = blur.scatter if form == "scatter" else blur.gather
    y = fn(xw, beta, full, TH, TH)
    assert np.max(np.abs(y - y_exact)) < 1e-12 * max(1.0, np.max(np.abs(y_exact)))


@pytest.mark.parametrize("form", ["scatter", "gather"])
@pytest.mark.parametrize("h,w", [(16, 16), (64, 64)])
def test_truncation_residual_identity(h, w, form):
    _, part = _bases()
    _, (xw, hp, y_exact) = _frame(h, w, form)
    beta = hp.reshape(h, w, -1) @ part.T
    resid = hp - (beta @ part).reshape(hp.shape)
    fn, ex = (blur.scatter, blur.exact) if form == "scatter" else (blur.gather, blur.exact_gather)
    diff = y_exact - fn(xw, beta, part, TH, TH)
    assert np.max(np.abs(diff - ex(xw, resid))) < 1e-12
    # K = 20 leaves a visible truncation error: the identity is not vacuous
    assert np.max(np.abs(diff)) > 1e-4


def test_exact_forms_match_their_definitions():
    """Both Eq. 3 forms as dense operators on a tiny frame, entry by entry against the
    definitions S[q, p] = h_p[q - p] (scatter) and G[q, p] = h_q[q - p] (gather)."""
    rng = np.random.default_rng(5)
    h, w, th, tw = 6, 7, 3, 5
    hp = rng.normal(size=(h, w, th, tw))
    n = h * w
    S = np.zeros((n, n))
    G = np.zeros((n, n))
    for i in range(n):
        e = np.zeros((h, w, 1))
        e.flat[i] = 1.0
        S[:, i] = blur.exact(e, hp).ravel()
        G[:, i] = blur.exact_gather(e, hp).ravel()
    for q in range(n):
        for pp in range(n):
            dy = q // w - pp // w + th // 2
            dx = q % w - pp % w + tw // 2
            inside = 0 <= dy < th and 0 <= dx < tw
            assert S[q, pp] == (hp.reshape(n, th, tw)[pp, dy, dx] if inside else 0.0)
            assert G[q, pp] == (hp.reshape(n, th, tw)[q, dy, dx] if inside else 0.0)
