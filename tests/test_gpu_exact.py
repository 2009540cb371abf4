"""The CUDA blur against Eq. 3 (Sec. 3.1) by brute force: every pixel's PSF formed from its
own Zernike vector by the pupil FFT (Eq. 2), projected on a FULL basis (K = T = 81 for
9x9 taps, so Eq. 4 is an identity), and that projected beta fed through p2s_stage_blur
in FP32.  The scatter form must then equal the exact per-pixel convolution, and the
gather form (Eq. 5) its row form, within the FP32 tolerance."""
import functools

import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_FP32, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TH = 9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@functools.lru_cache(maxsize=None)
def _full_basis():
    z, dr0 = inputs.dictionary_draws(600, 35, (0.5, 6.0), 2021)
    H, _ = oracle.psf.make_basis(z, dr0, K=TH * TH, taps=TH)
    assert np.max(np.abs(H @ H.T - np.eye(TH * TH))) < 1e-12
    return H


@pytest.mark.parametrize("form", ["scatter", "gather"])
@pytest.mark.parametrize("h,w,c,dr", [(48, 72, 3, 3.0), (33, 20, 1, 5.0)])
def test_blur_of_projected_beta_equals_exact(form, h, w, c, dr):
    from paper_2107_11627_gb300 import p2s

    H = _full_basis()
    layers = inputs.mlp_weights([33, 64, TH * TH], 42)  # unused by the blur stage
    sim = p2s.Simulator(H, (TH, TH), layers, precision="fp32", form=form)
    x = inputs.blob_image(h, w, c, 1003)
    xw, hp, _ = oracle.frame.exact_frame(x.astype(np.float64), 10**6 + 9, dr, CorrParams(8, (16.0,)), (TH, TH),
                                         form=form)
    xw32 = xw.astype(np.float32)
    beta = (hp.reshape(h, w, -1) @ H.T).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw32).cuda(), torch.from_numpy(beta).cuda()).cpu().numpy()
    ex = oracle.blur.exact if form == "scatter" else oracle.blur.exact_gather
    ref = ex(xw32.astype(np.float64), hp)
    close(y, ref, TOL_FP32, form)
    sim.close()
