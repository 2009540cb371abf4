"""Wavelength-dependent colour (Sec. 3.5) through the CUDA path: three bases (570, 540,
450 nm), the network's input scaled by lambda_ref / lambda_c per channel, one field draw
and one warp; p2s_simulate_spectral against oracle.spectral, FP32 (17x17 taps) and FP16
tensor-core gather (33x33 taps)."""
import functools

import numpy as np
import pytest

import oracle
from oracle import spectral
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_BF16, TOL_FP32, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@functools.lru_cache(maxsize=None)
def _bases(K, taps, n_dict):
    z, dr0 = inputs.dictionary_draws(n_dict, 35, (0.5, 6.0), 2021)
    return tuple(spectral.make_basis_at(z, dr0, K, taps, spectral.phase_scale(lam))[0]
                 for lam in spectral.WAVELENGTHS_NM)


@pytest.mark.parametrize("prec,K,taps,dims,n_dict,tol",
                         [("fp32", 20, 17, [33, 64, 64, 20], 2000, TOL_FP32),
                          ("fp16", 100, 33, [33, 128, 128, 100], 4000, TOL_BF16)])
def test_spectral_frames_match_oracle(prec, K, taps, dims, n_dict, tol):
    from paper_2107_11627_gb300 import p2s

    bases = _bases(K, taps, n_dict)
    layers = inputs.mlp_weights(dims, 42)
    sim = p2s.SpectralSimulator(list(bases), (taps, taps), layers, anchor_spacing=8, corr_len_px=(16.0,),
                                precision=prec, form="gather")
    shapes = [(64, 96), (37, 50)]
    xs = [inputs.blob_image(h, w, 3, 1100 + i) for i, (h, w) in enumerate(shapes)]
    dr, seeds = [2.0, 5.0], [10**6 + 40, 10**6 + 41]
    ys = sim.simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    sim.check()
    sc = [spectral.phase_scale(lam) for lam in spectral.WAVELENGTHS_NM]
    for i in range(len(xs)):
        ref = spectral.simulate_spectral(xs[i].astype(np.float64), seeds[i], dr[i], list(bases), layers, sc,
                                         CorrParams(8, (16.0,)), (taps, taps), form="gather")
        close(ys[i].cpu().numpy(), ref, tol, f"{prec} {shapes[i]}")
    # the three channels differ from the single-wavelength frame (the blue PSF is narrower)
    one = oracle.frame.simulate(xs[0].astype(np.float64), seeds[0], dr[0], bases[1], layers,
                                CorrParams(8, (16.0,)), (taps, taps), form="gather").y
    assert np.max(np.abs(ys[0].cpu().numpy()[..., 2] - one[..., 2])) > 10 * tol * np.max(np.abs(one))
    sim.close()


def test_spectral_rejects_mismatched_contexts():
    from paper_2107_11627_gb300 import p2s

    bases = _bases(20, 17, 2000)
    layers = inputs.mlp_weights([33, 64, 64, 20], 42)
    sim = p2s.SpectralSimulator(list(bases), (17, 17), layers, precision="fp32", form="gather")
    sim.sims[2].close()
    sim.sims[2] = p2s.Simulator(bases[2], (17, 17), layers, anchor_spacing=4, precision="fp32", form="gather")
    x = torch.zeros((16, 16, 3), device="cuda")
    with pytest.raises(p2s.P2SError):
        sim.simulate([x], [2.0], [1])
    sim.close()
