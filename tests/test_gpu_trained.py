"""The trained P2S network (Sec. 3.3) through the CUDA path: weights fitted on the
dictionary by train.py run in p2s_simulate and must match the FP64 oracle run with
the same weights (FP32 path, both blur forms, the 64x64 grey workload's basis)."""
import functools

import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_FP32, basis, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@functools.lru_cache(maxsize=None)
def _trained():
    from paper_2107_11627_gb300 import train

    H = basis(20, 17, 2000)
    layers, rep = train.train_p2s(H, [33, 64, 64, 20], n_dict=3000, taps=17, epochs=12, batch=128, cache=False)
    return H, layers, rep


@pytest.mark.parametrize("form", ["scatter", "gather"])
def test_trained_weights_through_the_cuda_path(form):
    from paper_2107_11627_gb300 import p2s

    H, layers, rep = _trained()
    assert rep["val_beta_mse"] < 0.2 * rep["val_beta_mse_zero_predictor"]
    sim = p2s.Simulator(H, (17, 17), layers, anchor_spacing=8, corr_len_px=(16.0,), precision="fp32", form=form)
    x = inputs.block_image(64, 64, 8, 1, 1000)
    xs = [x, inputs.blob_image(40, 56, 3, 1001)]
    dr, seeds = [2.0, 4.0], [10**6, 10**6 + 1]
    ys = sim.simulate([torch.from_numpy(v).cuda() for v in xs], dr, seeds)
    sim.check()
    for i, v in enumerate(xs):
        ref = oracle.frame.simulate(v.astype(np.float64), seeds[i], dr[i], H, layers, CorrParams(8, (16.0,)),
                                    (17, 17), form=form)
        close(ys[i].cpu().numpy(), ref.y, TOL_FP32, i)
    sim.close()
