"""GPU parity of the batched-FFT evaluation of the scatter blur (the comparison
variant, FP32) against the FP64 oracle's direct scatter sum."""
import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_FP32, cfg2, rel, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _sim(form="fft"):
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    return p2s.Simulator(c["H"], c["taps"], c["layers"], anchor_spacing=8, corr_len_px=(16.0,), precision="fp32",
                         form=form)


@pytest.mark.parametrize("c", [3, 1])
@pytest.mark.parametrize("h,w", [(40, 130), (1, 1), (70, 300), (96, 97)])
def test_fft_blur_stage(c, h, w):
    sim = _sim()
    rng = np.random.default_rng(41)
    xw = inputs.blob_image(h, w, c, 1007)
    beta = (rng.normal(0.0, 0.05, size=(h, w, 100)) + 0.3 * (np.arange(100) == 0)).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw).cuda(), torch.from_numpy(beta).cuda())
    sim.check()
    ref = oracle.blur.scatter(xw.astype(np.float64), beta.astype(np.float64), cfg2()["H"], 33, 33)
    close(y.cpu().numpy(), ref, TOL_FP32)


def test_fft_frames_match_oracle_and_direct_path():
    shapes = [(96, 80), (50, 200)]
    xs = [inputs.blob_image(h, w, 3, 1100 + i) for i, (h, w) in enumerate(shapes)]
    dr, seeds = [2.0, 4.5], [31, 32]
    fft = _sim().simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    direct = _sim("scatter").simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    for i in range(2):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), seeds[i], dr[i], cfg2()["H"], cfg2()["layers"],
                                    CorrParams(8, (16.0,)), (33, 33), form="scatter")
        close(fft[i].cpu().numpy(), ref.y, TOL_FP32)
        close(fft[i].cpu().numpy(), direct[i].cpu().numpy(), TOL_FP32)


def test_fft_needs_fp32():
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    with pytest.raises(p2s.P2SError):
        p2s.Simulator(c["H"], c["taps"], c["layers"], precision="fp16", form="fft")
