"""GPU parity of the FP8 E4M3 contraction (Sec. 3.1, Eq. 4-5 with E4M3 operands):
beta and the basis each as an E4M3 hi/lo pair with per-basis power-of-two scales,
G = b_hi H_hi + b_lo H_hi + b_hi H_lo accumulated in FP32 by tcgen05.mma
(.kind::f8f6f4), the network in FP16.  Rounding points checked against the oracle
with exactly those roundings; whole frames against the FP64 oracle at the FP8
tolerance (1e-2 relative L2)."""
import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from oracle.precision import e4m3
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_FP8, cfg2, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _sim(form="gather"):
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    return p2s.Simulator(c["H"], c["taps"], c["layers"], anchor_spacing=8, corr_len_px=(16.0,), precision="fp8",
                         form=form)


def _hi_lo(v, f32):
    """E4M3 hi/lo pair of v: hi = e4m3(v), lo = e4m3(v - hi), the difference in FP32 (device
    side, beta) or FP64 (host side, the basis)."""
    hi = e4m3(v)
    r = (np.asarray(v, np.float32) - np.asarray(hi, np.float32)).astype(np.float64) if f32 else v - hi
    return hi, e4m3(r)


def _gather_with_g(x, G, th, tw):
    h, w, _ = x.shape
    y = np.zeros(x.shape, dtype=np.float64)
    for i, (dy, dx) in enumerate(oracle.blur.tap_offsets(th, tw)):
        y += G[:, :, i : i + 1] * oracle.blur._shifted(x, dy, dx)
    return y


def test_fp8_blur_stage_rounding_points():
    """beta scaled and split into E4M3 hi/lo on the device, the basis scaled and split on the
    host, the three products summed (FP32), G rounded to FP16, x_w to FP16, tap sums in FP32
    times 2^-c: the kernel against the oracle with exactly those roundings."""
    sim = _sim()
    scale, inv_c = sim.contraction_scales()
    K = cfg2()["H"].shape[0]
    assert np.all(scale[:K] > 0) and inv_c > 0
    # powers of two
    assert np.all(np.frexp(scale[: K + 2])[0] == 0.5) and np.frexp(inv_c)[0] == 0.5
    rng = np.random.default_rng(33)
    h, w = 48, 160
    xw = inputs.blob_image(h, w, 3, 1005)
    beta = (rng.normal(0.0, 0.05, size=(h, w, K)) + 0.3 * (np.arange(K) == 0)).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw).cuda(), torch.from_numpy(beta).cuda())
    sim.check()
    y = y.cpu().numpy()
    Hb = cfg2()["H"]
    bs = (beta * scale[None, None, :K]).astype(np.float32).astype(np.float64)
    bhi, blo = _hi_lo(bs, True)
    rows = Hb / (scale[:K, None].astype(np.float64) * inv_c)  # H_k 2^c / scale_k
    hhi, hlo = _hi_lo(rows, False)
    b2h, b2l = bhi.reshape(h * w, K), blo.reshape(h * w, K)
    G = (b2h @ hhi + b2l @ hhi + b2h @ hlo).reshape(h, w, -1)
    G16 = G.astype(np.float16).astype(np.float64)
    x16 = xw.astype(np.float16).astype(np.float64)
    emu = inv_c * _gather_with_g(x16, G16, 33, 33)
    close(y, emu, 2e-5)
    # and within the FP8 tolerance of the unrounded blur
    close(y, oracle.blur.gather(xw.astype(np.float64), beta.astype(np.float64), Hb, 33, 33), TOL_FP8)


@pytest.mark.parametrize("shapes,dr", [([(96, 80), (50, 200), (33, 129)], [1.5, 4.0, 6.0]), ([(512, 512)], [3.0])])
def test_fp8_frames_within_contract(shapes, dr):
    sim = _sim()
    xs = [inputs.blob_image(h, w, 3, 1000 + i) for i, (h, w) in enumerate(shapes)]
    seeds = [10**6 + 20 + i for i in range(len(xs))]
    ys = sim.simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    sim.check()
    for i in range(len(xs)):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), seeds[i], dr[i], cfg2()["H"], cfg2()["layers"],
                                    CorrParams(8, (16.0,)), (33, 33), form="gather")
        close(ys[i].cpu().numpy(), ref.y, TOL_FP8, f"{shapes[i]} D/r0={dr[i]}")


def test_fp8_unsupported_combinations():
    from paper_2107_11627_gb300 import p2s

    with pytest.raises(p2s.P2SError):
        _sim(form="scatter")
    sim = _sim()
    with pytest.raises(p2s.P2SError):
        sim.set_option("gather_split", 0)
    assert sim.get_option("gather_split") == 1
