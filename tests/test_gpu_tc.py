"""GPU parity of the tensor-core path (tcgen05): the network stage, the blur
stage and whole frames against the FP64 oracle, FP16 and BF16 operands."""
import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from oracle.precision import bf16
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_BF16, cfg2, rel, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _sim(prec, form="gather", s=8):
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    return p2s.Simulator(c["H"], c["taps"], c["layers"], anchor_spacing=s, corr_len_px=(16.0,), precision=prec,
                         form=form)


def _alpha_f32(seed, dr, h, w, s=8):
    a = oracle.fields.alpha_anchors(seed, dr, h, w, CorrParams(s, (16.0,))).astype(np.float32)
    full = np.zeros(a.shape[:2] + (36,), dtype=np.float32)
    full[..., 1:] = a
    return full


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("h,w", [(64, 128), (37, 150), (2, 3)])
def test_tc_network_stage(prec, h, w):
    sim = _sim(prec)
    al = _alpha_f32(21, 4.0, h, w)
    beta = sim.stage_mlp(h, w, torch.from_numpy(al).cuda())
    sim.check()
    beta = beta.cpu().numpy()
    ap = oracle.fields.alpha_pixels(al[..., 1:].astype(np.float64), h, w, 8)
    ref = oracle.mlp.forward(ap[..., 2:], cfg2()["layers"])
    close(beta, ref, TOL_BF16)


@pytest.mark.parametrize("split", [1, 2, 3, 4, 0])
@pytest.mark.parametrize("c", [3, 1])
@pytest.mark.parametrize("h,w", [(40, 130), (33, 64), (1, 1), (70, 300)])
def test_tc_blur_stage_fp16(c, h, w, split):
    """Every gather kernel: the four blur-only ones fed 16-bit beta (split = 1, the
    default; 2 and 3, the fragment kernels; 4, packed FP16 products) and the fused one
    (split = 0)."""
    sim = _sim("fp16")
    sim.set_option("gather_split", split)
    rng = np.random.default_rng(31)
    xw = inputs.blob_image(h, w, c, 1003)
    beta = (rng.normal(0.0, 0.05, size=(h, w, 100)) + 0.3 * (np.arange(100) == 0)).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw).cuda(), torch.from_numpy(beta).cuda())
    sim.check()
    y = y.cpu().numpy()
    ref = oracle.blur.gather(xw.astype(np.float64), beta.astype(np.float64), cfg2()["H"], 33, 33)
    close(y, ref, TOL_BF16)


def _shift(src, dy, dx):
    """out[i, j] = src[i - dy, j - dx], zero outside the frame."""
    h, w = src.shape[:2]
    out = np.zeros_like(src)
    ys, ye, xs, xe = max(0, -dy), min(h, h - dy), max(0, -dx), min(w, w - dx)
    if ys < ye and xs < xe:
        out[ys + dy : ye + dy, xs + dx : xe + dx] = src[ys:ye, xs:xe]
    return out


def _gather_rounded_g(x, beta, Hb, th, tw, g_round):
    """Eq. 5 gather with every G[q, t] = sum_k beta[q, k] H[k, t] passed through g_round
    before the tap products (FP64 otherwise): the split kernel's extra rounding point."""
    h, w, _ = x.shape
    G = (beta.reshape(h * w, -1).astype(np.float64) @ Hb.astype(np.float64)).reshape(h, w, -1)
    G = g_round(G)
    y = np.zeros(x.shape, dtype=np.float64)
    for i, (dy, dx) in enumerate(oracle.blur.tap_offsets(th, tw)):
        y += G[:, :, i : i + 1] * _shift(x, dy, dx)
    return y


@pytest.mark.parametrize("split", [1, 2, 3, 0])
def test_tc_blur_stage_bf16_rounding_points(split):
    """BF16 operands: each gather kernel must round exactly beta and H to BF16; the fused
    kernel (0) and the FP16-x blur-only kernels (1, 2) also the staged x_w window to FP16,
    the latter two G to FP16 before the tap products; the FP32-x kernel (3) nothing else.
    Checked against the oracle with exactly those tensors rounded; everything else FP32."""
    sim = _sim("bf16")
    sim.set_option("gather_split", split)
    rng = np.random.default_rng(32)
    h, w = 48, 160
    xw = inputs.blob_image(h, w, 3, 1004)
    beta = (rng.normal(0.0, 0.05, size=(h, w, 100)) + 0.3 * (np.arange(100) == 0)).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw).cuda(), torch.from_numpy(beta).cuda()).cpu().numpy()
    # round-to-nearest-even, as the FP16-x kernels stage it
    x16 = xw.astype(np.float16).astype(np.float64) if split != 3 else xw.astype(np.float64)
    bb, hb = bf16(beta), bf16(cfg2()["H"])
    emu = oracle.blur.gather(x16, bb, hb, 33, 33)
    if split in (1, 2):
        # the emulation without its rounding is the oracle's gather itself
        assert rel(_gather_rounded_g(x16, bb, hb, 33, 33, lambda g: g), emu) < 1e-12
        emu = _gather_rounded_g(x16, bb, hb, 33, 33, lambda g: g.astype(np.float16).astype(np.float64))
    close(y, emu, 2e-5)


@pytest.mark.parametrize("s", [8, 1])
def test_tc_frames_fp16(s):
    sim = _sim("fp16", s=s)
    shapes = [(96, 80), (50, 200), (96, 80)]
    xs = [inputs.blob_image(h, w, 3, 1000 + i) for i, (h, w) in enumerate(shapes)]
    dr, seeds = [1.5, 4.0, 6.0], [10**6, 10**6 + 1, 10**6 + 2]
    ys = sim.simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    sim.check()
    for i in range(3):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), seeds[i], dr[i], cfg2()["H"], cfg2()["layers"],
                                    CorrParams(s, (16.0,)), (33, 33), form="gather")
        close(ys[i].cpu().numpy(), ref.y, TOL_BF16, i)


def test_tc_full_size_frame_fp16():
    """One 512 x 512 RGB frame of the benchmark workload, whole frame checked."""
    sim = _sim("fp16")
    x = inputs.blob_image(512, 512, 3, 1000)
    (y,) = sim.simulate([torch.from_numpy(x).cuda()], [3.0], [10**6])
    ref = oracle.frame.simulate(x.astype(np.float64), 10**6, 3.0, cfg2()["H"], cfg2()["layers"],
                                CorrParams(8, (16.0,)), (33, 33), form="gather")
    close(y.cpu().numpy(), ref.y, TOL_BF16)


def test_benchmark_batch_64_frames_512_rgb():
    """The benchmark's launch configuration: 64 RGB frames of 512 x 512 in one call (one field,
    warp, network and packed-FP16 gather launch over all of them, D/r0 spread over [1, 5]).
    The first and the last frame are checked whole against the oracle, and both equal the
    same frame simulated alone, bit for bit."""
    sim = _sim("fp16")
    n = 64
    xs = [inputs.blob_image(512, 512, 3, 3000 + i) for i in range(n)]
    dr = [1.0 + 4.0 * i / (n - 1) for i in range(n)]
    seeds = [2 * 10**6 + i for i in range(n)]
    ys = sim.simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    sim.check()
    for i in (0, n - 1):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), seeds[i], dr[i], cfg2()["H"], cfg2()["layers"],
                                    CorrParams(8, (16.0,)), (33, 33), form="gather")
        close(ys[i].cpu().numpy(), ref.y, TOL_BF16, i)
        (alone,) = sim.simulate([torch.from_numpy(xs[i]).cuda()], [dr[i]], [seeds[i]])
        sim.check()
        assert torch.equal(alone, ys[i]), i


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("c,h,w", [(3, 48, 160), (1, 37, 150)])
def test_tc_blur_stage_h2_rounding_points(prec, c, h, w):
    """The packed-FP16 gather kernel (4) against an emulation of its arithmetic in its order
    (tests/kernel_emulation.py): beta and H rounded to the operand type, G and x_w to FP16,
    FP16 sums of 12 products (two per chunk, channel and row, by tap-column parity) flushed
    into FP32, tap column 32 as FP32 sums, the groups' sums added in order.  The tensor core's
    FP32 sums for G differ from the emulation's FP64 G in the last bit, which now and then
    flips G's FP16 rounding and, through the FP16 sums, an FP16 ulp of a partial sum (2.5e-5
    measured with sums of 24 products).  FP32 sums of the same products (kernel 1's
    arithmetic) are 2.3e-4 from the emulation on these inputs, four times the tolerance, so
    the test tells the two apart.  The odd last row pair and the ragged column tail are
    covered."""
    import kernel_emulation

    sim = _sim(prec)
    sim.set_option("gather_split", 4)
    rng = np.random.default_rng(33)
    xw = inputs.blob_image(h, w, c, 1005)
    beta = (rng.normal(0.0, 0.05, size=(h, w, 100)) + 0.3 * (np.arange(100) == 0)).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw).cuda(), torch.from_numpy(beta).cuda())
    sim.check()
    y = y.cpu().numpy()
    rnd = bf16 if prec == "bf16" else (lambda v: v.astype(np.float16).astype(np.float64))
    emu = kernel_emulation.gather_h2(xw, beta, cfg2()["H"], rnd)
    close(y, emu, 6e-5)
    ref = oracle.blur.gather(xw.astype(np.float64), beta.astype(np.float64), cfg2()["H"], 33, 33)
    assert rel(emu, ref) > 1e-4  # the FP16 sums are what the emulation models


@pytest.mark.parametrize("split", [4])
def test_tc_full_size_frame_fp16_kernel4(split):
    """One 512 x 512 RGB frame through the packed-FP16 gather kernel, whole frame checked."""
    sim = _sim("fp16")
    sim.set_option("gather_split", split)
    x = inputs.blob_image(512, 512, 3, 1000)
    (y,) = sim.simulate([torch.from_numpy(x).cuda()], [3.0], [10**6])
    sim.check()
    ref = oracle.frame.simulate(x.astype(np.float64), 10**6, 3.0, cfg2()["H"], cfg2()["layers"],
                                CorrParams(8, (16.0,)), (33, 33), form="gather")
    close(y.cpu().numpy(), ref.y, TOL_BF16)
