"""GPU parity: each stage and the whole path through the C ABI against the
FP64 oracle, on seeded inputs, at sizes spanning several tiles with ragged
tails, plus edge cases (1x1 frames, C = 1, mixed sizes, empty batches)."""
import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_FIELD, TOL_FP32, cfg1, cfg2, rel, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sim(cfg, s=8, ell=(16.0,), form="scatter", precision="fp32"):
    from paper_2107_11627_gb300 import p2s

    return p2s.Simulator(cfg["H"], cfg["taps"], cfg["layers"], anchor_spacing=s, corr_len_px=ell,
                         precision=precision, form=form)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("seed,mode,fh,fw", [(10**6, 0, 16, 16), (2**63 + 5, 34, 128, 64), (7, 3, 2, 2), (1, 1, 256, 4)])
def test_noise(seed, mode, fh, fw):
    sim = _sim(cfg1())
    z = sim.stage_noise(seed, mode, fh, fw).cpu().numpy().astype(np.float64)
    ref = oracle.philox.normals(seed, mode, fh * fw).reshape(fh, fw)
    close(z, ref, TOL_FIELD / 4)
    assert np.max(np.abs(z - ref)) < 2e-6


# (128, 128, 1): 129 x 129 anchors on a 256 x 256 torus, several CTAs per field in both passes
@pytest.mark.parametrize("h,w,s,ell", [(64, 64, 8, (16.0,)), (64, 64, 1, (16.0,)), (256, 256, 8, (16.0,)),
                                       (37, 53, 4, (6.0,)), (1, 1, 8, (16.0,)), (128, 128, 1, (16.0,)),
                                       (120, 72, 8, (24.0, 20.0, 16.0, 12.0, 10.0, 8.0, 6.0))])
def test_fields(h, w, s, ell):
    sim = _sim(cfg1(), s=s, ell=ell)
    p = CorrParams(s, ell)
    seeds = [10**6 + 3, 2**40 + 1]
    dr = [2.0, 4.5]
    a = sim.stage_fields(h, w, dr, seeds).cpu().numpy().astype(np.float64)
    assert np.all(a[..., 0] == 0)
    for i in range(2):
        ref = oracle.fields.alpha_anchors(seeds[i], dr[i], h, w, p)
        assert a.shape[1:3] == ref.shape[:2]
        close(a[i, ..., 1:], ref, TOL_FIELD, i)


def _alpha_f32(seed, dr, h, w, p):
    """Oracle anchors rounded once to float32: the input both sides then share."""
    a = oracle.fields.alpha_anchors(seed, dr, h, w, p).astype(np.float32)
    full = np.zeros(a.shape[:2] + (36,), dtype=np.float32)
    full[..., 1:] = a
    return full


@pytest.mark.parametrize("h,w,c,s,dr", [(64, 64, 1, 8, 2.0), (57, 91, 3, 8, 5.0), (40, 40, 3, 1, 6.0), (1, 1, 3, 8, 3.0)])
def test_warp(h, w, c, s, dr):
    sim = _sim(cfg1(), s=s)
    p = CorrParams(s, (16.0,))
    al = _alpha_f32(11, dr, h, w, p)
    x = inputs.blob_image(h, w, c, 1001)
    xw = sim.stage_warp(torch.from_numpy(x).cuda(), torch.from_numpy(al).cuda()).cpu().numpy()
    ap = oracle.fields.alpha_pixels(al[..., 1:].astype(np.float64), h, w, s)
    ref = oracle.warp.warp(x.astype(np.float64), ap, oracle.warp.kappa())
    close(xw, ref, TOL_FIELD)


@pytest.mark.parametrize("which,h,w", [("cfg1", 64, 64), ("cfg2", 45, 70)])
def test_mlp(which, h, w):
    cfg = cfg1() if which == "cfg1" else cfg2()
    sim = _sim(cfg)
    p = CorrParams(8, (16.0,))
    al = _alpha_f32(12, 3.0, h, w, p)
    beta = sim.stage_mlp(h, w, torch.from_numpy(al).cuda()).cpu().numpy()
    ap = oracle.fields.alpha_pixels(al[..., 1:].astype(np.float64), h, w, 8)
    ref = oracle.mlp.forward(ap[..., 2:], cfg["layers"])
    close(beta, ref, TOL_FP32)


@pytest.mark.parametrize("form", ["scatter", "gather"])
@pytest.mark.parametrize("which,h,w,c", [("cfg1", 64, 64, 1), ("cfg2", 40, 56, 3), ("cfg2", 1, 1, 3), ("cfg1", 17, 5, 3)])
def test_blur(form, which, h, w, c):
    cfg = cfg1() if which == "cfg1" else cfg2()
    sim = _sim(cfg, form=form)
    rng = np.random.default_rng(13)
    xw = inputs.blob_image(h, w, c, 1002)
    beta = rng.normal(0.0, 0.05, size=(h, w, cfg["H"].shape[0])).astype(np.float32)
    y = sim.stage_blur(torch.from_numpy(xw).cuda(), torch.from_numpy(beta).cuda()).cpu().numpy()
    fn = oracle.blur.scatter if form == "scatter" else oracle.blur.gather
    ref = fn(xw.astype(np.float64), beta.astype(np.float64), cfg["H"], *cfg["taps"])
    close(y, ref, TOL_FP32)


@pytest.mark.parametrize("form", ["scatter", "gather"])
@pytest.mark.parametrize("s", [8, 1])
def test_frame_cfg1(form, s):
    cfg = cfg1()
    sim = _sim(cfg, s=s, form=form)
    x = inputs.block_image(64, 64, 8, 1, 1000)
    (y,) = sim.simulate([torch.from_numpy(x).cuda()], [2.0], [10**6])
    ref = oracle.frame.simulate(x.astype(np.float64), 10**6, 2.0, cfg["H"], cfg["layers"], CorrParams(s, (16.0,)),
                                cfg["taps"], form=form)
    close(y.cpu().numpy(), ref.y, TOL_FP32)


def test_frame_cfg2_batch_and_invariance():
    cfg = cfg2()
    sim = _sim(cfg)
    shapes = [(96, 80), (50, 33), (96, 80)]
    xs = [inputs.blob_image(h, w, 3, 1000 + i) for i, (h, w) in enumerate(shapes)]
    dr = [1.5, 4.0, 5.0]
    seeds = [10**6, 10**6 + 1, 10**6 + 2]
    xt = [torch.from_numpy(x).cuda() for x in xs]
    ys = sim.simulate(xt, dr, seeds)
    for i in range(3):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), seeds[i], dr[i], cfg["H"], cfg["layers"],
                                    CorrParams(8, (16.0,)), cfg["taps"])
        close(ys[i].cpu().numpy(), ref.y, TOL_FP32, i)
        (alone,) = sim.simulate([xt[i]], [dr[i]], [seeds[i]])
        close(alone.cpu().numpy(), ys[i].cpu().numpy(), 1e-6)
    assert sim.simulate([], [], []) == []


def test_frame_cfg2_full_size_batch():
    """The 256 x 256 RGB, 16-frame FP32 workload in one call; frames 0 and 11 checked whole."""
    cfg = cfg2()
    sim = _sim(cfg)
    n = 16
    xs = inputs.blob_batch(n, 256, 256, 3, 1000)
    dr = inputs.frame_strengths(n, 1.0, 5.0, 7)
    seeds = inputs.frame_seeds(n)
    ys = sim.simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    for i in (0, 11):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), int(seeds[i]), float(dr[i]), cfg["H"], cfg["layers"],
                                    CorrParams(8, (16.0,)), cfg["taps"])
        close(ys[i].cpu().numpy(), ref.y, TOL_FP32, i)


def test_host_entry_point_matches_device():
    cfg = cfg1()
    sim = _sim(cfg)
    x = inputs.block_image(64, 64, 8, 1, 1000)
    (yd,) = sim.simulate([torch.from_numpy(x).cuda()], [2.0], [10**6])
    (yh,) = sim.simulate_host([x], [2.0], [10**6])
    close(yh, yd.cpu().numpy(), 1e-6)


def test_invalid_arguments():
    from paper_2107_11627_gb300 import p2s

    sim = _sim(cfg1())
    x = torch.zeros((8, 8, 2), device="cuda")
    with pytest.raises(p2s.P2SError):
        sim.simulate([x], [2.0], [1])
    x = torch.zeros((8, 8, 3), device="cuda")
    with pytest.raises(p2s.P2SError):
        sim.simulate([x], [0.0], [1])
    with pytest.raises(p2s.P2SError):
        sim.simulate([x], [2.0], [1], out=[x])
