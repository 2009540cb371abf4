"""The dense anchor draw (Sec. 3.4, f = chol(Sigma) w over the anchors) on the GPU
against the FP64 oracle, alone and inside whole frames."""
import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_BF16, TOL_FIELD, cfg1, cfg2, rel, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _sim(c, s=8, ell=(16.0,), precision="fp32", form="scatter"):
    from paper_2107_11627_gb300 import p2s

    sim = p2s.Simulator(c["H"], c["taps"], c["layers"], anchor_spacing=s, corr_len_px=ell, precision=precision,
                        form=form)
    sim.set_option("field_method", 1)
    return sim


@pytest.mark.parametrize("h,w,s,ell", [(64, 64, 8, (16.0,)), (256, 256, 8, (16.0,)), (37, 53, 4, (6.0,)),
                                       (1, 1, 8, (16.0,)), (120, 72, 8, (24.0, 20.0, 16.0, 12.0, 10.0, 8.0, 6.0)),
                                       (1000, 600, 8, (16.0,))])
def test_dense_fields(h, w, s, ell):
    sim = _sim(cfg1(), s=s, ell=ell)
    p = CorrParams(s, ell)
    seeds = [10**6 + 5, 2**41 + 3]
    dr = [1.5, 5.0]
    a = sim.stage_fields(h, w, dr, seeds).cpu().numpy().astype(np.float64)
    assert np.all(a[..., 0] == 0)
    for i in range(2):
        ref = oracle.fields.alpha_anchors(seeds[i], dr[i], h, w, p, method="dense")
        close(a[i, ..., 1:], ref, TOL_FIELD, i)


def test_dense_fields_frames_tensor_core():
    sim = _sim(cfg2(), precision="fp16", form="gather")
    shapes = [(96, 160), (64, 64)]
    xs = [inputs.blob_image(h, w, 3, 2400 + i) for i, (h, w) in enumerate(shapes)]
    dr, seeds = [3.0, 1.0], [71, 72]
    ys = sim.simulate([torch.from_numpy(x).cuda() for x in xs], dr, seeds)
    sim.check()
    for i in range(2):
        ref = oracle.frame.simulate(xs[i].astype(np.float64), seeds[i], dr[i], cfg2()["H"], cfg2()["layers"],
                                    CorrParams(8, (16.0,)), (33, 33), form="gather", field_method="dense")
        close(ys[i].cpu().numpy(), ref.y, TOL_BF16, i)


def test_dense_fields_too_many_anchors_are_refused():
    from paper_2107_11627_gb300 import p2s

    sim = _sim(cfg1())
    with pytest.raises(p2s.P2SError):
        sim.stage_fields(1100, 64, [1.0], [1])
