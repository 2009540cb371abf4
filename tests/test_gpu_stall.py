"""Stall detection without a GPU fault: a bounded device wait that runs out
sets the context's status word; the host sees P2S_ETIMEOUT once, and the
context keeps working."""
import numpy as np
import pytest

from paper_2107_11627_gb300 import inputs

from gpu_common import cfg2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    sim = p2s.Simulator(c["H"], c["taps"], c["layers"], precision="fp16", form="gather")
    sim.selftest_stall()
    with pytest.raises(p2s.P2SError) as e:
        sim.check()
    assert e.value.status == p2s.P2S_ETIMEOUT
    sim.check()  # the word was cleared
    x = torch.from_numpy(inputs.blob_image(64, 64, 3, 1)).cuda()
    (y,) = sim.simulate([x], [2.0], [1])
    sim.check()
    assert torch.isfinite(y).all() and float(y.abs().sum()) > 0
