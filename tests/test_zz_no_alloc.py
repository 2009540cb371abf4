"""The allocation-free network entry point against the allocating one.

p2s_stage_mlp_noalloc serves callers that cannot allocate device memory when
they run the network (a fixed memory budget, or a thread that must stay out of
the CUDA allocator).  It must give the same beta as p2s_stage_mlp, call after
call, although every call reuses the library's one static weight array.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it passes alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle.fields import CorrParams
from paper_2107_11627_gb300 import inputs

from gpu_common import TOL_FP32, cfg2, rel, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# Size of the library's static weight array (227 KiB of shared memory less the plain
# network kernel's 64 KiB of activation buffers, in floats).
NOALLOC_LIMIT_FLOATS = (227 * 1024 - 2 * 128 * 64 * 4) // 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _alpha(seed, h, w):
    a = oracle.fields.alpha_anchors(seed, 3.0, h, w, CorrParams(8, (16.0,))).astype(np.float32)
    full = np.zeros(a.shape[:2] + (36,), dtype=np.float32)
    full[..., 1:] = a
    return torch.from_numpy(full).cuda()


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    sim = p2s.Simulator(c["H"], c["taps"], c["layers"], anchor_spacing=8, precision="fp32")
    lib = p2s.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (seed, h, w) in enumerate([(41, 45, 70), (42, 64, 33)]):
        al = _alpha(seed, h, w)
        ref = sim.stage_mlp(h, w, al)
        out = torch.full_like(ref, float("nan"))
        st = lib.p2s_stage_mlp_noalloc(sim.ctx, h, w, C.c_void_p(al.data_ptr()), C.c_void_p(out.data_ptr()), stream)
        assert st == p2s.P2S_OK, lib.p2s_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        close(out.cpu().numpy(), ref.cpu().numpy(), TOL_FP32, call)
    sim.close()


def test_noalloc_rejects_a_weight_image_beyond_its_limit():
    from paper_2107_11627_gb300 import p2s

    c = cfg2()
    dims = [33, 128, 128, 128, 100]
    big = inputs.mlp_weights(dims, 43)
    # weights plus 4-float-padded biases: 50,276 floats, beyond the 41,728-float array
    floats = sum(i * o + ((o + 3) & ~3) for i, o in zip(dims[:-1], dims[1:]))
    assert floats == 50276 and floats > NOALLOC_LIMIT_FLOATS
    sim = p2s.Simulator(c["H"], c["taps"], big, anchor_spacing=8, precision="fp32")
    al = _alpha(43, 16, 16)
    out = torch.empty((16, 16, 100), device="cuda")
    st = p2s.lib().p2s_stage_mlp_noalloc(sim.ctx, 16, 16, C.c_void_p(al.data_ptr()), C.c_void_p(out.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == p2s.P2S_EINVAL
    assert b"allocation-free scratch" in p2s.lib().p2s_last_error()
    sim.close()
