"""CPU checks of the C ABI: the library loads, exports every declared symbol,
validates arguments before touching the GPU, and its host-side FP64 set-up
agrees with the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_11627_gb300 import p2s

    if not os.path.exists(p2s.LIB_PATH):
        from paper_2107_11627_gb300 import build

        build.build()
    return p2s.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "p2s.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(p2s_[a-z_]+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    from paper_2107_11627_gb300 import p2s

    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
        assert s in p2s._SIGS, f"binding lacks {s}"


def test_status_strings(lib):
    assert lib.p2s_status_string(0) == b"ok"
    assert lib.p2s_status_string(1) == b"invalid argument"


def test_noll_covariance_matches_oracle(lib):
    from oracle import noll
    from paper_2107_11627_gb300 import p2s

    R = p2s.noll_covariance(36)
    ref = noll.noll_cov(36)
    assert np.max(np.abs(R - ref)) < 1e-14
    assert lib.p2s_noll_covariance(2, None) == p2s.P2S_EINVAL


def test_create_rejects_bad_shapes_without_gpu(lib):
    from paper_2107_11627_gb300 import p2s

    H = np.zeros((4, 9))
    ell = np.array([16.0])
    b = p2s.p2s_basis(H.ctypes.data_as(C.POINTER(C.c_double)), 4, 3, 3)
    dims = (C.c_int * 2)(33, 4)
    W = np.zeros((4, 33))
    bb = np.zeros(4)
    Wp = (C.POINTER(C.c_double) * 1)(W.ctypes.data_as(C.POINTER(C.c_double)))
    bp = (C.POINTER(C.c_double) * 1)(bb.ctypes.data_as(C.POINTER(C.c_double)))
    m = p2s.p2s_mlp(1, dims, Wp, bp)
    cp = p2s.p2s_corr_params(8, 1, ell.ctypes.data_as(C.POINTER(C.c_double)), -1, 0.0)
    ctx = C.c_void_p()
    even = p2s.p2s_basis(H.ctypes.data_as(C.POINTER(C.c_double)), 4, 2, 3)
    assert lib.p2s_create(C.byref(even), C.byref(m), C.byref(cp), 0, 0, C.byref(ctx)) == p2s.P2S_EINVAL
    badk = p2s.p2s_basis(H.ctypes.data_as(C.POINTER(C.c_double)), 5, 3, 3)
    assert lib.p2s_create(C.byref(badk), C.byref(m), C.byref(cp), 0, 0, C.byref(ctx)) == p2s.P2S_EINVAL
    cp0 = p2s.p2s_corr_params(0, 1, ell.ctypes.data_as(C.POINTER(C.c_double)), -1, 0.0)
    assert lib.p2s_create(C.byref(b), C.byref(m), C.byref(cp0), 0, 0, C.byref(ctx)) == p2s.P2S_EINVAL
    assert ctx.value is None
    assert b"anchor_spacing" in lib.p2s_last_error()


def test_stage_calls_reject_null(lib):
    from paper_2107_11627_gb300 import p2s

    assert lib.p2s_stage_noise(None, 0, 0, 4, 4, None, None) == p2s.P2S_EINVAL
    assert lib.p2s_simulate(None, None, 0, None, None, None, None) == p2s.P2S_EINVAL


def test_product_basis_builder_matches_oracle():
    from oracle import psf
    from paper_2107_11627_gb300 import basis, inputs

    z, dr0 = inputs.dictionary_draws(600, 35, (0.5, 6.0), 2021)
    Ho, _ = psf.make_basis(z, dr0, K=12, taps=9)
    Hp = basis.build_basis(12, 9, 600, cache=False)
    assert np.max(np.abs(Ho - Hp)) < 1e-12
