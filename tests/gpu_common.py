"""Shared fixtures for the GPU parity tests: bases and weights built by the
oracle from seeded inputs (so no expected value comes from the CUDA path)."""
import functools

import numpy as np

import oracle
from paper_2107_11627_gb300 import inputs

TOL_FIELD = 1e-6  # fields and warp, relative L2 vs FP64
TOL_FP32 = 1e-5   # plain FP32 path
TOL_BF16 = 2e-3
TOL_FP8 = 1e-2


@functools.lru_cache(maxsize=None)
def basis(K: int, taps: int, n_dict: int):
    z, dr0 = inputs.dictionary_draws(n_dict, 35, (0.5, 6.0), 2021)
    H, _ = oracle.psf.make_basis(z, dr0, K=K, taps=taps)
    return H


def cfg1():
    """64x64 grey block image, K=20 of 17x17 taps from 2000 PSFs, MLP 33-64-64-20, D/r0 = 2."""
    return dict(H=basis(20, 17, 2000), taps=(17, 17), layers=inputs.mlp_weights([33, 64, 64, 20], 42))


def cfg2():
    """K=100 of 33x33 taps, MLP 33-128-128-100 (dictionary reduced to 4000 PSFs for test speed)."""
    return dict(H=basis(100, 33, 4000), taps=(33, 33), layers=inputs.mlp_weights([33, 128, 128, 100], 42))


# Element-wise bound: every |a - ref| <= MAXABS_FACTOR * tol * max|ref|.  The relative-L2
# tolerance bounds the rms error; the tail of the element errors of a correct kernel sits a
# few rms above it, while one wrong tile or border strip shows up as an error of the order
# of the values themselves, far above this bound.
MAXABS_FACTOR = 10.0

# (test, what, rel_l2, max_abs, max_abs_bound, tol) of every comparison, printed at the end of
# the run by conftest.py so that the log's tail carries the figures.
RECORDS: list = []


def rel(a, b):
    return oracle.frame.rel_l2(a, b)


def close(a, ref, tol, what=""):
    """Assert relative L2 < tol and the element-wise bound above; record both figures."""
    import os

    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert a.shape == ref.shape, (what, a.shape, ref.shape)
    r = rel(a, ref)
    mx = float(np.max(np.abs(a - ref))) if a.size else 0.0
    bound = MAXABS_FACTOR * tol * (float(np.max(np.abs(ref))) if ref.size else 0.0)
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0].split("::")[-1]
    RECORDS.append((test, str(what), r, mx, bound, tol))
    assert np.all(np.isfinite(a)), (what, "non-finite output")
    assert r < tol, (what, "rel_l2", r, tol)
    assert mx <= bound, (what, "max_abs", mx, bound)
    return r, mx
