"""Pins of oracle.philox: bit-exact against cuRAND's host Philox4_32_10 generator.

cuRAND is run as a library on the CPU (curandCreateGeneratorHost); its output
block i is Philox4x32-10 at counter (0, 0, i, 0) with key = the 64-bit seed.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import philox


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 10**6 + 17, 2**64 - 1])
def test_matches_curand_host(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    n = 256
    out = (ctypes.c_uint * n)()
    assert lib.curandGenerate(gen, out, n) == 0
    lib.curandDestroyGenerator(gen)
    ref = np.array(list(out), dtype=np.uint64).reshape(-1, 4)
    k0, k1 = philox.key_of_seed(seed)
    i = np.arange(n // 4, dtype=np.uint64)
    ours = np.stack(philox.philox4x32_10(0, 0, i, 0, k0, k1), axis=1)
    assert np.array_equal(ours, ref)


def test_stream_layout_and_uniform_range():
    w = philox.words(5, 3, 10)
    k0, k1 = philox.key_of_seed(5)
    b0 = philox.philox4x32_10(0, 3, 0, 0, k0, k1)
    b2 = philox.philox4x32_10(2, 3, 0, 0, k0, k1)
    assert [int(v) for v in w[:4]] == [int(v) for v in b0]
    assert [int(v) for v in w[8:10]] == [int(v) for v in b2[:2]]
    u = philox.uniforms(np.array([0, 2**32 - 1], dtype=np.uint64))
    assert u[0] == 0.5 * 2**-32 and u[1] == 1 - 0.5 * 2**-32


def test_normal_moments_and_independence():
    n = 400_000
    z = philox.normals(99, 0, n)
    z2 = philox.normals(99, 1, n)
    z3 = philox.normals(100, 0, n)
    se = 1 / np.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1) < 5 * np.sqrt(2) * se
    assert abs(np.mean(z**3)) < 5 * np.sqrt(15) * se
    assert abs(np.mean(z**4) - 3) < 5 * np.sqrt(96) * se
    assert abs(np.mean(z * z2)) < 5 * se
    assert abs(np.mean(z * z3)) < 5 * se
    assert abs(np.mean(z[:-1] * z[1:])) < 5 * se
