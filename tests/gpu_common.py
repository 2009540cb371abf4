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


def rel(a, b):
    return oracle.frame.rel_l2(a, b)
