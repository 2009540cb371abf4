"""Pins of oracle.mlp."""
import numpy as np

from oracle import mlp


def test_identity_layers():
    v = np.abs(np.random.default_rng(9).normal(size=(5, 33)))
    eye = [(np.eye(33), np.zeros(33))] * 3
    assert np.array_equal(mlp.forward(v, eye), v)


def test_layers_elementwise():
    rng = np.random.default_rng(10)
    layers = [(rng.normal(size=(4, 3)), rng.normal(size=4)), (rng.normal(size=(2, 4)), rng.normal(size=2))]
    v = rng.normal(size=3)
    h = [max(0.0, sum(layers[0][0][o, i] * v[i] for i in range(3)) + layers[0][1][o]) for o in range(4)]
    out = [sum(layers[1][0][o, i] * h[i] for i in range(4)) + layers[1][1][o] for o in range(2)]
    assert np.allclose(mlp.forward(v, layers), out, atol=1e-14)
