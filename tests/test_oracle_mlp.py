"""Pins for the learned-lambda network oracle (oracle/mlp.py): backward pass
against central finite differences, Adam against its closed form on one step,
GELU against known values."""
import math

import numpy as np

from oracle import mlp


def test_gelu_values():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # GELU(1) = Phi(1) = 0.8413447460685429
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array([-1.0]))[0] + 1.0 - 0.8413447460685429) < 1e-15


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(mlp.nparams()) * 0.2
    X = rng.standard_normal((7, 36))
    T = rng.standard_normal((7, 2))
    L, g = mlp.loss_and_grad(theta, X, T)
    idx = rng.choice(mlp.nparams(), 60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_adam_first_step_is_signed_lr():
    # With m = v = 0 and t = 1 the bias-corrected step is lr * g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_layout():
    al = np.arange(1, 14, dtype=float)
    be = np.arange(2, 16, dtype=float)
    ph = np.arange(3, 15, dtype=float)
    f = mlp.features(al, be, ph)
    assert f.shape == (36,)
    assert math.isclose(f[0], math.log(1 / 2)) and math.isclose(f[12], math.log(3 / 2))
    assert math.isclose(f[24], math.log(3 / 2))
