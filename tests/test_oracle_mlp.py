"""Pins of the FP64 warm-start MLP reference."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_closed_form_points():
    # GELU(z) = z Phi(z): Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (standard normal CDF).
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert mlp.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, rel=1e-15)
    assert mlp.gelu(np.array(-1.0)) == pytest.approx(-1.0 * (1 - 0.8413447460685429), rel=1e-13)
    assert mlp.gelu(np.array(8.0)) == pytest.approx(8.0, rel=1e-12)
    # derivative at 0 is Phi(0) = 1/2
    assert mlp.gelu_grad(np.array(0.0)) == 0.5


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    i, h, o, n = 5, 7, 3, 11
    params = rng.standard_normal(sum(int(np.prod(s)) for s in mlp.shapes(i, h, o))) * 0.5
    X = rng.standard_normal((n, i))
    T = rng.standard_normal((n, o))
    _, g = mlp.loss_and_grad(params, X, T, i, h, o)
    eps = 1e-6
    for q in range(params.size):
        pp, pm = params.copy(), params.copy()
        pp[q] += eps
        pm[q] -= eps
        lp, _ = mlp.loss_and_grad(pp, X, T, i, h, o)
        lm, _ = mlp.loss_and_grad(pm, X, T, i, h, o)
        fd = (lp - lm) / (2 * eps)
        assert g[q] == pytest.approx(fd, rel=1e-6, abs=1e-9), q


def test_features_hand_row():
    # Row with items 0 and 2, ratings 1 and 3, Y rows [1,2] and [3,-1]:
    # weighted mean = (1*[1,2] + 3*[3,-1]) / 4 = [2.5, -0.25]; log(1+2); mean 2.
    indptr = np.array([0, 2, 2])
    indices = np.array([0, 2], np.int32)
    values = np.array([1.0, 3.0], np.float32)
    Y = np.array([[1.0, 2.0], [9.0, 9.0], [3.0, -1.0]], np.float32)
    F = mlp.features(indptr, indices, values, Y)
    np.testing.assert_allclose(F[0], [2.5, -0.25, math.log(3.0), 2.0], rtol=1e-15)
    np.testing.assert_allclose(F[1], [0.0, 0.0, 0.0, 0.0])


def test_adam_first_step_is_signed_lr():
    # With zero state, the first bias-corrected Adam step is lr * g / (|g| + eps).
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    newp, _, _ = mlp.adam(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(newp, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
