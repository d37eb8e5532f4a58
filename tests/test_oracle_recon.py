"""Pins of the oracle's reconstruction pieces (Sec. 7.1, Eq. 12): Adam
against properties that fix it, and the posterior gradient against central
finite differences in FP64."""
import math

import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

COSMO = dict(inputs.COSMO_DEFAULT)


def test_adam_first_step_is_lr_times_sign():
    # m_hat = g and v_hat = g^2 at t = 1, so the step is lr g / (|g| + eps)
    r = np.random.default_rng(3)
    x = r.standard_normal(1000)
    g = r.standard_normal(1000)
    x1, m, v = O.adam_step(x, g, np.zeros_like(x), np.zeros_like(x), 1, lr=0.01)
    np.testing.assert_allclose(x1, x - 0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_keeps_unit_steps():
    # with a constant gradient the bias corrections make m_hat = g, v_hat = g^2 at every t
    x = np.zeros(4)
    g = np.array([2.0, -0.5, 1e-3, -7.0])
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 21):
        x, m, v = O.adam_step(x, g, m, v, t, lr=0.05, eps=0.0)
    np.testing.assert_allclose(x, -20 * 0.05 * np.sign(g), rtol=1e-12)


def test_adam_minimises_a_quadratic():
    c = np.array([1.0, -2.0, 0.5])
    x = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 3001):
        x, m, v = O.adam_step(x, x - c, m, v, t, lr=0.01)
    np.testing.assert_allclose(x, c, atol=1e-3)


def test_posterior_gradient_by_central_differences(monkeypatch):
    monkeypatch.setattr(O, "POSITIONS_FP32", False)
    n, nc, box = 8, 8, 60.0
    stages = np.linspace(0.1, 0.6, 3)
    w = inputs.white_noise(n, 41).astype(np.float64)
    target = inputs.random_field(nc, 42).astype(np.float64) * 0.1
    f, g = O.posterior_and_grad(w, target, nc, box, COSMO, stages)
    u = np.random.default_rng(43).standard_normal(w.shape)
    eps = 1e-4
    fp, _ = O.posterior_and_grad(w + eps * u, target, nc, box, COSMO, stages)
    fm, _ = O.posterior_and_grad(w - eps * u, target, nc, box, COSMO, stages)
    fd = (fp - fm) / (2 * eps)
    assert abs(fd - float((g * u).sum())) < 1e-6 * abs(fd)
