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


def test_white_noise_prior_is_the_fourier_space_prior(monkeypatch):
    """Eq. 12's prior s^dagger S^-1 s / 2 written in Fourier space over the
    linear field (S = P(k) N^3 / V per DFT mode, k != 0) plus the mean mode
    of the white noise (which the data never see) equals the posterior's
    prior term w^T w / 2 (Parseval over the half spectrum)."""
    monkeypatch.setattr(O, "POSITIONS_FP32", False)
    n, box = 8, 60.0
    stages = np.linspace(0.1, 0.4, 2)
    w = inputs.white_noise(n, 51).astype(np.float64)
    target = inputs.random_field(n, 52).astype(np.float64) * 0.1
    lin = O.linear_field(w, box, COSMO)
    nx, ny, nz = O.half_spectrum_wavenumbers(n)
    k = 2 * math.pi / box * np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        S = O.linear_pk(k, COSMO) * n ** 3 / box ** 3
    mult = np.where((nz == 0) | (nz == n // 2), 1.0, 2.0) * np.ones_like(k)
    ratio = np.zeros_like(k)
    ratio[k > 0] = (np.abs(lin) ** 2)[k > 0] / S[k > 0]
    fourier = float((mult * ratio).sum()) / n ** 3
    mean_mode = float(w.sum()) ** 2 / n ** 3
    post, gpost = O.posterior_and_grad(w, target, n, box, COSMO, stages)
    chi2, gchi2 = O.chi2_and_grad(w, target, n, box, COSMO, stages)
    assert abs((post - 0.5 * chi2) - 0.5 * (fourier + mean_mode)) < 1e-10 * post
    np.testing.assert_allclose(gpost - 0.5 * gchi2, w, atol=1e-12)
