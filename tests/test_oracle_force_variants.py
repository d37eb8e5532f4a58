"""Pins of the oracle's force variants (Sec. 2, Eqs. 3-5): the Green's
function of Eq. 4 (the discrete Laplacian) and the exact i k gradient,
beside the default naive Green's function and Eq. 5's difference.

The expected values come from real-space stencils (np.roll) and from the
analytic derivatives of plane waves, never from the oracle's spectral
symbols; the transposes are pinned by the dot-product identity and the
accuracy by the periodic Ewald pair force.
"""
import math

import numpy as np
import pytest

from oracle import fpm_oracle as O
from test_oracle_pins import OM, _ewald_force

VARIANTS = [(g, d) for g in O.GREENS for d in O.GRADIENTS]


def _d4(f, axis):
    """Eq. 5's four-point difference in real space, cell units."""
    r = lambda k: np.roll(f, -k, axis=axis)
    return (8.0 * (r(1) - r(-1)) - (r(2) - r(-2))) / 12.0


def _lap7(f):
    """The seven-point discrete Laplacian in real space, cell units."""
    return sum(np.roll(f, 1, a) + np.roll(f, -1, a) - 2.0 * f for a in range(3))


def _plane_waves(n):
    """Three cosines with integer wave vectors below the Nyquist frequency:
    the field, its analytic Laplacian and its analytic gradient."""
    x = np.indices((n, n, n), dtype=np.float64)
    waves = [((1, 0, 0), 0.7, 0.3), ((2, -3, 1), -0.4, 1.1), ((-5, 4, 6), 0.25, -0.6)]
    phi = np.zeros((n, n, n))
    lap = np.zeros((n, n, n))
    grad = np.zeros((3, n, n, n))
    for k, amp, th in waves:
        w = 2.0 * math.pi * np.array(k, dtype=np.float64) / n
        arg = sum(w[d] * x[d] for d in range(3)) + th
        phi += amp * np.cos(arg)
        lap -= amp * float(w @ w) * np.cos(arg)
        for d in range(3):
            grad[d] -= amp * w[d] * np.sin(arg)
    return phi, lap, grad


@pytest.mark.parametrize("green,gradient", VARIANTS)
def test_variant_force_of_plane_waves(green, gradient):
    """F = -grad phi with lap phi = 1.5 Om delta: build delta from a known
    potential with the variant's Laplacian and compare F with the variant's
    derivative of that potential."""
    n = 16
    phi, lap_exact, grad_exact = _plane_waves(n)
    lap = lap_exact if green == "naive" else _lap7(phi)
    delta = lap / (1.5 * OM)
    F = O.force_from_delta(delta, OM, green, gradient)
    want = -grad_exact if gradient == "exact" else -np.stack([_d4(phi, d) for d in range(3)])
    np.testing.assert_allclose(F, want, atol=1e-12 * np.abs(want).max())


def test_discrete_green_inverts_the_seven_point_laplacian():
    """For any zero-mean potential, Eq. 4's Green's function undoes the
    seven-point Laplacian exactly (all modes, Nyquist planes included)."""
    n = 12
    rng = np.random.default_rng(7)
    phi = rng.normal(size=(n, n, n))
    phi -= phi.mean()
    F = O.force_from_delta(_lap7(phi) / (1.5 * OM), OM, "discrete", "fd4")
    want = -np.stack([_d4(phi, d) for d in range(3)])
    np.testing.assert_allclose(F, want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("green,gradient", VARIANTS)
def test_variant_force_adjoint_dot_product(green, gradient):
    n = 10
    rng = np.random.default_rng(3)
    delta = rng.normal(size=(n, n, n))
    gF = rng.normal(size=(3, n, n, n))
    lhs = float((O.force_from_delta(delta, OM, green, gradient) * gF).sum())
    rhs = float((delta * O.force_adj(gF, OM, green, gradient)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def _pair_error(sep, trial, green, gradient, nc=48):
    rng = np.random.default_rng(int(sep * 10) + 1000 * trial)
    x1 = np.array([10.3, 20.7, 5.45]) + rng.uniform(0, 1, 3)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    pos = np.stack([x1, x1 + sep * u], 1)
    cell = np.floor(pos).astype(np.int64) % nc
    t = pos - np.floor(pos)
    rho = O.paint_cells(cell, t, np.array([1.0, 1.0]), nc)
    f = O.readout_cells(O.force_from_delta(rho - rho.mean(), OM, green, gradient), cell, t)
    np.testing.assert_allclose(f[:, 0], -f[:, 1], atol=1e-14)        # Newton's third law
    ref = _ewald_force(pos[:, 0] - pos[:, 1], nc, 1.0, OM)
    return np.linalg.norm(f[:, 0] - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("green,gradient", VARIANTS)
def test_variant_pair_force_matches_ewald_at_long_range(green, gradient):
    errs = [_pair_error(sep, tr, green, gradient) for sep in (8.6, 12.1) for tr in range(3)]
    assert max(errs) < 0.05, errs


def test_fd_gradient_beats_exact_gradient_at_short_range():
    """The exact gradient's symbol jumps from pi to 0 at the Nyquist
    frequency; its real-space kernel rings, and at a few cells the pair
    force is worse than with Eq. 5's difference, whose symbol goes to 0
    smoothly."""
    fd = np.mean([_pair_error(5.3, tr, "naive", "fd4") for tr in range(4)])
    ex = np.mean([_pair_error(5.3, tr, "naive", "exact") for tr in range(4)])
    assert fd < 0.05 and ex > fd, (fd, ex)
