"""Pins of the oracle's adjoint: dot-product identities for the linear maps
and central finite differences (in FP64, positions not rounded to float32)
for the nonlinear ones.  A dropped term, a wrong sign or a transposed
operand in any reverse step breaks one of these."""
import math

import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

COSMO = dict(inputs.COSMO_DEFAULT)
OM = COSMO["omega_m"]


@pytest.fixture
def fp64_positions(monkeypatch):
    monkeypatch.setattr(O, "POSITIONS_FP32", False)


def _rng(seed):
    return np.random.default_rng(seed)


def test_force_adj_dot_product():
    n = 16
    r = _rng(1)
    u = r.standard_normal((n, n, n))
    v = r.standard_normal((3, n, n, n))
    lhs = float((O.force_from_delta(u, OM) * v).sum())
    rhs = float((u * O.force_adj(v, OM)).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_readout_adj_mesh_part_dot_product():
    np_, nc = 8, 16
    dx = inputs.random_displacements(np_, 3.0, 4)
    r = _rng(2)
    F = r.standard_normal((3, nc, nc, nc))
    gf = r.standard_normal((3, np_ ** 3))
    lhs = float((O.readout(F, dx, np_, nc) * gf).sum())
    g_F, _ = O.readout_adj(F, dx, gf, np_, nc)
    rhs = float((F * g_F).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_paint_adj_and_readout_position_part_by_finite_differences(fp64_positions):
    np_, nc = 8, 16
    r = _rng(3)
    dx = r.uniform(-3, 3, size=(3, np_ ** 3))
    u = r.standard_normal((3, np_ ** 3))
    g_rho = r.standard_normal((nc, nc, nc))
    eps = 1e-7
    jd = (O.paint(dx + eps * u, np_, nc) - O.paint(dx - eps * u, np_, nc)) / (2 * eps)
    lhs = float((jd * g_rho).sum())
    rhs = float((u * O.paint_adj(g_rho, dx, np_, nc)).sum())
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)
    F = r.standard_normal((3, nc, nc, nc))
    gf = r.standard_normal((3, np_ ** 3))
    jr = (O.readout(F, dx + eps * u, np_, nc) - O.readout(F, dx - eps * u, np_, nc)) / (2 * eps)
    _, g_dx = O.readout_adj(F, dx, gf, np_, nc)
    assert abs(float((jr * gf).sum()) - float((u * g_dx).sum())) < 1e-6 * abs(float((jr * gf).sum()))


def test_particle_force_adj_by_finite_differences(fp64_positions):
    np_, nc = 8, 16
    r = _rng(5)
    dx = r.uniform(-2, 2, size=(3, np_ ** 3))
    u = r.standard_normal((3, np_ ** 3))
    gf = r.standard_normal((3, np_ ** 3))
    eps = 1e-7
    jf = (O.particle_force(dx + eps * u, np_, nc, OM) - O.particle_force(dx - eps * u, np_, nc, OM)) / (2 * eps)
    lhs = float((jf * gf).sum())
    rhs = float((u * O.particle_force_adj(dx, gf, np_, nc, OM)).sum())
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)


def test_lpt_adj_by_central_differences():
    """lpt is quadratic in the linear field, so central differences are exact
    up to rounding."""
    n, nc, box = 16, 32, 100.0
    lk = O.linear_field(inputs.white_noise(n, 8), box, COSMO)
    r = _rng(6)
    du = r.standard_normal((n, n, n)) * 1e-3           # a real-field perturbation of delta_L
    dk = np.fft.rfftn(du)
    gdx = r.standard_normal((3, n ** 3))
    gp = r.standard_normal((3, n ** 3))
    for order in (1, 2):
        p_dx, p_p = O.lpt(lk + dk, nc, 0.1, COSMO, order)
        m_dx, m_p = O.lpt(lk - dk, nc, 0.1, COSMO, order)
        lhs = float(((p_dx - m_dx) * gdx).sum() + ((p_p - m_p) * gp).sum()) / 2
        G = O.lpt_adj(lk, nc, 0.1, COSMO, gdx, gp, order)
        # G = FFT(g) with g the real-field cotangent: the pairing is sum du * g
        rhs = float((du * np.fft.irfftn(G, s=(n, n, n), axes=(0, 1, 2))).sum())
        assert abs(lhs - rhs) < 1e-8 * abs(lhs), (order, lhs, rhs)


def test_linear_field_adj_dot_product():
    n, box = 16, 100.0
    r = _rng(7)
    w = r.standard_normal((n, n, n))
    g = r.standard_normal((n, n, n))
    dl = np.fft.irfftn(O.linear_field(w, box, COSMO), s=(n, n, n), axes=(0, 1, 2))
    lhs = float((dl * g).sum())
    rhs = float((w * O.linear_field_adj(np.fft.rfftn(g), box, COSMO)).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_kdk_adj_by_finite_differences(fp64_positions):
    np_, nc = 8, 16
    stages = np.linspace(0.2, 0.6, 3)
    r = _rng(9)
    dx0 = r.uniform(-1, 1, size=(3, np_ ** 3))
    p0 = r.standard_normal((3, np_ ** 3)) * 0.3
    gdx = r.standard_normal((3, np_ ** 3))
    gp = r.standard_normal((3, np_ ** 3))
    u = r.standard_normal((3, np_ ** 3))
    w = r.standard_normal((3, np_ ** 3))
    eps = 1e-7

    def run(x, p):
        rec = []
        xn, pn = O.kdk(x, p, stages, np_, nc, OM, round_to_float32=False, record=rec)
        return xn, pn, [a for a, _ in rec] + [xn]

    xp, pp, _ = run(dx0 + eps * u, p0 + eps * w)
    xm, pm, _ = run(dx0 - eps * u, p0 - eps * w)
    lhs = float(((xp - xm) * gdx).sum() + ((pp - pm) * gp).sum()) / (2 * eps)
    _, _, xs = run(dx0, p0)
    g0x, g0p = O.kdk_adj(xs, stages, gdx, gp, np_, nc, OM)
    rhs = float((u * g0x).sum() + (w * g0p).sum())
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)


def test_full_chain_gradient_by_finite_differences(fp64_positions):
    """d chi^2 / d w on 16 random voxels, central differences in FP64."""
    n, nc, box = 16, 16, 100.0
    stages = np.linspace(0.1, 1.0, 3)
    w = inputs.white_noise(n, 1).astype(np.float64)
    target = _rng(11).standard_normal((nc, nc, nc)) * 0.5

    def loss(wv):
        lk = O.linear_field(wv, box, COSMO)
        dx0, p0 = O.lpt(lk, nc, stages[0], COSMO)
        dx, _ = O.kdk(dx0, p0, stages, n, nc, OM, round_to_float32=False)
        return O.chi2(O.paint(dx, n, nc), target)[0]

    L0, g = O.chi2_and_grad(w, target, nc, box, COSMO, stages)
    assert abs(L0 - loss(w)) < 1e-12 * L0
    idx = _rng(12).choice(n ** 3, size=16, replace=False)
    eps = 1e-4
    fd = []
    for i in idx:
        e = np.zeros(n ** 3)
        e[i] = eps
        e = e.reshape(n, n, n)
        fd.append((loss(w + e) - loss(w - e)) / (2 * eps))
    fd = np.array(fd)
    ad = g.reshape(-1)[idx]
    assert np.linalg.norm(ad - fd) < 1e-5 * np.linalg.norm(fd)
