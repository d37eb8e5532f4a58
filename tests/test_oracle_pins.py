"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, brute force on tiny inputs, invariants, independent quadrature, and
limits.  None of them needs a GPU.
"""
import math

import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

COSMO = dict(inputs.COSMO_DEFAULT)
OM = COSMO["omega_m"]


# --------------------------------------------------------------------------
# growth and FastPM factors
# --------------------------------------------------------------------------
def _heath_d1(a, om):
    """Linear growth of flat LCDM in closed integral form (Heath 1977):
    D1 propto E(a) int_0^a da' / (a' E(a'))^3."""
    from scipy.integrate import quad
    E = lambda x: math.sqrt(om / x ** 3 + 1 - om)
    val, _ = quad(lambda x: 1.0 / (x * E(x)) ** 3, 0.0, a, epsabs=0, epsrel=1e-13, limit=200)
    return E(a) * val


@pytest.mark.parametrize("om", [0.25, 0.3075, 0.35])
def test_growth_d1_matches_heath_integral(om):
    a = np.array([0.05, 0.1, 0.3, 0.55, 0.8, 1.0])
    g = O.growth(a, om)
    ref = np.array([_heath_d1(x, om) for x in a]) / _heath_d1(1.0, om)
    np.testing.assert_allclose(g["D1"], ref, rtol=2e-9)
    # f1 = dlnD/dlna against a centred difference of the closed form
    eps = 1e-5
    for x, f in zip(a[:-1], g["f1"][:-1]):
        num = (math.log(_heath_d1(x * (1 + eps), om)) - math.log(_heath_d1(x * (1 - eps), om))) / (
            math.log(1 + eps) - math.log(1 - eps))
        assert abs(f - num) < 1e-7


def test_growth_second_order_close_to_bouchet_fit():
    # D2 ~ -3/7 D1^2 Om(a)^(-1/143) (Bouchet et al. 1995), good to well below 1%
    a = np.array([0.1, 0.3, 0.6, 1.0])
    g = O.growth(a, OM)
    om_a = OM * a ** -3 / O.hubble_E(a, OM) ** 2
    fit = -3.0 / 7.0 * g["D1"] ** 2 * om_a ** (-1.0 / 143.0)
    np.testing.assert_allclose(g["D2"], fit, rtol=5e-3)
    assert np.all(g["D2"] < 0)
    # in matter domination D2 -> -3/7 D1^2 and f2 -> 2
    ge = O.growth([1e-3], OM)
    assert abs(ge["D2"][0] / (-3 / 7 * ge["D1"][0] ** 2) - 1) < 1e-6
    assert abs(ge["f2"][0] - 2.0) < 1e-6 and abs(ge["f1"][0] - 1.0) < 1e-6


def test_fastpm_factors_reproduce_linear_growth_exactly():
    """In linear theory x = D1 Psi, p = a^3 E dD1/da Psi and the force is
    1.5 Om D1 Psi: the FastPM kick/drift factors must carry this solution
    exactly from stage to stage, whatever the step size."""
    for stages in (np.linspace(0.1, 1.0, 3), np.linspace(0.1, 1.0, 11), np.array([0.2, 0.9])):
        k1, dr, k2 = O.fastpm_factors(stages, OM)
        g = O.growth(stages, OM)
        x = g["D1"][0]
        p = stages[0] ** 3 * g["E"][0] * g["dD1da"][0]
        for k in range(len(stages) - 1):
            p = p + k1[k] * 1.5 * OM * g["D1"][k]
            x = x + dr[k] * p
            p = p + k2[k] * 1.5 * OM * g["D1"][k + 1]
            assert abs(x / g["D1"][k + 1] - 1) < 1e-10
            pref = stages[k + 1] ** 3 * g["E"][k + 1] * g["dD1da"][k + 1]
            assert abs(p / pref - 1) < 1e-10


def test_kick_rate_identity():
    """g_f = 1.5 Om D1/(a^2 E) is the derivative of G_f = a^3 E dD1/da."""
    a = np.array([0.2, 0.5, 0.9])
    eps = 1e-4            # FD truncation ~1e-8; RK4 rounding noise ~3e-12 / eps
    gp = O.growth(a * (1 + eps), OM)
    gm = O.growth(a * (1 - eps), OM)
    Gf = lambda aa, g: aa ** 3 * g["E"] * g["dD1da"]
    num = (Gf(a * (1 + eps), gp) - Gf(a * (1 - eps), gm)) / (2 * eps * a)
    g0 = O.growth(a, OM)
    np.testing.assert_allclose(num, 1.5 * OM * g0["D1"] / (a ** 2 * g0["E"]), rtol=3e-7)


# --------------------------------------------------------------------------
# linear power spectrum
# --------------------------------------------------------------------------
def test_sigma8_normalisation_independent_quadrature():
    from scipy.integrate import quad
    A = O.pk_amplitude(COSMO)

    def integrand(lnk):
        k = math.exp(lnk)
        return k ** 3 * float(O.linear_pk(k, COSMO, A)) * float(O.tophat_window(8 * k)) ** 2
    val, _ = quad(integrand, math.log(1e-6), math.log(50.0), limit=500, epsrel=1e-11)
    assert abs(math.sqrt(val / (2 * math.pi ** 2)) / COSMO["sigma8"] - 1) < 2e-6


def test_eh_nowiggle_limits_and_scaling():
    T = lambda k, c=COSMO: O.eh_nowiggle_transfer(np.asarray(k, dtype=float), c)
    assert abs(T(1e-7) - 1) < 1e-5
    k = np.logspace(-4, 2, 200)
    assert np.all(np.diff(T(k)) < 0)
    # large-q asymptote T -> ln(1.8 q) / (14.2 q^2)
    c0 = dict(COSMO, omega_b=1e-12)
    om, h = c0["omega_m"], c0["h"]
    th2 = (c0["t_cmb"] / 2.7) ** 2
    kk = 1e4 * om * h / th2                      # q = 1e4 without baryons
    q = kk * th2 / (om * h)
    assert abs(T(kk, c0) * 14.2 * q * q / math.log(1.8 * q) - 1) < 2e-2
    # without baryons T depends on k only through k / (Om h)  [k in h/Mpc]
    c1 = dict(c0, omega_m=0.25)
    c2 = dict(c0, omega_m=0.35)
    kk = np.logspace(-3, 1, 30)
    np.testing.assert_allclose(T(kk, c1), T(kk * 0.35 / 0.25, c2), rtol=1e-10)
    c3 = dict(c0, h=0.6)
    np.testing.assert_allclose(T(kk, c0), T(kk * 0.6 / c0["h"], c3), rtol=1e-10)


def test_linear_field_power_matches_input_spectrum():
    n, box = 32, 100.0
    acc = None
    nseed = 48
    for s in range(nseed):
        lk = O.linear_field(inputs.white_noise(n, 1000 + s), box, COSMO)
        assert lk[0, 0, 0] == 0
        delta = np.fft.irfftn(lk, s=(n, n, n), axes=(0, 1, 2))
        k, pk, cnt = O.power_spectrum(delta, box)
        acc = pk if acc is None else acc + pk
    pk_mean = acc / nseed
    # expected: the input P averaged over the modes of each bin
    nx, ny, nz = O.half_spectrum_wavenumbers(n)
    kmag = 2 * math.pi / box * np.sqrt((nx ** 2 + ny ** 2 + nz ** 2).astype(float))
    with np.errstate(divide="ignore"):
        pin = O.linear_pk(kmag, COSMO)
    j, w, _ = O._bin_weights(n)
    sel = (j >= 1) & (j <= n // 2)
    exp_ = np.bincount(j[sel], weights=(w * pin)[sel], minlength=n // 2 + 1)[1:] / cnt
    sigma = exp_ * np.sqrt(2.0 / cnt / nseed)        # Gaussian field: var |d|^2 = P^2
    assert np.all(np.abs(pk_mean - exp_) < 4 * sigma)


# --------------------------------------------------------------------------
# LPT
# --------------------------------------------------------------------------
def _g(w):
    return (8 * math.sin(w) - math.sin(2 * w)) / 6


def test_lpt_plane_wave_is_zeldovich():
    n, j, A = 32, 3, 0.01
    w = 2 * math.pi * j / n
    q = np.arange(n)
    delta = A * np.cos(w * q)[:, None, None] * np.ones((n, n, n))
    psi1, psi2 = O.lpt_fields(np.fft.rfftn(delta))
    expect_x = -A * _g(w) / w ** 2 * np.sin(w * q)[:, None, None] * np.ones((n, n, n))
    np.testing.assert_allclose(psi1[0], expect_x, atol=1e-15)
    assert np.abs(psi1[1:]).max() < 1e-15
    assert np.abs(psi2).max() < 1e-15


def test_lpt_two_orthogonal_waves_second_order_closed_form():
    n, j, A, B = 32, 2, 0.3, 0.2
    w = 2 * math.pi * j / n
    q = np.arange(n)
    qx = q[:, None, None] * np.ones((n, n, n))
    qy = q[None, :, None] * np.ones((n, n, n))
    delta = A * np.cos(w * qx) + B * np.cos(w * qy)
    psi1, psi2 = O.lpt_fields(np.fft.rfftn(delta))
    g = _g(w)
    # phi_xx = g^2/w^2 A cos(w qx), phi_yy likewise, phi_xy = 0
    c = 0.5 * A * B * (g * g / (w * w)) ** 2
    sp, sm = np.sin(w * (qx + qy)), np.sin(w * (qx - qy))
    ex = c * g / (2 * w * w) * (sp + sm)
    ey = c * g / (2 * w * w) * (sp - sm)
    np.testing.assert_allclose(psi2[0], ex, atol=1e-14)
    np.testing.assert_allclose(psi2[1], ey, atol=1e-14)
    assert np.abs(psi2[2]).max() < 1e-14


def test_lpt_momentum_and_units():
    n, nc = 16, 32
    lk = O.linear_field(inputs.white_noise(n, 5), 100.0, COSMO)
    dx, p = O.lpt(lk, nc, 0.1, COSMO)
    psi1, psi2 = O.lpt_fields(lk)
    g = O.growth([0.1], OM)
    r = nc / n
    np.testing.assert_allclose(dx, ((g["D1"][0] * psi1 + g["D2"][0] * psi2) * r).reshape(3, -1), atol=1e-14)
    # p = a^3 E dx/da: check by a finite difference in a of the displacement
    e = 1e-6
    d_hi, _ = O.lpt(lk, nc, 0.1 * (1 + e), COSMO)
    d_lo, _ = O.lpt(lk, nc, 0.1 * (1 - e), COSMO)
    dxda = (d_hi - d_lo) / (0.2 * e)
    np.testing.assert_allclose(p, 0.1 ** 3 * g["E"][0] * dxda, rtol=1e-6, atol=1e-12)


# --------------------------------------------------------------------------
# paint / keys / sort / readout
# --------------------------------------------------------------------------
def _brute_paint(dx, np_, nc):
    rho = np.zeros((nc, nc, nc))
    m = (nc / np_) ** 3
    r = nc // np_
    for i in range(np_ ** 3):
        q = [(i // (np_ * np_)) * r, ((i // np_) % np_) * r, (i % np_) * r]
        pos = [q[d] + float(dx[d, i]) for d in range(3)]
        base = [math.floor(x) for x in pos]
        t = [pos[d] - base[d] for d in range(3)]
        for bx in (0, 1):
            for by in (0, 1):
                for bz in (0, 1):
                    wgt = (t[0] if bx else 1 - t[0]) * (t[1] if by else 1 - t[1]) * (t[2] if bz else 1 - t[2])
                    rho[(base[0] + bx) % nc, (base[1] + by) % nc, (base[2] + bz) % nc] += m * wgt
    return rho


@pytest.mark.parametrize("np_,nc", [(4, 4), (4, 8)])
def test_paint_matches_brute_force(np_, nc):
    dx = inputs.random_displacements(np_, 2.5, 3)
    np.testing.assert_allclose(O.paint(dx, np_, nc), _brute_paint(dx, np_, nc), atol=1e-12)


def test_paint_mass_and_lattice():
    for np_, nc in ((16, 16), (8, 16)):
        dx = inputs.random_displacements(np_, 4.0, 7)
        assert abs(O.paint(dx, np_, nc).sum() - nc ** 3) < 1e-9 * nc ** 3
    rho = O.paint(np.zeros((3, 16 ** 3), np.float32), 16, 16)
    np.testing.assert_allclose(rho, 1.0, atol=0)
    rho = O.paint(np.zeros((3, 8 ** 3), np.float32), 8, 16)
    assert np.all(rho[::2, ::2, ::2] == 8.0) and rho.sum() == 16 ** 3


def test_single_particle_weights_closed_form():
    dx = np.zeros((3, 1), np.float32)
    dx[:, 0] = [0.25, -0.5, 1.75]
    rho = O.paint(dx, 1, 16)
    # base cell (0, -1, 1) -> wraps to (0, 15, 1); fractions (0.25, 0.5, 0.75)
    assert rho[0, 15, 1] / 4096 == pytest.approx(0.75 * 0.5 * 0.25)
    assert rho[1, 0, 2] / 4096 == pytest.approx(0.25 * 0.5 * 0.75)
    assert np.count_nonzero(rho) == 8


def test_keys_and_stable_order_brute_force():
    np_, nc = 8, 32
    dx = inputs.random_displacements(np_, 6.0, 11)
    cell, _ = O.cic_cells(dx, np_, nc)
    keys = O.cell_keys(cell, nc)
    for i in range(0, np_ ** 3, 37):
        c = [int(cell[d, i]) for d in range(3)]
        nt = nc // 16
        tile = ((c[0] // 16) * nt + c[1] // 16) * nt + c[2] // 16
        local = ((c[0] % 16) * 16 + c[1] % 16) * 16 + c[2] % 16
        assert keys[i] == tile * 4096 + local
        q = [(i // 64) * 4, ((i // 8) % 8) * 4, (i % 8) * 4]
        assert c == [(q[d] + math.floor(float(dx[d, i]))) % nc for d in range(3)]
    order = O.sort_order(keys)
    ref = sorted(range(np_ ** 3), key=lambda i: (int(keys[i]), i))
    assert list(order) == ref


def test_paint_readout_adjointness():
    np_, nc = 8, 16
    dx = inputs.random_displacements(np_, 3.0, 2)
    F = inputs.random_field(nc, 9).astype(np.float64)
    lhs = float((O.paint(dx, np_, nc) * F).sum())
    m = (nc / np_) ** 3
    rhs = m * float(O.readout(F[None], dx, np_, nc).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_readout_of_linear_field_is_exact():
    np_, nc = 8, 16
    dx = (inputs.random_displacements(np_, 1.0, 4) * 0.3).astype(np.float32)
    x = np.arange(nc, dtype=float)
    F = np.broadcast_to(0.5 + 0.25 * x[None, :, None], (nc, nc, nc))
    out = O.readout(np.ascontiguousarray(F)[None], dx, np_, nc)[0]
    cell, t = O.cic_cells(dx, np_, nc)
    pos_y = cell[1] + t[1]
    inside = (cell[1] < nc - 1)
    np.testing.assert_allclose(out[inside], 0.5 + 0.25 * pos_y[inside], rtol=1e-14)


# --------------------------------------------------------------------------
# force
# --------------------------------------------------------------------------
def test_zero_force_on_unperturbed_lattice():
    for np_, nc in ((16, 16), (8, 16)):
        f = O.particle_force(np.zeros((3, np_ ** 3), np.float32), np_, nc, OM)
        assert np.abs(f).max() < 1e-12


def test_force_plane_wave_closed_form():
    n, j, A = 16, 3, 0.02
    w = 2 * math.pi * j / n
    x = np.arange(n)
    delta = A * np.cos(w * x)[None, None, :] * np.ones((n, n, n))     # along z
    F = O.force_from_delta(delta, OM)
    expect = -1.5 * OM * A * _g(w) / w ** 2 * np.sin(w * x)[None, None, :]
    np.testing.assert_allclose(F[2], np.broadcast_to(expect, (n, n, n)), atol=1e-15)
    assert np.abs(F[:2]).max() < 1e-15


def test_force_matches_brute_force_dft():
    n = 6
    delta = inputs.random_field(n, 17).astype(np.float64)
    delta -= delta.mean()
    F = O.force_from_delta(delta, OM)
    idx = np.arange(n)
    xs = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), 0).reshape(3, -1)
    out = np.zeros((3, n ** 3))
    for ks in xs.T:
        kv = np.where(ks >= n // 2, ks - n, ks) if n % 2 == 0 else ks
        if not kv.any():
            continue
        wv = 2 * math.pi * kv / n
        ph = np.exp(-1j * (wv[:, None] * xs).sum(0))
        dk = (delta.reshape(-1) * ph).sum()
        k2 = float((wv ** 2).sum())
        for d in range(3):
            gd = 0.0 if kv[d] == -n // 2 else _g(wv[d])
            out[d] += (1j * gd * 1.5 * OM * dk / k2 * np.conj(ph)).real / n ** 3
    np.testing.assert_allclose(F.reshape(3, -1), out, atol=1e-13)


def test_force_is_four_point_difference_of_potential():
    """Eq. 5's g(w) = (8 sin w - sin 2w)/6 is the symbol of the real-space
    difference [8 (f(x+1) - f(x-1)) - (f(x+2) - f(x-2))] / 12, so the force
    equals that stencil applied to phi = IFFT(1.5 Om delta / |w|^2) on each
    axis (the form the CUDA path evaluates); Nyquist needs no special case."""
    n = 12
    delta = inputs.random_field(n, 23).astype(np.float64)
    k = 2 * math.pi * np.fft.fftfreq(n)
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[0, 0, 0] = 1.0
    dk = np.fft.fftn(delta) / k2
    dk[0, 0, 0] = 0.0
    phi = np.fft.ifftn(1.5 * OM * dk).real
    F = O.force_from_delta(delta, OM)
    for d in range(3):
        r = lambda s: np.roll(phi, -s, axis=d)        # r(s)[x] = phi[x + s]
        stencil = (8 * (r(1) - r(-1)) - (r(2) - r(-2))) / 12
        np.testing.assert_allclose(F[d], stencil, atol=1e-13)


def test_lpt_fields_are_real_space_differences_of_one_potential():
    """The 2LPT operators of the oracle (spectral g_i g_j / |w|^2 and
    i g_d / |w|^2) equal real-space four-point differences of
    psi = IFFT(delta_L / |w|^2): phi_ij = -D_i D_j psi, Psi1_d = D_d psi, and
    Psi2_d = D_d phi2 with phi2 = -IFFT(S(k) / |w|^2) -- the form the CUDA path
    evaluates for power-of-two lattices."""
    n, box = 16, 100.0
    lk = O.linear_field(inputs.white_noise(n, 29), box, COSMO)
    psi1, psi2 = O.lpt_fields(lk)
    k = 2 * math.pi * np.fft.fftfreq(n)
    kz = 2 * math.pi * np.fft.rfftfreq(n)
    KX, KY, KZ = np.meshgrid(k, k, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    inv = 1.0 / k2
    inv[0, 0, 0] = 0.0
    psi = np.fft.irfftn(lk * inv, s=(n, n, n), axes=(0, 1, 2))

    def D(f, ax):
        r = lambda s: np.roll(f, -s, axis=ax)
        return (8 * (r(1) - r(-1)) - (r(2) - r(-2))) / 12

    ph = {(i, j): -D(D(psi, i), j) for i in range(3) for j in range(i, 3)}
    S = (ph[0, 0] * ph[1, 1] + ph[0, 0] * ph[2, 2] + ph[1, 1] * ph[2, 2]
         - ph[0, 1] ** 2 - ph[0, 2] ** 2 - ph[1, 2] ** 2)
    phi2 = -np.fft.irfftn(np.fft.rfftn(S) * inv, s=(n, n, n), axes=(0, 1, 2))
    scale = np.abs(psi1).max()
    for d in range(3):
        np.testing.assert_allclose(psi1[d], D(psi, d), atol=1e-12 * scale)
        np.testing.assert_allclose(psi2[d], D(phi2, d), atol=1e-12 * max(np.abs(psi2).max(), 1e-30))


def _ewald_force(r, L, m, om, alpha=None):
    """Periodic point-mass acceleration at displacement r from the source,
    for lap phi = 1.5 Om (rho - mean), by Ewald summation."""
    from scipy.special import erfc
    alpha = alpha or 2.4 / L
    out = np.zeros(3)
    rng = range(-3, 4)
    for i in rng:
        for j in rng:
            for k in rng:
                v = r + L * np.array([i, j, k])
                d = np.linalg.norm(v)
                out -= v / d * (erfc(alpha * d) / d ** 2 + 2 * alpha / math.sqrt(math.pi) * math.exp(-(alpha * d) ** 2) / d)
    V = L ** 3
    kr = range(-10, 11)
    for i in kr:
        for j in kr:
            for k in kr:
                if i == j == k == 0:
                    continue
                kv = 2 * math.pi / L * np.array([i, j, k])
                k2 = kv @ kv
                out -= 4 * math.pi / V * kv / k2 * math.exp(-k2 / (4 * alpha ** 2)) * math.sin(kv @ r)
    return 1.5 * om * m / (4 * math.pi) * out


def test_ewald_reference_is_self_consistent():
    r = np.array([3.3, -1.2, 5.0])
    a = _ewald_force(r, 32.0, 1.0, OM, alpha=2.0 / 32)
    b = _ewald_force(r, 32.0, 1.0, OM, alpha=3.0 / 32)
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("sep", [5.3, 8.6, 12.1])
def test_pm_pair_force_matches_ewald(sep):
    nc = 48
    rng = np.random.default_rng(int(sep * 10))
    x1 = np.array([10.3, 20.7, 5.45])
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    x2 = x1 + sep * u
    pos = np.stack([x1, x2], 1)
    cell = np.floor(pos).astype(np.int64) % nc
    t = pos - np.floor(pos)
    m = 1.0
    rho = O.paint_cells(cell, t, np.array([m, m]), nc)
    F = O.force_from_delta(rho - rho.mean(), OM)
    f = O.readout_cells(F, cell, t)
    ref1 = _ewald_force(x1 - x2, nc, m, OM)
    rel = np.linalg.norm(f[:, 0] - ref1) / np.linalg.norm(ref1)
    assert rel < 0.06, rel
    np.testing.assert_allclose(f[:, 0], -f[:, 1], atol=1e-14)       # Newton's third law


# --------------------------------------------------------------------------
# time integration
# --------------------------------------------------------------------------
def _plane_wave_ic(n, amp, a0):
    """Zel'dovich plane wave along x: Psi_x = amp sin(2 pi q_x / n) (cells).

    All particles are also shifted by +1/2 cell along x.  A uniform shift
    exerts no force, and it keeps sub-cell displacements of either sign on
    one side of the mesh nodes: with particles exactly on nodes, CIC of a
    displacement that changes sign is one-sided (a +-1/2-cell shift of the
    density), an O(k x0) artefact of the lattice, not of the integrator."""
    g = O.growth([a0], OM)
    q = np.arange(n ** 3) // (n * n)
    psi = np.zeros((3, n ** 3))
    psi[0] = amp * np.sin(2 * math.pi * q / n)
    dx = g["D1"][0] * psi
    dx[0] += 0.5
    p = a0 ** 2 * g["E"][0] * g["f1"][0] * g["D1"][0] * psi
    return psi, dx, p


def test_kdk_plane_wave_follows_zeldovich_growth():
    n = 32
    psi, dx, p = _plane_wave_ic(n, 0.3, 0.1)
    dxn, pn = O.kdk(dx, p, np.linspace(0.1, 1.0, 6), n, n, OM, round_to_float32=False)
    # D1(1) = 1: final displacement equals Psi up to the mesh transfer of
    # CIC paint+readout and the FD gradient at this wavelength (~2 %)
    sel = np.abs(psi[0]) > 0.5 * 0.3
    ratio = (dxn[0][sel] - 0.5) / psi[0][sel]
    assert np.all(np.abs(ratio - 1) < 3e-2), (ratio.min(), ratio.max())
    assert np.abs(dxn[1:]).max() < 1e-12
    # velocities follow p = a^2 E f1 D1 Psi at a = 1
    g = O.growth([1.0], OM)
    pref = g["E"][0] * g["f1"][0] * psi[0][sel]
    assert np.all(np.abs(pn[0][sel] / pref - 1) < 5e-2)


def test_kdk_step_count_independent_in_linear_regime():
    n = 16
    psi, dx, p = _plane_wave_ic(n, 0.05, 0.1)
    a5, _ = O.kdk(dx, p, np.linspace(0.1, 1.0, 6), n, n, OM, round_to_float32=False)
    a40, _ = O.kdk(dx, p, np.linspace(0.1, 1.0, 41), n, n, OM, round_to_float32=False)
    sel = np.abs(psi[0]) > 0.025
    np.testing.assert_allclose(a5[0][sel] - 0.5, a40[0][sel] - 0.5, rtol=2e-3)


# --------------------------------------------------------------------------
# power spectrum
# --------------------------------------------------------------------------
def test_power_single_cosine_closed_form():
    n, L, j, A = 16, 50.0, 3, 0.7
    x = np.arange(n)
    field = A * np.cos(2 * math.pi * j * x / n)[:, None, None] * np.ones((n, n, n))
    k, P, cnt = O.power_spectrum(field, L)
    expect = L ** 3 * A * A / (2 * cnt[j - 1])
    assert P[j - 1] == pytest.approx(expect, rel=1e-12)
    others = np.delete(P, j - 1)
    assert np.abs(others).max() < 1e-20 * expect


def test_power_mode_counts_brute_force():
    n = 12
    _, _, cnt = O.power_spectrum(np.zeros((n, n, n)), 1.0)
    ref = np.zeros(n // 2)
    f = np.fft.fftfreq(n, 1.0 / n)
    for a in f:
        for b in f:
            for c in f:
                r = math.sqrt(a * a + b * b + c * c)
                jj = int(math.floor(r + 0.5))
                if 1 <= jj <= n // 2:
                    ref[jj - 1] += 1
    # the full-grid count has each mode once, except that the Nyquist plane
    # n_z = -n/2 appears only as +n/2 in the half spectrum (counted once)
    np.testing.assert_array_equal(cnt, ref)


def test_transfer_and_cross_correlation_identities():
    f = inputs.random_field(16, 3).astype(float)
    _, pa, _ = O.power_spectrum(f, 10.0)
    _, pab, _ = O.power_spectrum(f, 10.0, other=2 * f)
    _, pb, _ = O.power_spectrum(2 * f, 10.0)
    np.testing.assert_allclose(O.transfer_function(pb, pa), 2.0, rtol=1e-12)
    np.testing.assert_allclose(O.cross_correlation(pab, pa, pb), 1.0, rtol=1e-12)
