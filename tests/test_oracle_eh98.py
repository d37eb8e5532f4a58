"""Pins of the oracle's Eisenstein & Hu (1998) no-wiggle transfer function
against EH98's own physical definitions and its full transfer function.

The no-wiggle form (EH98 eqs. 26, 28-31) is a fit: its sound horizon s
(eq. 26) approximates the sound horizon at the drag epoch computed from the
physical quantities z_eq, k_eq, z_d and R (eqs. 2-6), and its small-scale
shape parameter alpha_Gamma (eq. 31) approximates the baryon suppression of
the full transfer function with acoustic oscillations (eqs. 7-24).  The full
function is written out below from those equations, independently of the
oracle, and the oracle's s and alpha_Gamma are recovered from its T(k)
alone by inverting T for q (eq. 28-29).  A mistyped coefficient in the
oracle's s, alpha_Gamma, Gamma_eff or C0 moves one of these checks by more
than its tolerance (checked by planting such typos in a copy of the oracle).
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

COSMO = dict(inputs.COSMO_DEFAULT)


# --------------------------------------------------------------------------
# EH98's physical scales and full transfer function (eqs. 2-24), k in 1/Mpc
# --------------------------------------------------------------------------
def eh98_scales(cosmo):
    om, ob, h = cosmo["omega_m"], cosmo["omega_b"], cosmo["h"]
    th = cosmo["t_cmb"] / 2.7
    wm, wb = om * h * h, ob * h * h
    z_eq = 2.50e4 * wm * th ** -4                                  # eq. 2
    k_eq = 7.46e-2 * wm * th ** -2                                 # eq. 3, 1/Mpc
    b1 = 0.313 * wm ** -0.419 * (1.0 + 0.607 * wm ** 0.674)        # eq. 4
    b2 = 0.238 * wm ** 0.223
    z_d = 1291.0 * wm ** 0.251 / (1.0 + 0.659 * wm ** 0.828) * (1.0 + b1 * wb ** b2)

    def R(z):                                                      # eq. 5
        return 31.5 * wb * th ** -4 * (z / 1.0e3) ** -1

    R_d, R_eq = R(z_d), R(z_eq)
    s = (2.0 / (3.0 * k_eq) * math.sqrt(6.0 / R_eq)                # eq. 6, Mpc
         * math.log((math.sqrt(1.0 + R_d) + math.sqrt(R_d + R_eq)) / (1.0 + math.sqrt(R_eq))))
    k_silk = 1.6 * wb ** 0.52 * wm ** 0.73 * (1.0 + (10.4 * wm) ** -0.95)   # eq. 7
    return dict(z_eq=z_eq, k_eq=k_eq, z_d=z_d, R_d=R_d, R_eq=R_eq, s=s, k_silk=k_silk)


def eh98_full_transfer(k_mpc, cosmo):
    """Full EH98 transfer function with baryon acoustic oscillations (eq. 16)."""
    om, ob, h = cosmo["omega_m"], cosmo["omega_b"], cosmo["h"]
    wm = om * h * h
    fb = ob / om
    fc = 1.0 - fb
    sc = eh98_scales(cosmo)
    k = np.asarray(k_mpc, dtype=np.float64)
    s, k_eq = sc["s"], sc["k_eq"]
    q = k / (13.41 * k_eq)                                         # eq. 10
    a1 = (46.9 * wm) ** 0.670 * (1.0 + (32.1 * wm) ** -0.532)      # eq. 11
    a2 = (12.0 * wm) ** 0.424 * (1.0 + (45.0 * wm) ** -0.582)
    alpha_c = a1 ** (-fb) * a2 ** (-fb ** 3)
    bb1 = 0.944 / (1.0 + (458.0 * wm) ** -0.708)                   # eq. 12
    bb2 = (0.395 * wm) ** -0.0266
    beta_c = 1.0 / (1.0 + bb1 * (fc ** bb2 - 1.0))

    def t0(ac, bc):                                                # eqs. 19-20
        L = np.log(math.e + 1.8 * bc * q)
        C = 14.2 / ac + 386.0 / (1.0 + 69.9 * q ** 1.08)
        return L / (L + C * q * q)

    f = 1.0 / (1.0 + (k * s / 5.4) ** 4)                           # eq. 18
    T_c = f * t0(1.0, beta_c) + (1.0 - f) * t0(alpha_c, beta_c)    # eq. 17

    y = (1.0 + sc["z_eq"]) / (1.0 + sc["z_d"])
    G = y * (-6.0 * math.sqrt(1.0 + y) + (2.0 + 3.0 * y)           # eq. 15
             * math.log((math.sqrt(1.0 + y) + 1.0) / (math.sqrt(1.0 + y) - 1.0)))
    alpha_b = 2.07 * k_eq * s * (1.0 + sc["R_d"]) ** -0.75 * G     # eq. 14
    beta_node = 8.41 * wm ** 0.435                                 # eq. 23
    beta_b = 0.5 + fb + (3.0 - 2.0 * fb) * math.sqrt((17.2 * wm) ** 2 + 1.0)   # eq. 24
    ks = k * s
    s_tilde = s / (1.0 + (beta_node / ks) ** 3) ** (1.0 / 3.0)     # eq. 22
    x = k * s_tilde
    j0 = np.where(x > 1e-8, np.sin(x) / np.where(x > 1e-8, x, 1.0), 1.0)
    T_b = (t0(1.0, 1.0) / (1.0 + (ks / 5.2) ** 2)                  # eq. 21
           + alpha_b / (1.0 + (beta_b / ks) ** 3) * np.exp(-(k / sc["k_silk"]) ** 1.4)) * j0
    return fb * T_b + fc * T_c                                     # eq. 16


# --------------------------------------------------------------------------
# the oracle's s and alpha_Gamma, recovered from its T(k) alone
# --------------------------------------------------------------------------
def _q_of_T(T):
    """Invert T = L0 / (L0 + C0 q^2) (eq. 29) for q; T is decreasing in q."""
    def f(lq):
        q = math.exp(lq)
        L0 = math.log(2.0 * math.e + 1.8 * q)
        C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
        return L0 / (L0 + C0 * q * q) - T
    return math.exp(brentq(f, math.log(1e-8), math.log(1e8), xtol=1e-15, rtol=1e-15))


def recovered_shape(T_nw, cosmo):
    """Gamma_eff(k) / (Om h) of a no-wiggle T (eq. 28: q = k Theta^2 / Gamma_eff,
    k in h/Mpc), then alpha_Gamma from its small-scale limit and s from
    Gamma_eff = Om h [alpha + (1 - alpha) / (1 + (0.43 k s)^4)] (eq. 30) at a
    wavenumber in the cross-over."""
    om, h = cosmo["omega_m"], cosmo["h"]
    th2 = (cosmo["t_cmb"] / 2.7) ** 2

    def g(k_h):
        T = float(T_nw(np.array([k_h]), cosmo)[0])
        return k_h * th2 / _q_of_T(T) / (om * h)

    alpha = g(30.0)                                    # (0.43 k s)^4 ~ 1e12 here
    k_h = 1.0 / (0.43 * 150.0 * h)                      # (0.43 k s)^4 ~ 1 for s ~ 150 Mpc
    gm = g(k_h)
    s = ((1.0 - alpha) / (gm - alpha) - 1.0) ** 0.25 / (0.43 * k_h * h)
    return alpha, s


def bao_period_means(T_nw, cosmo, k_lo=0.01, k_hi=0.4):
    """Mean of T_full / T_nw over consecutive whole acoustic periods
    (Delta k = 2 pi / s) between k_lo and k_hi h/Mpc: the oscillation
    averages out and the no-wiggle form should sit on the midpoints."""
    h = cosmo["h"]
    s = eh98_scales(cosmo)["s"]
    per = 2.0 * math.pi / s / h                        # period in h/Mpc
    means = []
    k0 = k_lo
    while k0 + per <= k_hi:
        k = np.linspace(k0, k0 + per, 401)
        r = eh98_full_transfer(k * h, cosmo) / T_nw(k, cosmo)
        w = np.ones_like(k)
        w[0] = w[-1] = 0.5
        means.append(float(np.sum(w * r) / np.sum(w)))
        k0 += per
    return np.array(means)


def small_scale_ratio(T_nw, cosmo, k=(0.5, 1.0, 2.0, 5.0, 10.0)):
    """T_full / T_nw where the oscillations are Silk-damped (k in h/Mpc)."""
    k = np.asarray(k, dtype=np.float64)
    return eh98_full_transfer(k * cosmo["h"], cosmo) / T_nw(k, cosmo)


COSMOS = [
    COSMO,
    dict(COSMO, omega_m=0.25, omega_b=0.04),
    dict(COSMO, omega_m=0.35, omega_b=0.055, h=0.72),
]


# --------------------------------------------------------------------------
# sanity of the independent EH98 scales themselves
# --------------------------------------------------------------------------
def test_eh98_scales_are_physical():
    sc = eh98_scales(COSMO)
    # matter-radiation equality and the drag epoch of a Planck-like universe
    assert 3000 < sc["z_eq"] < 3800
    assert 950 < sc["z_d"] < 1100
    assert 140 < sc["s"] < 160                       # Mpc
    # eq. 6 is the closed form of the integral of the sound speed
    # c_s = 1 / sqrt(3 (1 + R)) over conformal time up to z_d (radiation +
    # matter background, R propto a): integrate it numerically
    from scipy.integrate import quad
    om, h = COSMO["omega_m"], COSMO["h"]
    th = COSMO["t_cmb"] / 2.7
    wm = om * h * h
    a_eq = 1.0 / (1.0 + sc["z_eq"])
    R_eq = sc["R_eq"]
    a_d = a_eq * sc["R_d"] / R_eq                     # R propto a: R(a_d) = R_d
    # conformal time d eta = da / (a^2 H), H^2 = H_eq^2/2 [(a_eq/a)^3 + (a_eq/a)^4];
    # k_eq = a_eq H_eq (the EH98 definition) fixes H_eq
    H_eq = sc["k_eq"] / a_eq                          # 1/Mpc (c = 1)

    def integrand(a):
        H = H_eq * math.sqrt(0.5 * ((a_eq / a) ** 3 + (a_eq / a) ** 4))
        R = R_eq * a / a_eq
        return 1.0 / (a * a * H) / math.sqrt(3.0 * (1.0 + R))
    s_num, _ = quad(integrand, 0.0, a_d, epsrel=1e-12, limit=400)
    assert abs(s_num / sc["s"] - 1) < 1e-6
    # the full transfer function: unity at large scales, decreasing envelope
    assert abs(float(eh98_full_transfer(np.array([1e-6]), COSMO)[0]) - 1) < 1e-5


@pytest.mark.parametrize("cosmo", COSMOS)
def test_nowiggle_sound_horizon_matches_physical(cosmo):
    """Eq. 26's s, recovered from the oracle's T(k), within EH98's stated
    ~2% of the physical sound horizon of eq. 6."""
    alpha, s = recovered_shape(O.eh_nowiggle_transfer, cosmo)
    assert 0.0 < alpha < 1.0
    assert abs(s / eh98_scales(cosmo)["s"] - 1) < 0.02, s


@pytest.mark.parametrize("cosmo", COSMOS)
def test_nowiggle_tracks_full_transfer_function(cosmo):
    """On acoustic scales the no-wiggle T passes through the middle of the
    full EH98 oscillations (period means within 1.5%); on Silk-damped scales
    it reproduces the full function's baryon suppression within 2%."""
    means = bao_period_means(O.eh_nowiggle_transfer, cosmo)
    assert len(means) >= 3
    assert np.max(np.abs(means - 1)) < 0.015, means
    r = small_scale_ratio(O.eh_nowiggle_transfer, cosmo)
    assert np.max(np.abs(r - 1)) < 0.02, r
