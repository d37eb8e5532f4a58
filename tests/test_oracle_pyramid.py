"""Pins of the oracle's multi-grid pyramid force (Sec. 3.1 Eqs. 6-9,
Algorithms 2-3): REDUCE and EXPAND against brute-force loops, the B-spline's
closed-form symbol and the transpose identity of Algorithm 2's kernels; the
local-FFT force against the plain force where the padded blocks wrap the
whole mesh and against translation by a block; the whole scheme against the
Ewald pair force and the plain force of a cosmological density.
"""
import math

import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs
from test_oracle_pins import OM, _ewald_force

COSMO = dict(inputs.COSMO_DEFAULT)


def _w(t):
    """Order-6 discrete B-spline weight at integer offset t (binomial row 6)."""
    return math.comb(6, t + 3) / 64.0 if -3 <= t <= 3 else 0.0


def test_bspline_kernel_is_the_binomial_row():
    np.testing.assert_allclose(O.bspline_kernel(6), [math.comb(6, j) / 64 for j in range(7)], rtol=0, atol=1e-16)
    assert abs(O.bspline_kernel(6).sum() - 1.0) < 1e-15


def test_reduce_once_by_brute_force():
    n = 8
    h = np.random.default_rng(1).normal(size=(n, n, n))
    got = O.reduce_once(h)
    for i in range(n // 2):
        for j in range(n // 2):
            for k in range(n // 2):
                acc = 0.0
                for a in range(-3, 4):
                    for b in range(-3, 4):
                        for c in range(-3, 4):
                            acc += _w(a) * _w(b) * _w(c) * h[(2 * i + a) % n, (2 * j + b) % n, (2 * k + c) % n]
                assert abs(got[i, j, k] - acc) < 1e-13


def test_expand_once_by_brute_force():
    m = 4
    d = np.random.default_rng(2).normal(size=(m, m, m))
    got = O.expand_once(d)
    n = 2 * m
    for x in range(n):
        for y in range(n):
            for z in range(n):
                acc = 0.0
                for i in range(m):
                    for j in range(m):
                        for k in range(m):
                            # periodic offsets between fine node x and coarse node i (at fine 2i)
                            tx = min(((x - 2 * i) % n, (x - 2 * i) % n - n), key=abs)
                            ty = min(((y - 2 * j) % n, (y - 2 * j) % n - n), key=abs)
                            tz = min(((z - 2 * k) % n, (z - 2 * k) % n - n), key=abs)
                            acc += 8.0 * _w(tx) * _w(ty) * _w(tz) * d[i, j, k]
                assert abs(got[x, y, z] - acc) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reduce_of_a_plane_wave_is_scaled_by_the_bspline_symbol(axis):
    """S[G * cos(w x)] = cos(w/2)^6 cos(2 w i): the binomial filter's symbol."""
    n, kk = 32, 5
    w = 2 * math.pi * kk / n
    x = np.indices((n, n, n))[axis].astype(np.float64)
    got = O.reduce_once(np.cos(w * x + 0.3))
    xi = np.indices((n // 2,) * 3)[axis].astype(np.float64)
    np.testing.assert_allclose(got, math.cos(w / 2) ** 6 * np.cos(2 * w * xi + 0.3), atol=1e-13)


def test_expand_is_eight_times_the_transpose_of_reduce():
    """Algorithm 2: EXPAND's kernel is the B-spline times 8, so EXPAND = 8 REDUCE^T."""
    r = np.random.default_rng(3)
    u = r.normal(size=(16, 16, 16))
    v = r.normal(size=(8, 8, 8))
    lhs = float((O.reduce_once(u) * v).sum())
    rhs = float((u * O.expand_once(v)).sum()) / 8.0
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_reduce_and_expand_keep_constants():
    np.testing.assert_allclose(O.reduce(np.full((16, 16, 16), 2.5), 2), 2.5, rtol=1e-15)
    np.testing.assert_allclose(O.expand(np.full((4, 4, 4), -1.5), 2), -1.5, rtol=1e-15)


@pytest.mark.parametrize("split,halo", [(1, 0), (2, 4)])
def test_local_force_with_blocks_wrapping_the_mesh_is_the_plain_force(split, halo):
    """A padded block of n cells is the whole periodic mesh, shifted: its
    periodic force is the plain force."""
    n = 16
    rho = 1.0 + 0.3 * inputs.random_field(n, 4).astype(np.float64)
    np.testing.assert_allclose(O.local_force(rho, OM, split, halo), O.force(rho, OM), atol=1e-13)


def test_local_force_is_covariant_under_translation_by_a_block():
    """The block grid is invariant under shifts by the block size m (not by
    one cell): shifting the density by m shifts the local force by m."""
    n, split, halo = 24, 3, 4
    m = n // split
    rho = 1.0 + 0.3 * np.random.default_rng(5).normal(size=(n, n, n))
    F = O.local_force(rho, OM, split, halo)
    for ax in range(3):
        Fs = O.local_force(np.roll(rho, m, axis=ax), OM, split, halo)
        np.testing.assert_allclose(Fs, np.roll(F, m, axis=ax + 1), atol=1e-12)
    F1 = O.local_force(np.roll(rho, 1, axis=0), OM, split, halo)
    assert np.abs(F1 - np.roll(F, 1, axis=1)).max() > 1e-3      # not covariant by one cell


READINGS = [("block", "matched"), ("global", "coarse")]


@pytest.mark.parametrize("reading", READINGS)
@pytest.mark.parametrize("sep", [8.6, 12.1])
def test_pyramid_pair_force_matches_ewald(sep, reading):
    """Two levels, 2^3 blocks with a 16-cell halo on 64^3: the pair force is
    within 5% of the periodic Ewald force (a missing 2^levels factor, a
    wrong sign of the band correction or an off-centre kernel is not)."""
    nc = 64
    for trial in range(3):
        rng = np.random.default_rng(int(sep * 10) + 1000 * trial)
        x1 = np.array([10.3, 20.7, 5.45]) + rng.uniform(0, 1, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.stack([x1, x1 + sep * u], 1)
        cell = np.floor(pos).astype(np.int64) % nc
        t = pos - np.floor(pos)
        rho = O.paint_cells(cell, t, np.array([1.0, 1.0]), nc) + 1.0 - 2.0 / nc ** 3
        F = O.pyramid_force(rho, OM, 2, 2, 16, bandpass=reading[0], coarse_kernel=reading[1])
        f = O.readout_cells(F, cell, t)
        ref = _ewald_force(pos[:, 0] - pos[:, 1], nc, 1.0, OM)
        assert np.linalg.norm(f[:, 0] - ref) / np.linalg.norm(ref) < 0.05


def _cosmological_density(n=64, box=200.0):
    lk = O.linear_field(inputs.white_noise(n, 3), box, COSMO)
    dx, _ = O.lpt(lk, n, 1.0, COSMO, order=1)
    return O.paint(dx.astype(np.float32), n, n)


def test_pyramid_force_of_a_cosmological_density_is_close_to_the_plain_force():
    """1LPT density at a = 1 in a 200 Mpc/h box on 64^3, relative L2 of the
    pyramid force against the plain force.  Band-pass on the assembled
    short-range mesh with coarse-cell kernels: below 2% with the paper's
    16-cell halo, a halo of 8 cells clearly worse.  Band-pass on each padded
    block with the fine mesh's kernels on the coarse mesh: below 0.3% with a
    16-cell halo and below 0.6% with 8 (the halo then matters only
    marginally, as the paper reports)."""
    rho = _cosmological_density()
    Fp = O.force(rho, OM)
    rel = lambda F: np.linalg.norm(F - Fp) / np.linalg.norm(Fp)
    r16 = rel(O.pyramid_force(rho, OM, 2, 2, 16, bandpass="global", coarse_kernel="coarse"))
    r8 = rel(O.pyramid_force(rho, OM, 2, 2, 8, bandpass="global", coarse_kernel="coarse"))
    assert r16 < 0.02 and r8 > 2 * r16, (r16, r8)
    b16 = rel(O.pyramid_force(rho, OM, 2, 2, 16))
    b8 = rel(O.pyramid_force(rho, OM, 2, 2, 8))
    assert b16 < 3e-3 and b8 < 6e-3, (b16, b8)


def test_matched_coarse_force_commutes_with_reduce():
    """For a field whose modes lie below the coarse Nyquist frequency (no
    aliasing in REDUCE), the coarse force with the fine mesh's kernel of a
    REDUCEd density equals the REDUCEd fine force exactly; the coarse-cell
    kernel does not (Eq. 5's difference is coarser there)."""
    n, levels = 32, 2
    x = np.arange(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    delta = np.zeros((n, n, n))
    rng = np.random.default_rng(21)
    for (a, b, c) in [(1, 0, 0), (0, 2, 1), (3, 1, 2), (1, 3, 3), (2, 2, 0)]:
        delta += rng.normal() * np.cos(2 * np.pi * (a * X + b * Y + c * Z) / n + rng.uniform(0, 6.28))
    Ff = O.force_from_delta(delta, OM)
    lhs = O.coarse_force(O.reduce(delta, levels), OM, 2.0 ** levels, "matched")
    rhs = np.stack([O.reduce(Ff[i], levels) for i in range(3)])
    np.testing.assert_allclose(lhs, rhs, atol=1e-12 * np.abs(rhs).max())
    coarse = O.coarse_force(O.reduce(delta, levels), OM, 2.0 ** levels, "coarse")
    assert np.abs(coarse - rhs).max() > 0.05 * np.abs(rhs).max()


def test_block_bandpass_is_the_global_one_for_a_single_unpadded_block():
    """One block without halo is the whole periodic mesh: band-passing the
    block or the assembled mesh is the same operation."""
    n = 32
    rho = 1.0 + 0.3 * np.random.default_rng(8).normal(size=(n, n, n))
    for kernel in ("matched", "coarse"):
        a = O.pyramid_force(rho, OM, 2, 1, 0, bandpass="block", coarse_kernel=kernel)
        b = O.pyramid_force(rho, OM, 2, 1, 0, bandpass="global", coarse_kernel=kernel)
        np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(b).max())
