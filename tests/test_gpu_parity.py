"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: cell keys and sort order bit-exact; density and force relative
L2 <= 1e-5; positions and momenta after a 5-step run <= 1e-4; binned P(k)
within 0.1 % below k_Nyq/2; linear field and 2LPT relative L2 <= 1e-5.
"""
import math

import numpy as np
import pytest

from oracle import fpm_oracle as O
from paper_2010_11847_gb300 import inputs

pytestmark = pytest.mark.gpu

COSMO = dict(inputs.COSMO_DEFAULT)


def rel_l2(a, b):
    dt = np.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else np.float64
    a = np.asarray(a, dtype=dt)
    b = np.asarray(b, dtype=dt)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_mod(cuda):
    import torch
    return torch


def make_plan(np_, nc, box=100.0, cosmo=COSMO):
    from paper_2010_11847_gb300.binding import Plan
    return Plan(np_, nc, box, cosmo)


def to_dev(x, torch):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def lin_k_to_numpy(lin_k):
    return lin_k.permute(0, 2, 1).contiguous().cpu().numpy()


def numpy_to_lin_k(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a.transpose(0, 2, 1)).astype(np.complex64)).cuda()


# ------------------------------------------------------------------ growth
def test_growth_matches_oracle(torch_mod):
    pl = make_plan(32, 32)
    a = np.array([0.1, 0.1 + 0.9 / 5, 0.37, 0.8, 1.0])
    g = pl.growth(a)
    ref = O.growth(a, COSMO["omega_m"])
    for j, k in enumerate(("D1", "D2", "f1", "f2", "E")):
        np.testing.assert_allclose(g[:, j], ref[k], rtol=2e-8)


# ------------------------------------------------------------------ FFT + force
@pytest.mark.parametrize("nc", [16, 32, 48, 96, 128, 192, 256])
def test_force_matches_oracle(torch_mod, nc):
    torch = torch_mod
    pl = make_plan(nc // 2 if nc in (32, 64, 96, 128, 192, 256) else nc, nc)
    rho = (1.0 + 0.5 * inputs.random_field(nc, 100 + nc)).astype(np.float32)
    F = pl.force(to_dev(rho, torch)).cpu().numpy()
    ref = O.force(rho.astype(np.float64), COSMO["omega_m"])
    for d in range(3):
        assert rel_l2(F[d], ref[d]) < 1e-5, (d, rel_l2(F[d], ref[d]))


def test_force_plane_wave_closed_form(torch_mod):
    torch = torch_mod
    n, j, A = 64, 5, 0.3
    pl = make_plan(n, n)
    w = 2 * math.pi * j / n
    x = np.arange(n)
    rho = (1 + A * np.cos(w * x))[None, :, None] * np.ones((n, n, n))
    F = pl.force(to_dev(rho.astype(np.float32), torch)).cpu().numpy()
    g = (8 * math.sin(w) - math.sin(2 * w)) / 6
    expect = -1.5 * COSMO["omega_m"] * A * g / w ** 2 * np.sin(w * x)[None, :, None]
    assert np.abs(F[1] - expect).max() < 1e-5 * np.abs(expect).max()
    assert np.abs(F[0]).max() < 1e-6 and np.abs(F[2]).max() < 1e-6


# ------------------------------------------------------------------ paint / sort
PAINT_CASES = [(16, 16, 3.0), (32, 32, 2.5), (32, 64, 6.0), (48, 96, 4.0), (64, 64, 10.0), (64, 256, 20.0)]


@pytest.mark.parametrize("np_,nc,scale", PAINT_CASES)
def test_paint_keys_perm_match_oracle(torch_mod, np_, nc, scale):
    torch = torch_mod
    pl = make_plan(np_, nc)
    dx = inputs.random_displacements(np_, scale, 7 + np_ + nc)
    rho, keys, perm = pl.paint(to_dev(dx, torch), keys=True, perm=True)
    torch.cuda.synchronize()
    assert pl.status() == 0
    rho = rho.cpu().numpy()
    ref = O.paint(dx, np_, nc)
    assert rel_l2(rho, ref) < 1e-5
    assert abs(rho.astype(np.float64).sum() / nc ** 3 - 1) < 1e-6
    cell, _ = O.cic_cells(dx, np_, nc)
    ref_keys = O.cell_keys(cell, nc)
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint32), ref_keys)
    np.testing.assert_array_equal(perm.cpu().numpy().view(np.uint32), O.sort_order(ref_keys))


def test_paint_is_deterministic_and_unperturbed_lattice_is_uniform(torch_mod):
    torch = torch_mod
    pl = make_plan(64, 64)
    dx = to_dev(inputs.random_displacements(64, 5.0, 3), torch)
    r1 = pl.paint(dx).cpu().numpy()
    r2 = pl.paint(dx).cpu().numpy()
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))
    z = torch.zeros(3, 64 ** 3, device="cuda")
    assert np.all(pl.paint(z).cpu().numpy() == 1.0)
    pl2 = make_plan(32, 64)
    r = pl2.paint(torch.zeros(3, 32 ** 3, device="cuda")).cpu().numpy()
    assert np.all(r[::2, ::2, ::2] == 8.0) and r.sum() == 64 ** 3


def test_paint_oversized_tile_path(torch_mod):
    """All particles in one 16^3 tile (more than fit the shared-memory sort)."""
    torch = torch_mod
    np_, nc = 32, 32
    pl = make_plan(np_, nc)
    rng = np.random.default_rng(5)
    lat = O.lattice(np_, nc).astype(np.float64)
    target = rng.uniform(0.0, 15.999, size=(3, np_ ** 3))
    dx = (target - lat).astype(np.float32)
    rho, keys, perm = pl.paint(to_dev(dx, torch), keys=True, perm=True)
    ref = O.paint(dx, np_, nc)
    assert rel_l2(rho.cpu().numpy(), ref) < 1e-5
    cell, _ = O.cic_cells(dx, np_, nc)
    ref_keys = O.cell_keys(cell, nc)
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint32), ref_keys)
    np.testing.assert_array_equal(perm.cpu().numpy().view(np.uint32), O.sort_order(ref_keys))


def test_paint_dense_clumps_hot_path(torch_mod):
    """The hot-path paint (no permutation) with every particle in one of five
    tight clumps: thousands of particles per cell, so warps hold long runs
    of one cell (merged before the atomics) and the cell sums overflow the
    low 32-bit word into its carry."""
    torch = torch_mod
    np_, nc = 32, 32
    pl = make_plan(np_, nc)
    rng = np.random.default_rng(15)
    centres = np.array([[3, 4, 5], [3, 4, 6], [20, 9, 30], [31, 31, 31], [16, 0, 8]], dtype=np.float64)
    pick = rng.integers(0, len(centres), size=np_ ** 3)
    target = centres[pick].T + rng.uniform(0.0, 0.3, size=(3, np_ ** 3))
    dx = (target - O.lattice(np_, nc)).astype(np.float32)
    d = to_dev(dx, torch)
    rho = pl.paint(d)
    again = pl.paint(d)
    torch.cuda.synchronize()
    assert pl.status() == 0
    assert torch.equal(rho, again)
    ref = O.paint(dx, np_, nc)
    assert ref.max() > 300.0                   # > 256 particles' worth of weight in a cell
    assert rel_l2(rho.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("np_,nc", [(32, 32), (32, 64), (64, 128)])
def test_readout_matches_oracle(torch_mod, np_, nc):
    torch = torch_mod
    pl = make_plan(np_, nc)
    dx = inputs.random_displacements(np_, 4.0, 11)
    F = np.stack([inputs.random_field(nc, 20 + d) for d in range(3)])
    f = pl.readout(to_dev(F, torch), to_dev(dx, torch)).cpu().numpy()
    ref = O.readout(F.astype(np.float64), dx, np_, nc)
    assert rel_l2(f, ref) < 1e-6


def test_paint_readout_adjointness_on_gpu(torch_mod):
    torch = torch_mod
    np_, nc = 64, 64
    pl = make_plan(np_, nc)
    dx = to_dev(inputs.random_displacements(np_, 6.0, 13), torch)
    F = inputs.random_field(nc, 5)
    rho = pl.paint(dx).cpu().numpy().astype(np.float64)
    f = pl.readout(to_dev(np.stack([F, F, F]), torch), dx).cpu().numpy().astype(np.float64)
    lhs = float((rho * F).sum())
    rhs = float(f[0].sum())
    assert abs(lhs - rhs) < 1e-6 * np.abs(rho * F).sum()


# ------------------------------------------------------------------ IC
@pytest.mark.parametrize("np_,box", [(32, 100.0), (96, 300.0), (128, 400.0)])
def test_linear_field_matches_oracle(torch_mod, np_, box):
    torch = torch_mod
    pl = make_plan(np_, np_, box)
    w = inputs.white_noise(np_, 21)
    lk = lin_k_to_numpy(pl.linear_field(to_dev(w, torch)))
    ref = O.linear_field(w, box, COSMO)
    assert rel_l2(lk, ref) < 1e-5


@pytest.mark.parametrize("np_,nc,order", [(32, 32, 2), (32, 64, 2), (48, 48, 1), (128, 128, 2)])
def test_lpt_matches_oracle(torch_mod, np_, nc, order):
    torch = torch_mod
    box = 100.0 * np_ / 32
    pl = make_plan(np_, nc, box)
    w = inputs.white_noise(np_, 33)
    ref_lk = O.linear_field(w, box, COSMO)
    dx, p = pl.lpt(numpy_to_lin_k(ref_lk, torch), 0.1, order)
    rdx, rp = O.lpt(ref_lk, nc, 0.1, COSMO, order=order)
    assert rel_l2(dx.cpu().numpy(), rdx) < 1e-5
    assert rel_l2(p.cpu().numpy(), rp) < 1e-5


# ------------------------------------------------------------------ full runs
def _run_both(wl, torch):
    w = inputs.white_noise(wl.np_, wl.seed)
    stages = wl.stages()
    pl = make_plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    dx, p, _ = pl.simulate(to_dev(w, torch), stages)
    rho = pl.paint(dx)
    k, pk, _ = pl.power(rho - 1.0)
    torch.cuda.synchronize()
    assert pl.status() == 0
    ref = O.simulate(w, wl.nc, wl.box, wl.cosmo, stages)
    return dict(dx=dx.cpu().numpy(), p=p.cpu().numpy(), rho=rho.cpu().numpy(), pk=pk), ref


def test_small_config_end_to_end(torch_mod):
    """32^3 particles on 32^3, 100 Mpc/h, 2LPT at a=0.1 + 5 KDK steps."""
    got, ref = _run_both(inputs.SMALL, torch_mod)
    assert rel_l2(got["dx"], ref["dx"]) < 1e-4
    assert rel_l2(got["p"], ref["p"]) < 1e-4
    assert rel_l2(got["rho"], ref["rho"]) < 1e-4
    nb = inputs.SMALL.nc // 4          # k < k_Nyq / 2
    np.testing.assert_allclose(got["pk"][:nb], ref["pk"][:nb], rtol=1e-3)


def test_medium_config_end_to_end(torch_mod):
    """128^3 particles on 256^3, 400 Mpc/h, 10 KDK steps."""
    got, ref = _run_both(inputs.MEDIUM, torch_mod)
    assert rel_l2(got["dx"], ref["dx"]) < 1e-4
    assert rel_l2(got["p"], ref["p"]) < 1e-4
    assert rel_l2(got["rho"], ref["rho"]) < 1e-4
    nb = inputs.MEDIUM.nc // 4
    np.testing.assert_allclose(got["pk"][:nb], ref["pk"][:nb], rtol=1e-3)


def test_single_step_density_and_force_match_oracle(torch_mod):
    """One step from oracle ICs: identical float32 positions on both sides."""
    torch = torch_mod
    wl = inputs.MEDIUM
    w = inputs.white_noise(wl.np_, 3)
    lk = O.linear_field(w, wl.box, wl.cosmo)
    dx0, _ = O.lpt(lk, wl.nc, 0.1, wl.cosmo)
    dx32 = dx0.astype(np.float32)
    pl = make_plan(wl.np_, wl.nc, wl.box, wl.cosmo)
    rho = pl.paint(to_dev(dx32, torch))
    F = pl.force(rho)
    ref_rho = O.paint(dx32, wl.np_, wl.nc)
    ref_F = O.force(ref_rho, wl.cosmo["omega_m"])
    assert rel_l2(rho.cpu().numpy(), ref_rho) < 1e-5
    assert rel_l2(F.cpu().numpy(), ref_F) < 1e-5
    f = pl.readout(F, to_dev(dx32, torch)).cpu().numpy()
    ref_f = O.readout(ref_F, dx32, wl.np_, wl.nc)
    assert rel_l2(f, ref_f) < 1e-5


def test_nan_input_sets_device_flag(torch_mod):
    torch = torch_mod
    pl = make_plan(32, 32)
    dx = torch.zeros(3, 32 ** 3, device="cuda")
    dx[1, 100] = float("nan")
    pl.paint(dx)
    assert pl.status() == -5
    assert pl.status() == 0          # the flag clears after it is read


def test_zero_steps_is_a_no_op(torch_mod):
    torch = torch_mod
    pl = make_plan(32, 32)
    dx = to_dev(inputs.random_displacements(32, 1.0, 2), torch)
    p = dx.clone()
    d0 = dx.clone()
    pl.kdk(dx, p, np.array([0.5]))
    assert torch.equal(dx, d0)
